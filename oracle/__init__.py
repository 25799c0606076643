"""CPU oracle for exact echelonisation over GF(p) -- test infrastructure only."""
