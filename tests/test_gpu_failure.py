"""Failure detection without a GPU fault: a bounded device wait on a barrier
that nothing completes gives up, reports GFE_ETIMEOUT, and the context keeps
working (GPU)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    L = gfe.lib()
    st = L.gfe_selftest_wait_timeout(20000, torch.cuda.current_stream().cuda_stream)   # 20 ms
    assert st == 3, L.gfe_last_error()                                                 # GFE_ETIMEOUT
    assert b"gave up" in L.gfe_last_error()
    # the context is still usable and results are still exact
    A = synth.matrix(7, 200, 150, seed=1)
    got = gfe.echelon(A.to("cuda:0"), 7)
    ref = O.echelon(A.numpy(), 7)
    assert got["rank"] == ref["rank"] and np.array_equal(got["R"].cpu().numpy(), ref["R"])


def test_selftest_rejects_bad_limit():
    assert gfe.lib().gfe_selftest_wait_timeout(0, None) == 1
