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


def test_mad_on_nonblocking_stream_returns_complete_result():
    """gfe_mad returns once the product is complete on the caller's stream,
    also when that stream does not synchronise with the legacy stream: its
    status word is read by a copy on that stream."""
    L = gfe.lib()
    p, m, n, k = 7, 2048, 3072, 4096
    A = synth.uniform_u8(m, k, p, 40, 1).to("cuda:0")
    B = synth.uniform_u8(k, n, p, 40, 2).to("cuda:0")
    side = torch.cuda.Stream()
    ws = torch.empty(L.gfe_mad_workspace(p, m, n, k), dtype=torch.uint8, device="cuda:0")
    C = torch.full((m, n), 255, dtype=torch.uint8, device="cuda:0")
    torch.cuda.synchronize()
    st = L.gfe_mad(p, m, n, k, None, 0, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, 0, ws.data_ptr(),
                   ws.numel(), side.cuda_stream)
    assert st == 0, L.gfe_last_error()
    got = C.cpu().numpy()  # a copy on the legacy stream, not ordered after `side`
    # float64 products of integers below 2^53 are exact (and use BLAS)
    exact = (A.cpu().numpy().astype(np.float64) @ B.cpu().numpy().astype(np.float64)).astype(np.int64) % p
    assert np.array_equal(got, exact)


def test_concurrent_calls_keep_their_own_status():
    """Each call owns its error word: echelon calls running on their own
    streams beside bounded-wait self-tests that give up (each setting an
    error word of its own) all return GFE_OK and exact results."""
    import threading
    A = synth.matrix(7, 1500, 1200, seed=3)
    ref = O.echelon(A.numpy(), 7)
    Ad = A.to("cuda:0")
    errs, stop = [], threading.Event()

    def selftests():
        s = torch.cuda.Stream()
        while not stop.is_set():
            if gfe.lib().gfe_selftest_wait_timeout(2000, s.cuda_stream) != 3:
                errs.append("self-test did not give up")

    def worker():
        s = torch.cuda.Stream()
        try:
            with torch.cuda.stream(s):
                for _ in range(3):
                    got = gfe.echelon(Ad, 7)
                    s.synchronize()
                    if got["rank"] != ref["rank"] or not np.array_equal(got["R"].cpu().numpy(), ref["R"]):
                        errs.append("wrong result")
        except Exception as e:  # a status error surfaces as GfeError
            errs.append(repr(e))

    t0 = threading.Thread(target=selftests)
    ws = [threading.Thread(target=worker) for _ in range(2)]
    t0.start()
    for t in ws:
        t.start()
    for t in ws:
        t.join()
    stop.set()
    t0.join()
    assert not errs, errs[:3]
