"""gfe_mad_noalloc, the multiply-add entry point for callers that cannot
allocate device memory (a fixed device budget owned by the caller, or a path
where cudaMalloc / cudaFree could block or synchronise).  It is checked
through the C ABI against gfe_mad, the entry point that takes a workspace,
on two calls in a row (the scratch array is shared between calls and keeps
the previous call's contents).  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def call_noalloc(L, p, W, A, B, C, stream):
    m, k = A.shape
    n = B.shape[1]
    return L.gfe_mad_noalloc(p, m, n, k, W.data_ptr() if W is not None else None, W.stride(0) if W is not None else 0,
                             A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(), C.stride(0), 0,
                             stream)


def test_mad_noalloc_matches_mad_on_two_calls():
    L = gfe.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(7, 300, 500, 700, True), (251, 129, 257, 1500, False), (2, 64, 1000, 200, True)]
    for i, (p, m, n, k, with_w) in enumerate(cases[:2] + cases[2:]):
        A = synth.uniform_u8(m, k, p, 10 + i, 1).to(DEV)
        B = synth.uniform_u8(k, n, p, 10 + i, 2).to(DEV)
        W = synth.uniform_u8(m, n, p, 10 + i, 0).to(DEV) if with_w else None
        C = torch.full((m, n), 255, dtype=torch.uint8, device=DEV)
        st = call_noalloc(L, p, W, A, B, C, stream)
        assert st == 0, L.gfe_last_error()
        ref = gfe.mad(W, A, B, p)
        torch.cuda.synchronize()
        assert torch.equal(C, ref), (p, m, n, k)
        exact = (A.cpu().numpy().astype(np.int64) @ B.cpu().numpy().astype(np.int64))
        if with_w:
            exact = exact + W.cpu().numpy().astype(np.int64)
        assert np.array_equal(C.cpu().numpy(), exact % p)


def test_mad_noalloc_second_call_allocates_nothing():
    """The first call on a device loads the library's device code and with it
    the 32 MiB array; a later call must leave free device memory unchanged,
    on the default stream and on a non-blocking one."""
    L = gfe.lib()
    p, m, n, k = 5, 256, 384, 512
    A = synth.uniform_u8(m, k, p, 30, 1).to(DEV)
    B = synth.uniform_u8(k, n, p, 30, 2).to(DEV)
    C = torch.empty((m, n), dtype=torch.uint8, device=DEV)
    assert call_noalloc(L, p, None, A, B, C, torch.cuda.current_stream().cuda_stream) == 0, L.gfe_last_error()
    torch.cuda.synchronize()
    exact = (A.cpu().numpy().astype(np.int64) @ B.cpu().numpy().astype(np.int64)) % p
    side = torch.cuda.Stream()  # non-blocking with respect to the legacy stream
    free0 = torch.cuda.mem_get_info()[0]
    for s in (torch.cuda.current_stream(), side):
        C.fill_(255)
        torch.cuda.synchronize()
        assert call_noalloc(L, p, None, A, B, C, s.cuda_stream) == 0, L.gfe_last_error()
        # the call returns once the product is complete on its stream
        assert np.array_equal(C.cpu().numpy(), exact)
    assert torch.cuda.mem_get_info()[0] == free0


def test_mad_noalloc_checks_p_first():
    L = gfe.lib()
    for p in (1, 4, 257):
        assert L.gfe_mad_noalloc(p, 0, 0, 0, None, 0, None, 0, None, 0, None, 0, 0, None) == 1
        assert b"prime" in L.gfe_last_error()


def test_mad_noalloc_rejects_oversize():
    L = gfe.lib()
    cap = L.gfe_mad_noalloc_max_bytes()
    assert cap == 32 << 20
    m = n = k = 4096  # GF(3) is e4m3 inside: 3 x 16 MiB of scratch, more than the array holds
    assert L.gfe_mad_workspace(3, m, n, k) > cap
    A = torch.zeros((m, k), dtype=torch.uint8, device=DEV)
    C = torch.zeros((m, n), dtype=torch.uint8, device=DEV)
    st = L.gfe_mad_noalloc(3, m, n, k, None, 0, A.data_ptr(), k, A.data_ptr(), n, C.data_ptr(), n, 0,
                           torch.cuda.current_stream().cuda_stream)
    assert st == 1
    assert b"more than the fixed" in L.gfe_last_error()
