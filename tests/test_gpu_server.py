"""The serving form: requests of mixed sizes and fields submitted while others
run; each result equals the same matrix echelonised alone (GPU)."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def requests(seed=0, count=16):
    rng = np.random.RandomState(seed)
    out = []
    for i in range(count):
        p = [2, 3, 7, 31, 251][i % 5]
        n = int(min(1500, 256 * (1 - rng.rand()) ** (-1 / 1.5)))   # Pareto(1.5) on [256, 1500]
        rank = int(0.6 * n) if i % 3 == 0 else None
        out.append((p, n, synth.matrix(p, n, n, seed=200 + i, rank=rank).to(DEV)))
    return out


def test_server_results_equal_alone():
    reqs = requests()
    one = max(gfe.query_workspace(A, p, n if p == 2 else None) for p, n, A in reqs)
    # cap: room for about two requests at once, so admission has to wait
    with gfe.Server(int(2.2 * one), workers=4) as srv:
        tickets = []
        for p, n, A in reqs:
            tickets.append(srv.submit(A, p, n if p == 2 else None))
            time.sleep(0.002)                              # arrivals spread over time
        got = [srv.wait(t) for t in tickets]
    for (p, n, A), g in zip(reqs, got):
        alone = gfe.echelon(A, p, n=n if p == 2 else None)
        assert g["rank"] == alone["rank"]
        for k in ("rho", "ups", "R", "M", "K"):
            assert torch.equal(g[k], alone[k]), (p, n, k)
        assert g["latency_us"] > 0


def test_server_small_requests_pass_a_large_one():
    """A large request waiting for memory does not block small ones that fit."""
    big = synth.matrix(7, 6000, 6000, seed=1).to(DEV)
    small = [synth.matrix(3, 300, 300, seed=10 + i).to(DEV) for i in range(6)]
    wbig = gfe.query_workspace(big, 7)
    wsmall = gfe.query_workspace(small[0], 3)
    with gfe.Server(wbig + 3 * wsmall, workers=3) as srv:
        tb = srv.submit(big, 7)
        ts = [srv.submit(A, 3) for A in small]
        rs = [srv.wait(t) for t in ts]
        rb = srv.wait(tb)
    assert max(r["latency_us"] for r in rs) < rb["latency_us"]
    ref = O.echelon(small[0].cpu().numpy(), 3)
    assert rs[0]["rank"] == ref["rank"] and np.array_equal(rs[0]["R"].cpu().numpy(), ref["R"])


def test_server_rejects_oversize_request():
    with gfe.Server(1 << 20, workers=1) as srv:
        A = synth.matrix(3, 2000, 2000, seed=1).to(DEV)
        with pytest.raises(gfe.GfeError):
            srv.submit(A, 3)


def test_server_groups_small_requests_into_one_launch():
    """A burst of small requests: a worker takes the queued ones together into
    the one-launch kernels, so the server makes far fewer echelonisation
    launches than requests (the per-request planner makes several leaves each);
    every result still equals the matrix echelonised alone."""
    fields = [2, 3, 7, 31, 251]
    reqs = [(p, 300, synth.matrix(p, 300, 300, seed=300 + i, rank=150 if i % 4 == 0 else None).to(DEV))
            for i, p in enumerate(fields * 8)]
    torch.cuda.synchronize()
    gfe.profile_enable(True, kinds=["other"])
    gfe.profile_read()
    gfe.lib().gfe_set_server_group_work(1e8)  # 300^3 is above the default
    try:
        with gfe.Server(8 << 30, workers=1) as srv:
            tickets = [srv.submit(A, p, n if p == 2 else None) for p, n, A in reqs]
            got = [srv.wait(t) for t in tickets]
        launches = gfe.profile_read()["launches"]["ech_leaf"]
    finally:
        gfe.profile_enable(False)
        gfe.lib().gfe_set_server_group_work(2e7)
    assert launches < len(reqs), launches
    for (p, n, A), g in zip(reqs, got):
        alone = gfe.echelon(A, p, n=n if p == 2 else None)
        assert g["rank"] == alone["rank"]
        for k in ("rho", "ups", "R", "M", "K"):
            assert torch.equal(g[k], alone[k]), (p, n, k)
