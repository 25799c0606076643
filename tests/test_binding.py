"""The Python binding's batched-result buffers (CPU only, no library call):
every matrix's slots are disjoint, the C result structs point at them, and a
BatchResult slices the same shapes echelon() returns."""
import torch

from paper_1806_04211_gb300 import gfe


def fake(p, m, n):
    if p == 2:
        return gfe.matrix_arg(torch.zeros((m, gfe.words_per_row(n)), dtype=torch.int64), 2, n)
    return gfe.matrix_arg(torch.zeros((m, n), dtype=torch.uint8), p)


def test_batch_buffers_are_disjoint_and_addressed():
    args = [fake(*s) for s in [(3, 5, 7), (2, 70, 130), (251, 1, 1), (2, 1, 65), (7, 40, 12)]]
    (idx, u8, wb), slots, res = gfe._alloc_results(args, "cpu", True)
    spans = {"idx": [], "u8": [], "w": []}
    for mat, sl, r in zip(args, slots, res):
        k = sl["k"]
        spans["idx"].append((sl["idx"], sl["idx"] + 1 + 2 * k))
        assert r.rank == idx.data_ptr() + 8 * sl["idx"]
        assert r.pivot_cols == r.rank + 8 and r.pivot_rows == r.rank + 8 * (1 + k)
        bits = mat.fmt == gfe.GFE_BITS64
        for key, ptr, ld in (("R", r.R, r.ldR), ("M", r.M, r.ldM), ("K", r.K, r.ldK)):
            off, rows, cols = sl[key]
            spans["w" if bits else "u8"].append((off, off + rows * cols))
            base, es = (wb.data_ptr(), 8) if bits else (u8.data_ptr(), 1)
            assert ptr == base + es * off and ld == es * cols
    for v in spans.values():  # no two slots overlap
        v.sort()
        assert all(a[1] <= b[0] for a, b in zip(v, v[1:]))
    assert spans["idx"][-1][1] == idx.numel()


def test_batch_result_shapes_follow_the_rank():
    args = [fake(7, 40, 12), fake(2, 70, 130)]
    bufs, slots, res = gfe._alloc_results(args, "cpu", True)
    a = gfe.BatchResult(bufs, args[0], slots[0], 9)
    assert a["rank"] == 9 and len(a) == 6 and set(a) == {"rank", "ups", "rho", "R", "M", "K"}
    assert a["ups"].shape == (9,) and a["R"].shape == (9, 3) and a["M"].shape == (9, 9) and a["K"].shape == (31, 9)
    b = gfe.BatchResult(bufs, args[1], slots[1], 65)
    assert b["R"].shape == (65, gfe.words_per_row(130 - 65)) and b["M"].shape == (65, gfe.words_per_row(65))
    assert b["K"].shape == (5, gfe.words_per_row(65))
    z = gfe.BatchResult(bufs, args[1], slots[1], 0)
    assert z["R"].shape[0] == 0 and z["ups"].numel() == 0
    bufs2, slots2, _ = gfe._alloc_results(args[:1], "cpu", False)
    c = gfe.BatchResult(bufs2, args[0], slots2[0], 4)
    assert "M" not in c and len(c) == 4


def test_workspace_cache_is_per_thread():
    """Concurrent calls from several host threads must not share a workspace."""
    import threading
    got = {}
    together = threading.Barrier(3)

    def grab(name):
        got[name] = gfe._workspace(1024, "cpu")
        together.wait()  # all three alive at once: three distinct threads

    ts = [threading.Thread(target=grab, args=(i,)) for i in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    ptrs = {got[i].data_ptr() for i in range(3)}
    assert len(ptrs) == 3
    gfe.release_workspace()
