"""dl_sim_join_noalloc: the allocation-free exact join, through the C ABI.

Some callers cannot allocate device memory when they run a join (a memory
planner owns the device, or a real-time loop must not enter the allocator).
They call dl_sim_join_noalloc with their own input and output buffers; its
working memory is a static device array inside the library. This test checks
that two calls in a row return exactly the pairs the regular dl_sim_join
returns (exact set equality, the tolerance of every parity test here), for an
R x S join and a self-join. It lives in its own file, collected last.
"""

import ctypes

import numpy as np
import pytest

from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(L, torch, R, rid, S, sid, eps, self_mode, cap):
    out_r = torch.empty(cap, dtype=torch.int64, device="cuda")
    out_s = torch.empty(cap, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64(-1)
    st = torch.cuda.current_stream().cuda_stream
    rc = L.dl_sim_join_noalloc(R.data_ptr(), rid.data_ptr(), R.shape[0],
                               None if S is None else S.data_ptr(), None if sid is None else sid.data_ptr(),
                               0 if S is None else S.shape[0], R.shape[1], eps, self_mode,
                               out_r.data_ptr(), out_s.data_ptr(), cap, ctypes.byref(n), st)
    assert rc == 0, L.dl_last_error()
    k = int(n.value)
    return set(zip(out_r[:k].cpu().tolist(), out_s[:k].cpu().tolist())), k


def test_noalloc_matches_dl_sim_join_twice():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_1812_07607_gb300 import build as B, dl
    B.build()
    L = dl.load()
    wl = W.rxs_histograms_2k()
    R = torch.from_numpy(wl.R).cuda()
    S = torch.from_numpy(wl.S).cuda()
    rid = torch.from_numpy(wl.r_ids).cuda()
    sid = torch.from_numpy(wl.s_ids).cuda()

    ref = dl.sim_join(dl.Store(rid, R), dl.Store(sid, S), wl.eps, precision="fp32")
    a, b = ref.pairs_host()
    want = set(zip(a.tolist(), b.tolist()))
    ref.free()
    assert len(want) > 1000
    for _ in range(2):
        got, k = _noalloc(L, torch, R, rid, S, sid, wl.eps, dl.DL_SELF_UPPER, 1 << 16)
        assert k == len(want) and got == want

    g = W.rng(5)
    X, _ = W.clustered_histograms(g, 3000, 64, 300, 0.01)
    Xd = torch.from_numpy(X).cuda()
    xid = torch.arange(3000, dtype=torch.int64, device="cuda") * 5 + 1
    ref = dl.sim_join(dl.Store(xid, Xd), None, 0.1, precision="fp32", self_mode="full")
    a, b = ref.pairs_host()
    want = set(zip(a.tolist(), b.tolist()))
    ref.free()
    for _ in range(2):
        got, k = _noalloc(L, torch, Xd, xid, None, None, 0.1, dl.DL_SELF_FULL, 1 << 20)
        assert k == len(want) and got == want

    # too small an output buffer: rejected with the required count
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64()
    rc = L.dl_sim_join_noalloc(R.data_ptr(), rid.data_ptr(), R.shape[0], S.data_ptr(), sid.data_ptr(),
                               S.shape[0], R.shape[1], wl.eps, 0, out.data_ptr(), out.data_ptr(), 2,
                               ctypes.byref(n), torch.cuda.current_stream().cuda_stream)
    assert rc == dl.DL_EOVERFLOW and n.value > 2
