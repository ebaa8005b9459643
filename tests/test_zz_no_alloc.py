"""dl_sim_join_noalloc: the allocation-free exact join, through the C ABI.

Some callers cannot allocate device memory when they run a join (a memory
planner owns the device, or a real-time loop must not enter the allocator).
They call dl_sim_join_noalloc with their own input and output buffers; its
working memory is a static device array inside the library, shared by every
call. This test checks, on two calls in a row each, that it returns exactly the
pairs of the FP64 oracle and of the regular dl_sim_join (exact set equality, the
tolerance of every parity test here) for an R x S join, a self-join in both
modes and an odd d (the scalar recheck path), and that it refuses what it must:
a band larger than the static array, a too-small output buffer, a feature out of
the domain and a misaligned row pointer. It lives in its own file, collected
last.
"""

import ctypes

import numpy as np
import pytest

import oracle
from oracle import MODE_RXS, MODE_SELF_FULL, MODE_SELF_UPPER
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_1812_07607_gb300 import build as B, dl
    B.build()
    return torch, dl, dl.load(), oracle.default()


def _call(L, torch, R, rid, S, sid, eps, self_mode, out_r, out_s, cap, d=None, nR=None):
    n = ctypes.c_int64(-1)
    st = torch.cuda.current_stream().cuda_stream
    rc = L.dl_sim_join_noalloc(R.data_ptr(), rid.data_ptr(), R.shape[0] if nR is None else nR,
                               None if S is None else S.data_ptr(), None if sid is None else sid.data_ptr(),
                               0 if S is None else S.shape[0], R.shape[1] if d is None else d, eps, self_mode,
                               out_r, out_s, cap, ctypes.byref(n), st)
    return rc, int(n.value)


def _noalloc(env, R, rid, S, sid, eps, self_mode, cap):
    torch, dl, L, _ = env
    out_r = torch.empty(cap, dtype=torch.int64, device="cuda")
    out_s = torch.empty(cap, dtype=torch.int64, device="cuda")
    rc, k = _call(L, torch, R, rid, S, sid, eps, self_mode, out_r.data_ptr(), out_s.data_ptr(), cap)
    assert rc == 0, L.dl_last_error()
    pairs = list(zip(out_r[:k].cpu().tolist(), out_s[:k].cpu().tolist()))
    assert len(set(pairs)) == len(pairs), "duplicate pair in output"
    return set(pairs)


def _regular(env, R, rid, S, sid, eps, self_mode):
    _, dl, _, _ = env
    res = dl.sim_join(dl.Store(rid, R), None if S is None else dl.Store(sid, S), eps, precision="fp32",
                      self_mode=self_mode)
    a, b = res.pairs_host()
    res.free()
    return set(zip(a.tolist(), b.tolist()))


def _oracle(env, Rh, rid, Sh, sid, eps, mode):
    orc = env[3]
    p = orc.join(Rh, Sh, eps, mode)
    rid_h = rid.cpu().numpy()
    sid_h = rid_h if Sh is None else sid.cpu().numpy()
    return set(zip(rid_h[p[:, 0]].tolist(), sid_h[p[:, 1]].tolist()))


def test_noalloc_rxs_matches_oracle_and_dl_sim_join_twice(env):
    torch = env[0]
    wl = W.rxs_histograms_2k()
    R, S = torch.from_numpy(wl.R).cuda(), torch.from_numpy(wl.S).cuda()
    rid, sid = torch.from_numpy(wl.r_ids).cuda(), torch.from_numpy(wl.s_ids).cuda()
    want = _oracle(env, wl.R, rid, wl.S, sid, wl.eps, MODE_RXS)
    assert len(want) > 1000
    assert _regular(env, R, rid, S, sid, wl.eps, "upper") == want
    for _ in range(2):
        assert _noalloc(env, R, rid, S, sid, wl.eps, 0, 1 << 16) == want


@pytest.mark.parametrize("mode", ["upper", "full"])
def test_noalloc_self_join_matches_oracle_twice(env, mode):
    torch, dl = env[0], env[1]
    X, _ = W.clustered_histograms(W.rng(5), 3000, 64, 300, 0.01)
    Xd = torch.from_numpy(X).cuda()
    xid = torch.arange(3000, dtype=torch.int64, device="cuda") * 5 + 1
    want = _oracle(env, X, xid, None, None, 0.1, MODE_SELF_UPPER if mode == "upper" else MODE_SELF_FULL)
    assert len(want) > 3000
    assert _regular(env, Xd, xid, None, None, 0.1, mode) == want
    sm = dl.DL_SELF_UPPER if mode == "upper" else dl.DL_SELF_FULL
    for _ in range(2):
        assert _noalloc(env, Xd, xid, None, None, 0.1, sm, 1 << 20) == want


def test_noalloc_odd_d_matches_oracle_twice(env):
    torch = env[0]
    g = W.rng(6)
    R = W.dirichlet_histograms(g, 700, 65)
    S = np.concatenate([R[:50], W.dirichlet_histograms(g, 650, 65)])
    D = env[3].dist_block(R[:64], S)
    eps = float(np.sqrt(np.quantile(D, 0.01)))
    Rd, Sd = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    rid = torch.arange(700, dtype=torch.int64, device="cuda") + 7
    sid = torch.arange(700, dtype=torch.int64, device="cuda") + (1 << 40)
    want = _oracle(env, R, rid, S, sid, eps, MODE_RXS)
    assert len(want) > 500
    assert _regular(env, Rd, rid, Sd, sid, eps, "upper") == want
    for _ in range(2):
        assert _noalloc(env, Rd, rid, Sd, sid, eps, 0, 1 << 16) == want


def test_noalloc_refusals_then_a_good_call(env):
    torch, dl, L, _ = env
    # one-hot rows: distinct rows are exactly sqrt(2) apart, so at eps = sqrt(2) nearly every
    # pair sits inside the FP32 error band -- far more than the static array holds
    H = torch.from_numpy(W.one_hot_rows(W.rng(7), 400, 16)).cuda()
    hid = torch.arange(400, dtype=torch.int64, device="cuda")
    out = torch.empty(1 << 18, dtype=torch.int64, device="cuda")
    rc, _ = _call(L, torch, H, hid, H, hid, float(np.sqrt(2.0)), 0, out.data_ptr(), out.data_ptr() + 8 * (1 << 17),
                  1 << 17)
    assert rc == dl.DL_EOVERFLOW, L.dl_last_error()

    wl = W.rxs_histograms_2k()
    R, S = torch.from_numpy(wl.R).cuda(), torch.from_numpy(wl.S).cuda()
    rid, sid = torch.from_numpy(wl.r_ids).cuda(), torch.from_numpy(wl.s_ids).cuda()
    # output buffer too small: refused with the required count
    small = torch.empty(4, dtype=torch.int64, device="cuda")
    rc, n = _call(L, torch, R, rid, S, sid, wl.eps, 0, small.data_ptr(), small.data_ptr() + 16, 2)
    assert rc == dl.DL_EOVERFLOW and n > 2

    # features outside the domain of the error bounds: refused
    for bad in (2.0 ** 41, float("nan"), float("inf")):
        Rb = R.clone()
        Rb[17, 3] = bad
        rc, _ = _call(L, torch, Rb, rid, S, sid, wl.eps, 0, out.data_ptr(), out.data_ptr() + 8 * 1024, 1024)
        assert rc == dl.DL_EINVAL, (bad, L.dl_last_error())
        rc, _ = _call(L, torch, R, rid, Rb, sid, wl.eps, 0, out.data_ptr(), out.data_ptr() + 8 * 1024, 1024)
        assert rc == dl.DL_EINVAL, (bad, L.dl_last_error())

    # a row pointer off its 16-byte boundary at d % 4 == 0: refused on the host, before any launch
    # (nR - 1 rows, so even the shifted range lies inside the buffer)
    n_out = ctypes.c_int64(-1)
    rc = L.dl_sim_join_noalloc(R.data_ptr() + 4, rid.data_ptr(), R.shape[0] - 1, S.data_ptr(), sid.data_ptr(),
                               S.shape[0], R.shape[1], wl.eps, 0, out.data_ptr(), out.data_ptr() + 8 * 1024, 1024,
                               ctypes.byref(n_out), torch.cuda.current_stream().cuda_stream)
    assert rc == dl.DL_EINVAL

    # the shared array keeps the refused calls' contents; the next call still starts clean
    want = _oracle(env, wl.R, rid, wl.S, sid, wl.eps, MODE_RXS)
    assert _noalloc(env, R, rid, S, sid, wl.eps, 0, 1 << 16) == want
