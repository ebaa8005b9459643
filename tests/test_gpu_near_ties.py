"""Pairs at eps to within 1e-6: the float-float stage decides them, the canonical FP64 sum
only the exact ties, and the result set still equals the FP64 oracle's.

The store is built so that thousands of pairs have squared distances 1 +- 2e-6 around
eps^2 = 1: inside the zone the FP32 bound leaves undecided ((d+8) 2^-24 relative), outside
the float-float zone ((d+34)^2 2^-48). Rows on a 2^-10 grid plus a unit step in one
coordinate give pairs at exactly eps (ties, accepted by the predicate's <=), and the same
plus 2^-10 in another coordinate pairs 2^-20 above it (rejected). Checked for the BF16,
FP8 and exact FP32 joins and for a batch request; the count of canonical FP64 decisions
must stay at the number of ties, where before the float-float stage every pair of the
FP32 zone took it.
"""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

D_DIM = 64
N_NEAR, N_TIE, N_ABOVE = 3000, 20, 20


@pytest.fixture(scope="module")
def dl():
    import torch
    from paper_1812_07607_gb300 import build as B, dl as D
    assert torch.cuda.is_available()
    B.build()
    D.load()
    return D


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.fixture(scope="module")
def rows():
    return make_rows()


def make_rows():
    g = np.random.default_rng(4242)
    n = N_NEAR + N_TIE + N_ABOVE
    Q = (g.integers(0, 1024, (n, D_DIM)) / 1024.0).astype(np.float32)
    u = g.standard_normal((N_NEAR, D_DIM))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    X = Q.copy()
    X[:N_NEAR] = (Q[:N_NEAR].astype(np.float64) + u * (1.0 + 1e-6 * g.uniform(-1, 1, (N_NEAR, 1)))).astype(np.float32)
    j = g.integers(0, D_DIM, N_TIE + N_ABOVE)
    t = np.arange(N_NEAR, n)
    X[t, j] += np.float32(1.0)                                  # exact: squared distance 1
    a = t[N_TIE:]
    j2 = (j[N_TIE:] + 1) % D_DIM
    X[a, j2] = np.where(X[a, j2] >= np.float32(0.5), X[a, j2] - np.float32(2.0 ** -10),
                        X[a, j2] + np.float32(2.0 ** -10))      # 1 + 2^-20
    return Q, X


def _store(dl, ids, X):
    import torch
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(), torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _want(orc, Q, X, qid, xid):
    p = orc.join(Q, X, 1.0, oracle.MODE_RXS)
    return set(zip(qid[p[:, 0]].tolist(), xid[p[:, 1]].tolist()))


def test_rows_straddle_eps(orc, rows):
    Q, X = rows
    D = orc.dist_block(Q[:N_NEAR], X[:N_NEAR])
    diag = np.diag(D)
    assert np.all(np.abs(diag - 1.0) < 3e-6)
    assert np.mean(np.abs(diag - 1.0) > (D_DIM + 8) * 2.0 ** -24 * 2) < 0.5   # most are in the FP32 zone
    t = np.arange(N_NEAR, N_NEAR + N_TIE + N_ABOVE)
    Dt = np.array([orc.dist_block(Q[i:i + 1], X[i:i + 1])[0, 0] for i in t])
    assert np.all(Dt[:N_TIE] == 1.0) and np.all(Dt[N_TIE:] == 1.0 + 2.0 ** -20)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_near_ties_exact_and_few_fp64(dl, orc, rows, prec):
    Q, X = rows
    qid = np.arange(Q.shape[0], dtype=np.int64) + 7
    xid = np.arange(X.shape[0], dtype=np.int64) + (1 << 33)
    res = dl.sim_join(_store(dl, qid, Q), _store(dl, xid, X), 1.0, precision=prec)
    a, b = res.pairs_host()
    st = res.stats()
    res.free()
    got = set(zip(a.tolist(), b.tolist()))
    want = _want(orc, Q, X, qid, xid)
    assert got == want
    assert len(want) > N_NEAR // 3 and len(want) < N_NEAR
    assert st["band_pairs"] >= N_NEAR // 2
    assert N_TIE <= st["fp64_pairs"] <= N_TIE + 10


def test_near_ties_in_a_batch(dl, orc, rows):
    import torch
    Q, X = rows
    xid = np.arange(X.shape[0], dtype=np.int64) * 5
    S = _store(dl, xid, X)
    qid = np.arange(Q.shape[0], dtype=np.int64) + 100
    half = Q.shape[0] // 2
    reqs = [{"kind": "eps", "q_begin": 0, "nq": half, "eps": 1.0},
            {"kind": "eps", "q_begin": half, "nq": Q.shape[0] - half, "eps": 1.0}]
    res = dl.batch_join(S, torch.from_numpy(qid).cuda(), torch.from_numpy(Q).cuda(), reqs)
    st = res.stats()
    got = set()
    for i in range(2):
        r, s = res.request_pairs(i)
        got |= set(zip(r.tolist(), s.tolist()))
    res.free()
    assert got == _want(orc, Q, X, qid, xid)
    assert N_TIE <= st["fp64_pairs"] <= N_TIE + 10
