"""Dynamic updates (Sec. 4, Algorithm 2) on FP32-certified handles.

The walk levels of such a handle are FP64 up to the switch level and FP32
from it on (Sec. 3 bounds widened by a proven rounding-error bound).  A
batch repairs both kinds of levels in the arithmetic and summation order the
ranking used, rebuilds the two partial sums, re-derives the bounds from
scratch and re-certifies.  Checks after every batch:
- the certified bounds bracket the exact Katz score of the updated graph (a
  sparse FP64 solve of (I - alpha A) y = alpha A 1);
- the ranking is the FP64 oracle's, up to ties within eps;
- the FP64 levels match the oracle's walk counts, the FP32 levels stay
  within FP32 rounding of them;
- repairing only the affected rows gives the bits of full-level repairs;
- a row grown far past its row mode's length widens the error bound and the
  bracketing still holds;
- an update that makes two top-k nodes exact twins stalls FP32 (no order
  of equal scores fits in the FP32 widening), and KATZ_FP32_CERT_AUTO
  recomputes the ranking in FP64."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import graphgen as gg
import oracle
from tests.parity import assert_close, assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _katz(g, alpha):
    """Katz scores sum_{i>=1} alpha^i A^i 1 of the graph, FP64 sparse solve."""
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    A = sp.csr_matrix((np.ones(g.nnz), (rows, g.col)), shape=(n, n))
    rhs = alpha * (A @ np.ones(n))
    return spla.spsolve((sp.identity(n, format="csc") - alpha * A).tocsc(), rhs)


def _bracket(h, g, alpha):
    lo, up, err = h.bounds()
    y = _katz(g, alpha)
    slack = 1e-10 * np.abs(y) + 1e-300
    bad_l = np.nonzero(lo > y + slack)[0]
    bad_u = np.nonzero(up < y - slack)[0]
    assert bad_l.size == 0, ("lower above Katz", bad_l[:5], lo[bad_l[:5]], y[bad_l[:5]])
    assert bad_u.size == 0, ("upper below Katz", bad_u[:5], up[bad_u[:5]], y[bad_u[:5]])
    return err


def _opts(**kw):
    base = dict(precision=K.KATZ_FP32_CERT, keep_history=1, r_max=256)
    base.update(kw)
    return K.katz_default_opts(**base)


def _batches(g, sizes, seed, directed, D):
    out, cur = [], g
    for b, m in enumerate(sizes):
        if directed:
            bt = gg.directed_update_batch(cur, m, seed=seed + b, deg_bound=D)
            cur = gg.apply_directed_batch(cur, *bt)
        else:
            bt = gg.update_batch(cur, m, seed=seed + b)
            cur = gg.apply_batch(cur, *bt)
        out.append((bt, cur))
    return out


@pytest.mark.parametrize("fp32_from", [0, 2, 4])
@pytest.mark.parametrize("directed", [False, True])
def test_fp32_updates_bracket_katz_and_rank_like_the_oracle(fp32_from, directed):
    g = gg.rmat(12, 16, seed=81)
    if directed:
        g = gg.orient(g, seed=82)
    D = g.deg_max() + 32
    k = 40
    eps = 1e-9 if fp32_from == 0 else 1e-4
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(deg_bound=D, fp32_from=fp32_from, undirected=0 if directed else 1))
    info = h.rank(0.0, k, eps)
    assert info.converged == 1
    alpha = info.alpha
    s = oracle.Session(g.rowptr, g.col, not directed, D)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    _bracket(h, g, alpha)
    for b, (bt, cur) in enumerate(_batches(g, [1, 30, 600, 3000], 900 + 10 * fp32_from, directed, D)):
        assert s.apply_update(*bt) == oracle.OK
        info = h.update(*bt)
        assert info.converged == 1 and info.nnz == cur.nnz
        if fp32_from:
            assert info.fp32_levels == info.r - fp32_from + 1, (b, info.fp32_levels, info.r)
        _bracket(h, cur, alpha)
        c, l, u = s.bounds()
        assert_same_ranking(h.ranking(k), s.ranking(), l, atol=eps)
        f = fp32_from or (info.r - info.fp32_levels + 1)
        for i in range(1, min(info.r, s.info()["r"]) + 1):
            want = s.alpha_pow(i) * s.omega(i)
            if i < f:
                assert_close(h.walk(i), want, what=f"s_{i} (FP64 level)")
            else:  # FP32 storage and sums: a few units of 2^-24 per level
                got = h.walk(i)
                tol = 4e-6 * i * np.abs(want) + 1e-37
                assert np.all(np.abs(got - want) <= tol), (b, i, np.max(np.abs(got - want) / (np.abs(want) + 1e-300)))
    h.close()


def _rmat_with_hub(scale, seed, hub_deg):
    """R-MAT plus a hub (node 0) joined to hub_deg random nodes: a row long
    enough for the chunked row mode."""
    g = gg.rmat(scale, 16, seed=seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    keep = rows < g.col
    extra = np.random.default_rng(seed).choice(np.arange(1, g.n), hub_deg, replace=False)
    u = np.concatenate([rows[keep], np.zeros(hub_deg, np.int64)])
    v = np.concatenate([g.col[keep], extra])
    return gg.from_edges(g.n, u, v)


@pytest.mark.parametrize("fp32_from", [2, 3, 0])
@pytest.mark.parametrize("directed", [False, True])
def test_fp32_row_repairs_have_the_bits_of_full_levels(fp32_from, directed):
    # the same batches through frontier repairs (default) and through full
    # levels only (frontier_abort_frac tiny): identical walks and bounds
    g = _rmat_with_hub(13, 83, 5000)
    if directed:
        g = gg.orient(g, seed=84)
    assert g.deg_max() > 2048  # a chunked (hub) row
    D = g.deg_max() + 32
    k, eps = 30, (1e-9 if fp32_from == 0 else 1e-4)
    common = dict(deg_bound=D, fp32_from=fp32_from, undirected=0 if directed else 1)
    a = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(**common))
    f = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(frontier_abort_frac=1e-12, **common))
    ia, if_ = a.rank(0.0, k, eps), f.rank(0.0, k, eps)
    assert ia.r == if_.r
    some_rows = False
    for bt, cur in _batches(g, [1, 5, 40, 400], 950, directed, D):
        ia, if_ = a.update(*bt), f.update(*bt)
        assert ia.r == if_.r and if_.full_levels >= 1
        some_rows |= ia.full_levels < ia.r
        for i in range(1, ia.r + 1):
            np.testing.assert_array_equal(a.walk(i), f.walk(i), err_msg=f"s_{i}")
        for x, y in zip(a.bounds(), f.bounds()):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(a.ranking(k), f.ranking(k))
    assert some_rows  # the frontier path was taken at least once
    a.close()
    f.close()


def test_fp32_a_long_row_widens_the_bound_and_stays_certified():
    # a node of degree <= 16 (THREAD rows: one lane, eight-term groups) gets
    # 600 new neighbours: its FP32 row sum chains ~80 groups instead of 2
    g = gg.rmat(12, 16, seed=85)
    deg = np.diff(g.rowptr)
    w = int(np.nonzero((deg >= 2) & (deg <= 8))[0][0])
    D = max(g.deg_max(), int(deg[w]) + 600) + 700
    k, eps = 30, 1e-4
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(deg_bound=D, fp32_from=2))
    info = h.rank(0.0, k, eps)
    alpha = info.alpha
    err0 = _bracket(h, g, alpha)
    h0_up = h.bounds()[1]
    nb = set(g.col[g.rowptr[w]:g.rowptr[w + 1]].tolist()) | {w}
    rng = np.random.default_rng(5)
    cand = np.array([v for v in rng.permutation(g.n).tolist() if v not in nb][:600], np.int32)
    src = np.full(len(cand), w, np.int32)
    ins = np.ones(len(cand), np.uint8)
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    assert s.apply_update(src, cand, ins) == oracle.OK
    info = h.update(src, cand, ins)
    cur = gg.apply_batch(g, src, cand, ins)
    assert info.converged == 1
    up0 = h0_up
    err1 = _bracket(h, cur, alpha)
    up1 = h.bounds()[1]
    # the rounding widening, relative to the score, grew with the depth
    pos = np.nonzero((up0 > 0) & (up1 > 0))[0]
    assert np.median(err1[pos] / up1[pos]) > 2.0 * np.median(err0[pos] / up0[pos])
    c, l, u = s.bounds()
    assert_same_ranking(h.ranking(k), s.ranking(), l, atol=eps)
    # and a second batch on the deepened handle still certifies
    bt = gg.update_batch(cur, 200, seed=86)
    assert s.apply_update(*bt) == oracle.OK
    info = h.update(*bt)
    assert info.converged == 1
    _bracket(h, gg.apply_batch(cur, *bt), alpha)
    h.close()


def _twin_batch(g, t):
    """Edge updates that give some node w (not adjacent to t) exactly t's
    neighbourhood: w and t then have equal Katz scores."""
    deg = np.diff(g.rowptr)
    nt = set(g.col[g.rowptr[t]:g.rowptr[t + 1]].tolist())
    for w in np.argsort(deg, kind="stable").tolist():
        if w == t or w in nt or deg[w] == 0:
            continue
        nw = set(g.col[g.rowptr[w]:g.rowptr[w + 1]].tolist())
        dele = sorted(nw - nt)
        add = sorted(nt - nw)
        src = np.array([w] * (len(dele) + len(add)), np.int32)
        dst = np.array(dele + add, np.int32)
        ins = np.array([0] * len(dele) + [1] * len(add), np.uint8)
        return w, src, dst, ins
    raise AssertionError("no twin candidate")


@pytest.mark.parametrize("auto", [False, True])
def test_fp32_update_making_exact_twins_stalls_or_escalates(auto):
    # eps far below the FP32 widening: the original top-4 certifies in FP32
    # (its gaps are wide), the twins' order never can
    g = gg.rmat(11, 16, seed=88)
    D = 2 * g.deg_max() + 8
    k, eps = 4, 1e-9
    pr = K.KATZ_FP32_CERT_AUTO if auto else K.KATZ_FP32_CERT
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(deg_bound=D, fp32_from=3, precision=pr))
    info = h.rank(0.0, k, eps)
    assert info.converged == 1 and info.escalated == 0 and info.fp32_levels > 0
    alpha = info.alpha
    top = int(h.ranking(1)[0])
    w, src, dst, ins = _twin_batch(g, top)
    cur = gg.apply_batch(g, src, dst, ins)
    y = _katz(cur, alpha)
    assert abs(y[w] - y[top]) <= 1e-12 * y[top]  # twins: equal scores
    if not auto:
        with pytest.raises(K.KatzError) as e:
            h.update(src, dst, ins)
        assert e.value.name == "KATZ_EPRECISION"
        _bracket(h, cur, alpha)  # the bounds stay certified; the order is not
        h.close()
        return
    info = h.update(src, dst, ins)
    assert info.escalated == 1 and info.converged == 1 and info.fp32_levels == 0
    ref = oracle.Session(cur.rowptr, cur.col, True, D)  # a static FP64 ranking of the updated graph
    assert ref.rank_static(0.0, k, eps, 256) == oracle.OK
    assert info.r == ref.info()["r"]
    c, l, u = ref.bounds()
    lo, up, _ = h.bounds()
    assert_close(lo, l, what="lower")
    assert_close(up, u, what="upper")
    assert_same_ranking(h.ranking(k), ref.ranking(), l)
    # the handle goes on in FP64
    bt = gg.update_batch(cur, 50, seed=89)
    s = oracle.Session(cur.rowptr, cur.col, True, D)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    assert s.apply_update(*bt) == oracle.OK
    info = h.update(*bt)
    assert info.converged == 1 and info.fp32_levels == 0 and info.r == s.info()["r"]
    c, l, u = s.bounds()
    assert_close(h.bounds()[0], l, what="lower after escalation")
    h.close()


def test_fp32_updates_continue_after_a_checkpoint():
    # the image carries the FP32 partial sum and the FP32 input of the first
    # FP32 level: a restored handle repairs the next batch to the same bits
    g = gg.rmat(12, 16, seed=90)
    D = g.deg_max() + 32
    k, eps = 30, 1e-4
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(deg_bound=D, fp32_from=3))
    h.rank(0.0, k, eps)
    cur = g
    for bt, cur in _batches(g, [20], 91, False, D):
        h.update(*bt)
    h2 = K.Katz.restore(h.checkpoint())
    for bt, _ in _batches(cur, [1, 300], 92, False, D):
        i1, i2 = h.update(*bt), h2.update(*bt)
        assert i1.r == i2.r and i1.fp32_levels == i2.fp32_levels
        for i in range(1, i1.r + 1):
            np.testing.assert_array_equal(h.walk(i), h2.walk(i))
        for x, y in zip(h.bounds(), h2.bounds()):
            np.testing.assert_array_equal(x, y)
    h.close()
    h2.close()
