"""Dynamic updates (Sec. 4, Algorithm 2) through katz_apply_update_batch,
compared after every batch with the oracle session (static recomputation of
omega_1..omega_r on the updated graph, reactivation, further iterations):
same r, same certified ranking, omega and bounds within 1e-12 relative."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.parity import assert_close, assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(g, k, eps, D, r_max=128):
    opts = K.katz_default_opts(keep_history=1, deg_bound=D, r_max=r_max)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(0.0, k, eps)
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps, r_max) == oracle.OK
    assert info.r == s.info()["r"]
    return h, s


def _compare(h, s, k, walks=True):
    inf = s.info()
    c, l, u = s.bounds()
    lo, up, _ = h.bounds()
    assert_close(lo, l, what="lower")
    assert_close(up, u, what="upper")
    kk = min(k, h.n)
    assert_same_ranking(h.ranking(kk), s.ranking(), l)
    if walks:
        for i in range(1, inf["r"] + 1):
            assert_close(h.walk(i), s.alpha_pow(i) * s.omega(i), what=f"s_{i}")


@pytest.mark.parametrize("scale,sizes", [(12, [1, 10, 100, 1000]), (14, [3, 300, 3000])])
def test_batches_match_oracle(scale, sizes):
    g = gg.rmat(scale, 16, seed=40 + scale)
    k, eps = 50, 1e-9
    D = g.deg_max() + 16
    h, s = _pair(g, k, eps, D)
    cur = g
    for b, m in enumerate(sizes):
        src, dst, ins = gg.update_batch(cur, m, seed=1000 * scale + b)
        st = s.apply_update(src, dst, ins)
        if st == oracle.EALPHA:
            with pytest.raises(K.KatzError):
                h.update(src, dst, ins)
            continue
        assert st == oracle.OK
        info = h.update(src, dst, ins)
        cur = gg.apply_batch(cur, src, dst, ins)
        assert info.r == s.info()["r"], (b, info.r, s.info()["r"])
        assert info.converged == 1 and info.nnz == cur.nnz
        _compare(h, s, k)


def test_deletion_batches_like_the_paper():
    # Sec. 5: random existing edges deleted in one batch, top-k re-certified
    g = gg.rmat(13, 16, seed=9)
    k, eps = 100, 1e-4
    h, s = _pair(g, k, eps, g.deg_max())
    cur = g
    for b, m in enumerate([1, 10, 100, 1000]):
        src, dst, ins = gg.update_batch(cur, m, seed=77 + b, p_insert=0.0)
        assert s.apply_update(src, dst, ins) == oracle.OK
        h.update(src, dst, ins)
        cur = gg.apply_batch(cur, src, dst, ins)
        _compare(h, s, k, walks=False)


def test_small_frontier_repairs_only_affected_rows():
    g = gg.path(5000)
    h, s = _pair(g, 5, 1e-6, 3)
    src, dst, ins = np.array([10], np.int32), np.array([12], np.int32), np.array([1], np.uint8)
    info = h.update(src, dst, ins)
    assert s.apply_update(src, dst, ins) == oracle.OK
    assert info.full_levels == 0 and 0 < info.affected < 200
    _compare(h, s, 5)


def test_large_frontier_switches_to_full_levels():
    g = gg.rmat(12, 16, seed=12)
    h, s = _pair(g, 20, 1e-9, g.deg_max() + 64)
    src, dst, ins = gg.update_batch(g, 500, seed=5)
    assert s.apply_update(src, dst, ins) == oracle.OK
    info = h.update(src, dst, ins)
    assert info.full_levels > 0
    _compare(h, s, 20)


def test_invalid_batches_change_nothing():
    g = gg.rmat(11, 8, seed=3)
    D = g.deg_max() + 2
    h, s = _pair(g, 10, 1e-9, D)
    before = (h.ranking(10).copy(), *[x.copy() for x in h.bounds()[:2]])
    a = int(np.argmax(np.diff(g.rowptr)))  # the node of largest degree
    nb = g.col[g.rowptr[a]:g.rowptr[a + 1]]
    non = next(v for v in range(g.n) if v != a and v not in set(nb.tolist()))
    cases = [
        ([a], [int(nb[0])], [1], "KATZ_EINVAL"),            # insert an existing edge
        ([a], [non], [0], "KATZ_EINVAL"),                   # delete an absent edge
        ([a, non], [non, a], [1, 1], "KATZ_EINVAL"),        # the same pair twice
        ([a], [a], [1], "KATZ_EINVAL"),                     # self-loop
        ([a], [g.n], [1], "KATZ_EINVAL"),                   # out of range
    ]
    others = [v for v in range(g.n) if v != a and v not in set(nb.tolist())][:3]
    cases.append(([a] * 3, others, [1, 1, 1], "KATZ_EALPHA"))  # deg(a) would exceed D
    for src, dst, ins, name in cases:
        with pytest.raises(K.KatzError) as e:
            h.update(np.array(src, np.int32), np.array(dst, np.int32), np.array(ins, np.uint8))
        assert e.value.name == name
        assert s.apply_update(src, dst, ins) != oracle.OK
    after = (h.ranking(10), *h.bounds()[:2])
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    # a valid batch still works afterwards
    src, dst, ins = gg.update_batch(g, 20, seed=8)
    assert s.apply_update(src, dst, ins) == oracle.OK
    h.update(src, dst, ins)
    _compare(h, s, 10)


def test_empty_batch_keeps_the_ranking():
    g = gg.rmat(11, 8, seed=4)
    h, s = _pair(g, 10, 1e-9, g.deg_max())
    r0 = h.ranking(10).copy()
    info = h.update(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint8))
    assert info.converged == 1 and np.array_equal(h.ranking(10), r0)


def _star_on_rmat(n_leaves=5000, seed=17):
    base = gg.rmat(13, 8, seed=seed)
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    sel = rows < base.col
    rng = np.random.default_rng(seed)
    leaves = rng.choice(np.arange(1, base.n), n_leaves, replace=False)
    u = np.concatenate([rows[sel], np.zeros(n_leaves, np.int64)])
    v = np.concatenate([base.col[sel], leaves])
    return gg.from_edges(base.n, u, v)


@pytest.mark.parametrize("served", [False, True])
def test_a_hub_row_emptied_and_refilled(served):
    # node 0 is a CHUNK row (degree > 2048); one batch deletes every edge of
    # it, so its row has no chunk left; the next batch gives it three edges
    g = _star_on_rmat()
    assert np.diff(g.rowptr)[0] > 4096
    k, eps = 30, 1e-9
    D = g.deg_max() + 8
    h, s = _pair(g, k, eps, D)
    nb = g.col[g.rowptr[0]:g.rowptr[1]]
    b1 = (np.zeros(len(nb), np.int32), nb.astype(np.int32), np.zeros(len(nb), np.uint8))
    b2 = (np.zeros(3, np.int32), nb[:3].astype(np.int32), np.ones(3, np.uint8))
    if served:
        srv = K.Server(workers=2, slots=2, slot_updates=len(nb))
        srv.attach(h, k)
        tickets = [srv.submit(h, *b) for b in (b1, b2)]
        results = [srv.wait(t, timeout_ms=120000) for t in tickets]
        srv.close()
    for j, b in enumerate((b1, b2)):
        assert s.apply_update(*b) == oracle.OK
        if served:
            status, ids, res = results[j]
            assert status == 0
            if j == 0:
                c, l, u = s.bounds()
                assert_same_ranking(ids, s.ranking(), l)
        else:
            h.update(*b)
            _compare(h, s, k)
    _compare(h, s, k)
    assert h.walk(1)[0] == s.alpha_pow(1) * 3


def test_a_large_degree_bound_and_the_histogram_theta0():
    # D = 2^30: alpha = 1/(D+1) is tiny, and after an update batch theta_0
    # comes from the degree histogram (the relabelling's classes are no
    # longer exact), which holds min(D, 2^24) + 1 bins, not D + 1
    g = gg.rmat(12, 16, seed=95)
    D = 1 << 30
    k, eps = 50, 1e-20
    h, s = _pair(g, k, eps, D)
    src, dst, ins = gg.update_batch(g, 300, seed=96)
    assert s.apply_update(src, dst, ins) == oracle.OK
    info = h.update(src, dst, ins)
    assert info.converged == 1 and info.r == s.info()["r"]
    _compare(h, s, k)
    cur = gg.apply_batch(g, src, dst, ins)
    info = h.rank(0.0, k, eps)  # a static ranking of the updated graph
    t = oracle.Session(cur.rowptr, cur.col, True, D)
    assert t.rank_static(0.0, k, eps, 128) == oracle.OK
    assert info.r == t.info()["r"]
    _compare(h, t, k)
