"""Dynamic updates on directed graphs (Sec. 4 with Sec. 2.1's ordered pairs):
an update a -> b changes the row of a alone, and the affected set grows
along in-arcs.  katz_apply_update_batch is compared after every batch with
the directed oracle session (static recomputation on the updated graph):
same r, same certified ranking, walks and bounds within 1e-12 relative."""
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


def _pair(g, k, eps, D, r_max=128, **kw):
    opts = K.katz_default_opts(undirected=0, keep_history=1, deg_bound=D, r_max=r_max, **kw)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(0.0, k, eps)
    s = oracle.Session(g.rowptr, g.col, False, D)
    assert s.rank_static(0.0, k, eps, r_max) == oracle.OK
    assert info.r == s.info()["r"]
    return h, s


def _compare(h, s, k, walks=True):
    inf = s.info()
    c, l, u = s.bounds()
    lo, up, _ = h.bounds()
    assert_close(lo, l, what="lower")
    assert_close(up, u, what="upper")
    assert_same_ranking(h.ranking(min(k, h.n)), s.ranking(), l)
    if walks:
        for i in range(1, inf["r"] + 1):
            assert_close(h.walk(i), s.alpha_pow(i) * s.omega(i), what=f"s_{i}")


def _run_batches(g, h, s, k, sizes, seed, D, walks=True):
    cur = g
    for b, m in enumerate(sizes):
        src, dst, ins = gg.directed_update_batch(cur, m, seed=seed + b, deg_bound=D)
        assert s.apply_update(src, dst, ins) == oracle.OK
        info = h.update(src, dst, ins)
        cur = gg.apply_directed_batch(cur, src, dst, ins)
        assert info.r == s.info()["r"], (b, info.r, s.info()["r"])
        assert info.converged == 1 and info.nnz == cur.nnz
        _compare(h, s, k, walks)
    return cur


@pytest.mark.parametrize("scale,sizes", [(12, [1, 10, 100, 1000]), (14, [3, 300, 3000])])
def test_directed_batches_match_oracle(scale, sizes):
    g = gg.orient(gg.rmat(scale, 16, seed=60 + scale), seed=scale)
    k, eps = 50, 1e-9
    D = g.deg_max() + 16
    h, s = _pair(g, k, eps, D)
    _run_batches(g, h, s, k, sizes, 2000 * scale, D)


def _hub_graph(n=8192, hub_out=6000, hub_in=7000, seed=3):
    """Oriented R-MAT plus node 5 pointing at hub_out nodes (a CHUNK row of
    the SpMV) and hub_in nodes pointing at node 7 (a large in-row)."""
    rng = np.random.default_rng(seed)
    base = gg.orient(gg.rmat(13, 8, seed=seed), seed=seed)
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    outs = rng.choice(n, hub_out, replace=False)
    ins = rng.choice(n, hub_in, replace=False)
    u = np.concatenate([rows, np.full(hub_out, 5), ins])
    v = np.concatenate([base.col, outs, np.full(hub_in, 7)])
    return gg.directed_from_arcs(n, u, v, "hubs")


def test_directed_hub_rows_and_in_hubs():
    g = _hub_graph()
    assert g.deg_max() > 4096
    k, eps = 40, 1e-9
    D = g.deg_max() + 8
    h, s = _pair(g, k, eps, D)
    cur = g
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    arcs = set(zip(rows.tolist(), g.col.tolist()))
    rows5 = set(cur.col[cur.rowptr[5]:cur.rowptr[5 + 1]].tolist())
    # arcs out of the out-hub deleted and inserted, arcs into the in-hub
    # deleted and inserted, and the arcs between the two hubs flipped
    dele = sorted(v for v in rows5 if v != 7)[:40]
    add = [v for v in range(cur.n) if v not in (5, 7) and v not in rows5][:40]
    into7 = [x for x in range(cur.n) if (x, 7) in arcs and x != 5][:30]
    new7 = [x for x in range(cur.n) if x not in (5, 7) and (x, 7) not in arcs and x not in add][:30]
    src = [5] * 80 + into7 + new7
    dst = dele + add + [7] * 60
    ins = [0] * 40 + [1] * 40 + [0] * 30 + [1] * 30
    for a, b in [(5, 7), (7, 5)]:
        src.append(a)
        dst.append(b)
        ins.append(0 if (a, b) in arcs else 1)
    src, dst, ins = np.array(src, np.int32), np.array(dst, np.int32), np.array(ins, np.uint8)
    assert len(set(zip(src.tolist(), dst.tolist()))) == len(src)
    st = s.apply_update(src, dst, ins)
    assert st == oracle.OK
    info = h.update(src, dst, ins)
    cur = gg.apply_directed_batch(cur, src, dst, ins)
    assert info.nnz == cur.nnz
    _compare(h, s, k)
    _run_batches(cur, h, s, k, [50, 2000], 77, D)


def test_reciprocal_arcs_in_one_batch():
    g = gg.orient(gg.rmat(11, 8, seed=21), seed=1)
    k, eps = 20, 1e-9
    D = g.deg_max() + 8
    h, s = _pair(g, k, eps, D)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    arcs = set(zip(rows.tolist(), g.col.tolist()))
    one_way = [(a, b) for a, b in sorted(arcs) if (b, a) not in arcs][:5]
    absent = [(a, b) for a in range(40) for b in range(40, 80) if (a, b) not in arcs and (b, a) not in arcs][:5]
    src = [b for a, b in one_way] + [a for a, b in absent] + [b for a, b in absent]
    dst = [a for a, b in one_way] + [b for a, b in absent] + [a for a, b in absent]
    ins = [1] * len(src)
    assert s.apply_update(src, dst, ins) == oracle.OK
    info = h.update(np.array(src, np.int32), np.array(dst, np.int32), np.array(ins, np.uint8))
    cur = gg.apply_directed_batch(g, src, dst, ins)
    assert info.nnz == cur.nnz == g.nnz + len(src)
    _compare(h, s, k)


def test_directed_invalid_batches_change_nothing():
    g = gg.orient(gg.rmat(11, 8, seed=5), seed=2)
    D = g.deg_max() + 2
    h, s = _pair(g, 10, 1e-9, D)
    before = (h.ranking(10).copy(), *[x.copy() for x in h.bounds()[:2]])
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    arcs = set(zip(rows.tolist(), g.col.tolist()))
    a, b = next((x, y) for x, y in sorted(arcs) if (y, x) not in arcs)  # a one-way arc a -> b
    top = int(np.argmax(np.diff(g.rowptr)))
    outs = set(g.col[g.rowptr[top]:g.rowptr[top + 1]].tolist())
    others = [v for v in range(g.n) if v != top and v not in outs][:3]
    cases = [
        ([a], [b], [1], "KATZ_EINVAL"),                   # insert an existing arc
        ([b], [a], [0], "KATZ_EINVAL"),                   # delete an absent arc (its reverse exists)
        ([b, b], [a, a], [1, 1], "KATZ_EINVAL"),          # the same ordered pair twice
        ([a], [a], [1], "KATZ_EINVAL"),                   # self-loop
        ([top] * 3, others, [1, 1, 1], "KATZ_EALPHA"),    # out-degree of top would exceed D
    ]
    for src, dst, ins, name in cases:
        with pytest.raises(K.KatzError) as e:
            h.update(np.array(src, np.int32), np.array(dst, np.int32), np.array(ins, np.uint8))
        assert e.value.name == name
        assert s.apply_update(src, dst, ins) != oracle.OK
    after = (h.ranking(10), *h.bounds()[:2])
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    # in-arcs do not count toward the bound; b -> a is valid now
    src = [v for v in range(g.n) if v not in (top, b) and (v, top) not in arcs][:3]
    dst, ins = [top] * 3, [1, 1, 1]
    assert s.apply_update(src, dst, ins) == oracle.OK
    h.update(np.array(src, np.int32), np.array(dst, np.int32), np.array(ins, np.uint8))
    assert s.apply_update([b], [a], [1]) == oracle.OK
    h.update(np.array([b], np.int32), np.array([a], np.int32), np.array([1], np.uint8))
    _compare(h, s, 10)


def test_directed_small_frontier_follows_in_arcs():
    # a directed path 0 -> 1 -> ... -> n-1: an arc out of 100 changes s_i of
    # 100 - i + 1 only, so the frontier stays one node per level
    n = 5000
    g = gg.directed_from_arcs(n, np.arange(n - 1), np.arange(1, n))
    h, s = _pair(g, 5, 1e-6, 2)
    src, dst, ins = np.array([100], np.int32), np.array([300], np.int32), np.array([1], np.uint8)
    assert s.apply_update(src, dst, ins) == oracle.OK
    info = h.update(src, dst, ins)
    assert info.full_levels == 0 and 0 < info.affected <= info.r + 1
    _compare(h, s, 5)


def test_directed_large_frontier_switches_to_full_levels():
    g = gg.orient(gg.rmat(12, 16, seed=13), seed=4)
    D = g.deg_max() + 64
    h, s = _pair(g, 20, 1e-9, D)
    src, dst, ins = gg.directed_update_batch(g, 600, seed=6, deg_bound=D)
    assert s.apply_update(src, dst, ins) == oracle.OK
    info = h.update(src, dst, ins)
    assert info.full_levels > 0
    _compare(h, s, 20)


def test_directed_serving_matches_oracle():
    g = gg.orient(gg.rmat(13, 16, seed=31), seed=8)
    k, eps = 30, 1e-9
    D = g.deg_max() + 32
    h, s = _pair(g, k, eps, D)
    srv = K.Server(workers=1, slots=2, slot_updates=4096)
    srv.attach(h, k)
    cur, batches = g, []
    for j in range(4):
        b = gg.directed_update_batch(cur, [5, 500, 50, 3000][j], seed=900 + j, deg_bound=D)
        batches.append(b)
        cur = gg.apply_directed_batch(cur, *b)
    tickets = [srv.submit(h, *b) for b in batches]
    results = [srv.wait(t, timeout_ms=60000) for t in tickets]
    srv.close()
    for j, (status, ids, res) in enumerate(results):
        assert status == 0
        assert s.apply_update(*batches[j]) == oracle.OK
        assert res.info.r == s.info()["r"]
        c, l, u = s.bounds()
        assert_same_ranking(ids, s.ranking(), l)
    _compare(h, s, k)
    h.close()
