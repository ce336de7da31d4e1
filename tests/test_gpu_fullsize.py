"""The benchmark configurations at full size, in the launch configuration
bench.py times (profiled host loop, two walk slots unless history is needed):

- R-MAT24 (FP64 and FP32-certified) against a complete oracle run;
- Chung-Lu n = 2^27 (int64 offsets) against a complete oracle run: the same
  r, ranking and per-node bounds in FP64; the FP32-certified ranking up to
  eps, each node's bounds within the reported widening of the oracle's at the
  same r; plus checks that hold at any size (sampled rows of s_r recomputed
  from the device's own s_{r-1}, Eq. 5; the top-k criterion re-checked on the
  host from the returned bounds);
- a graph just below the range of 32-bit row offsets and update batches that
  take it past that range (the handle moves to int64 offsets) and back,
  against the oracle session;
- the R-MAT23 serving stream: a few batches through katz_server against the
  oracle session fed the same batches.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.parity import assert_close, assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _rank(g, k, eps, precision=0, keep_history=0, D=0):
    opts = K.katz_default_opts(precision=precision, profile=1, keep_history=keep_history, deg_bound=D, r_max=256)
    h = K.Katz(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(), opts)
    info = h.rank(0.0, k, eps)
    return h, info


def _sampled_rows_exact(g, h, info, rng, rows=2000):
    """s_r(v) = alpha * sum_{v->x} s_{r-1}(x) for sampled v: the device's row
    sums are correctly rounded, so alpha * fsum(...) matches to an ulp or two."""
    r = info.r
    s_prev, s_cur = h.walk(r - 1), h.walk(r)
    deg = np.diff(g.rowptr)
    pick = np.concatenate([rng.integers(0, g.n, rows), np.argpartition(deg, -50)[-50:]])
    for v in pick.tolist():
        nb = g.col[g.rowptr[v]:g.rowptr[v + 1]]
        want = info.alpha * math.fsum(s_prev[nb].tolist())
        got = s_cur[v]
        assert abs(got - want) <= 4 * np.spacing(abs(want)) + 0.0, (v, got, want)


def _topk_certified(lo, up, ranking, eps):
    """The top-k criterion on the returned bounds: adjacent top-k pairs and the
    k-th node against every other node are eps-separated (Eq. 3)."""
    top = np.asarray(ranking, np.int64)
    lt, ut = lo[top], up[top]
    assert np.all(lt[:-1] >= lt[1:])
    assert np.all(ut[1:] - eps < lt[:-1])
    theta = lt[-1]
    rest = np.ones(len(lo), bool)
    rest[top] = False
    gap = (up[rest] - eps) - theta
    # nodes dropped at an earlier level met the test with their bounds then;
    # the final bounds are tighter up to rounding
    assert gap.max() < 1e-15 * max(theta, 1.0), gap.max()


def test_rmat24_top1000_against_the_oracle():
    g = gg.workload("rmat24")
    k, eps = 1000, 1e-9
    oracle.set_threads(0)
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, r_max=256)
    h, info = _rank(g, k, eps)
    assert info.r == ref["r"] and info.converged == 1
    lo, up, _ = h.bounds()
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"])
    assert_close(lo, ref["l"], what="lower")
    assert_close(up, ref["u"], what="upper")
    h.close()
    # FP32-certified: the same certified order up to eps
    h, info = _rank(g, k, eps, precision=1)
    assert info.converged == 1 and info.fp32_levels > 0
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"], atol=eps)
    h.close()


def test_chunglu27_top100_against_the_oracle():
    g = gg.workload("chunglu27")
    assert g.n + g.nnz >= 0x7fffffff  # int64 offsets
    k, eps = 100, 1e-9
    rng = np.random.default_rng(27)
    oracle.set_threads(0)
    s = oracle.Session(g.rowptr, g.col, True)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    ref = s.info()
    _, l_ref, u_ref = s.bounds()
    ranking_ref = s.ranking()
    h, info = _rank(g, k, eps)
    assert info.converged == 1 and info.r == ref["r"] and info.alpha == ref["alpha"]
    lo, up, _ = h.bounds()
    ranking = h.ranking(k)
    assert_same_ranking(ranking, ranking_ref, l_ref)
    assert_close(lo, l_ref, what="lower")
    assert_close(up, u_ref, what="upper")
    _topk_certified(lo, up, ranking, eps)
    _sampled_rows_exact(g, h, info, rng)
    h.close()
    h32, info32 = _rank(g, k, eps, precision=1)
    assert info32.converged == 1 and info32.fp32_levels > 0
    assert_same_ranking(h32.ranking(k), ranking_ref, l_ref, atol=eps)
    lo32, up32, err = h32.bounds()
    h32.close()
    if info32.r != ref["r"]:  # the oracle's bounds at the FP32 run's r
        assert s.run_fixed(0.0, info32.r) == oracle.OK
        _, l_ref, u_ref = s.bounds()
    assert np.all(np.abs(lo32 - l_ref) <= err + 1e-12 * np.abs(l_ref) + 1e-300)
    assert np.all(np.abs(up32 - u_ref) <= err + 1e-12 * np.abs(u_ref) + 1e-300)
    s.close()


def test_batches_across_the_int32_offset_limit():
    """A graph with n + nnz 64 below 2^31 - 1 (the largest value 32-bit row
    offsets reach): a Chung-Lu graph of 2^20 nodes padded by a band graph.
    The first batch inserts 100 edges and takes the handle past the limit
    (it moves to int64 offsets); the second deletes edges and inserts others
    on the int64 handle.  After each batch: the oracle session's r, ranking
    and bounds."""
    base = gg.chung_lu(1 << 20, 16.0, 2.1, seed=gg.SEED_BASE + 31)
    g = gg.padded_to(base, 0x7fffffff - 64)
    assert g.n + g.nnz < 0x7fffffff  # created with int32 offsets
    k, eps, r_max = 20, 1e-9, 64
    D = g.deg_max() + 64
    oracle.set_threads(0)
    h, info = _rank(g, k, eps, keep_history=1, D=D)
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps, r_max) == oracle.OK
    assert info.r == s.info()["r"]
    ins1 = gg.update_batch(g, 100, seed=gg.SEED_BASE + 32, p_insert=1.0)
    dels = gg.update_batch(g, 300, seed=gg.SEED_BASE + 33, p_insert=0.0)  # edges of g, kept by batch 1
    more = gg.update_batch(g, 200, seed=gg.SEED_BASE + 34, p_insert=1.0)
    taken = set(zip(np.minimum(ins1[0], ins1[1]).tolist(), np.maximum(ins1[0], ins1[1]).tolist()))
    keep = np.array([(min(a, b), max(a, b)) not in taken for a, b in zip(more[0], more[1])], bool)
    batch2 = tuple(np.concatenate([dels[q], more[q][keep]]) for q in range(3))
    for j, batch in enumerate((ins1, batch2)):
        inf = h.update(*batch)
        assert s.apply_update(*batch) == oracle.OK
        assert inf.r == s.info()["r"]
        _, l_ref, u_ref = s.bounds()
        assert_same_ranking(h.ranking(k), s.ranking(), l_ref)
        lo, up, _ = h.bounds()
        assert_close(lo, l_ref, what=f"lower after batch {j}")
        assert_close(up, u_ref, what=f"upper after batch {j}")
    h.close()
    s.close()


def test_rmat23_serving_stream_against_the_oracle_session():
    g = gg.workload("rmat23")
    D = g.deg_max() + 64
    k, eps = 100, 1e-9
    st = gg.stream(g, 3, seed=gg.SEED_BASE + 230, deg_bound=D)
    h, info = _rank(g, k, eps, keep_history=1, D=D)
    srv = K.Server(workers=2, slots=4, slot_updates=10000)
    srv.attach(h, k)
    tickets = [srv.submit(h, *st.batch(j)) for j in range(len(st))]
    results = [srv.wait(t, timeout_ms=120000) for t in tickets]
    srv.close()
    oracle.set_threads(0)
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    for j, (status, ids, res) in enumerate(results):
        assert status == 0
        assert s.apply_update(*st.batch(j)) == oracle.OK
        assert res.info.r == s.info()["r"], (j, res.info.r, s.info()["r"])
        c, l, u = s.bounds()
        assert_same_ranking(ids, s.ranking(), l)
    lo, up, _ = h.bounds()
    c, l, u = s.bounds()
    assert_close(lo, l, what="lower after the stream")
    assert_close(up, u, what="upper after the stream")
    h.close()
