"""The benchmark configurations at full size, in the launch configuration
bench.py times (profiled host loop, two walk slots unless history is needed):

- R-MAT24 (FP64 and FP32-certified) against a complete oracle run;
- Chung-Lu n = 2^27 (int64 offsets) by checks that hold at any size: sampled
  rows of s_r recomputed on the host from the device's own s_{r-1} (Eq. 5),
  l <= u, and the top-k criterion re-checked on the host from the returned
  bounds; FP32-certified against FP64 up to eps;
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


def test_chunglu27_top100_by_properties():
    g = gg.workload("chunglu27")
    assert g.n + g.nnz >= 0x7fffffff  # int64 offsets
    k, eps = 100, 1e-9
    rng = np.random.default_rng(27)
    h, info = _rank(g, k, eps)
    assert info.converged == 1
    lo, up, _ = h.bounds()
    assert np.all(lo <= up)
    ranking = h.ranking(k)
    _topk_certified(lo, up, ranking, eps)
    _sampled_rows_exact(g, h, info, rng)
    h.close()
    h32, info32 = _rank(g, k, eps, precision=1)
    assert info32.converged == 1
    assert_same_ranking(h32.ranking(k), ranking, lo, atol=eps)
    h32.close()


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
