"""The int64 row-offset instantiation of every kernel, on graphs small enough
for complete oracle runs: a handle created with katz_opts.offsets64 = 1 keeps
64-bit offsets (the layout a graph with n + nnz >= 2^31 - 1 gets, such as the
Chung-Lu n = 2^27 workload).  Static FP64 ranking (Algorithm 1), the
FP32-certified mode, the other criteria, directed graphs, update batches
(Algorithm 2) and a checkpoint round trip, each against the oracle."""
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


def _handle(g, **kw):
    kw.setdefault("r_max", 256)
    return K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(offsets64=1, **kw))


@pytest.mark.parametrize("graph,k", [("rmat15", 300), ("chunglu", 100)])
def test_static_fp64_matches_the_oracle(graph, k):
    g = gg.rmat(15, 16, seed=61) if graph == "rmat15" else gg.chung_lu(1 << 16, 16.0, 2.1, seed=62)
    eps = 1e-9
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, r_max=256)
    for use_graph in (1, 0):  # device-side loop and the host loop the benchmark times
        h = _handle(g, keep_history=1, use_graph=use_graph, profile=1 - use_graph)
        info = h.rank(0.0, k, eps)
        assert info.r == ref["r"] and info.converged == 1 and info.alpha == ref["alpha"]
        assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"])
        lo, up, _ = h.bounds()
        assert_close(lo, ref["l"], what="lower")
        assert_close(up, ref["u"], what="upper")
        s = ref["session"]
        for i in range(1, info.r + 1):
            assert_close(h.walk(i), s.alpha_pow(i) * s.omega(i), what=f"s_{i}")
        assert h.trace()[info.r - 1] == ref["active"]
        h.close()


def test_fp32_certified_matches_the_oracle():
    g = gg.chung_lu(1 << 16, 16.0, 2.1, seed=63)
    k, eps = 100, 1e-9
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, r_max=256)
    h = _handle(g, precision=K.KATZ_FP32_CERT)
    info = h.rank(0.0, k, eps)
    assert info.converged == 1 and info.fp32_levels > 0
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"], atol=eps)
    lo, up, err = h.bounds()
    s = oracle.Session(g.rowptr, g.col, True)
    assert s.run_fixed(0.0, info.r) == oracle.OK  # the oracle's bounds at the same r
    _, l_ref, u_ref = s.bounds()
    assert np.all(np.abs(lo - l_ref) <= err + 1e-12 * np.abs(l_ref) + 1e-300)
    assert np.all(np.abs(up - u_ref) <= err + 1e-12 * np.abs(u_ref) + 1e-300)
    h.close()


def test_ranking_criterion_matches_the_oracle():
    g = gg.rmat(11, 8, seed=64)
    eps = 1e-7
    s = oracle.Session(g.rowptr, g.col, True)
    assert s.rank(0.0, oracle.RANKING, eps) == oracle.OK
    h = _handle(g)
    info = h.rank_by(K.KATZ_CRIT_RANKING, eps=eps)
    assert info.r == s.info()["r"]
    _, l_ref, _ = s.bounds()
    assert_same_ranking(h.ranking(g.n), s.ranking(), l_ref)
    h.close()


@pytest.mark.parametrize("precision", [K.KATZ_FP64, K.KATZ_FP32_CERT])
def test_update_batches_match_the_oracle_session(precision):
    g = gg.rmat(13, 16, seed=65)
    k, eps = 50, 1e-9
    D = g.deg_max() + 16
    st = gg.stream(g, 4, seed=66, min_size=1, max_size=2000, deg_bound=D)
    h = _handle(g, keep_history=1, deg_bound=D, r_max=128, precision=precision)
    h.rank(0.0, k, eps)
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps, 128) == oracle.OK
    for j in range(len(st)):
        info = h.update(*st.batch(j))
        assert s.apply_update(*st.batch(j)) == oracle.OK
        _, l_ref, u_ref = s.bounds()
        if precision == K.KATZ_FP64:
            assert info.r == s.info()["r"]
            assert_same_ranking(h.ranking(k), s.ranking(), l_ref)
            lo, up, _ = h.bounds()
            assert_close(lo, l_ref, what=f"lower after batch {j}")
            assert_close(up, u_ref, what=f"upper after batch {j}")
        else:
            assert info.converged == 1
            assert_same_ranking(h.ranking(k), s.ranking(), l_ref, atol=eps)
    # a checkpoint of the int64-offset handle restores and continues
    h2 = K.Katz.restore(h.checkpoint())
    np.testing.assert_array_equal(h2.ranking(k), h.ranking(k))
    h2.close()
    h.close()


def test_directed_update_batches_match_the_oracle_session():
    g = gg.orient(gg.rmat(12, 16, seed=67), seed=68)
    k, eps = 40, 1e-9
    D = int(np.diff(g.rowptr).max()) + 8
    h = _handle(g, undirected=0, keep_history=1, deg_bound=D, r_max=128)
    h.rank(0.0, k, eps)
    s = oracle.Session(g.rowptr, g.col, False, D)
    assert s.rank_static(0.0, k, eps, 128) == oracle.OK
    cur = g
    for j, m in enumerate((5, 300)):
        src, dst, ins = gg.directed_update_batch(cur, m, seed=69 + j, deg_bound=D)
        info = h.update(src, dst, ins)
        assert s.apply_update(src, dst, ins) == oracle.OK
        cur = gg.apply_directed_batch(cur, src, dst, ins)
        assert info.r == s.info()["r"]
        _, l_ref, u_ref = s.bounds()
        assert_same_ranking(h.ranking(k), s.ranking(), l_ref)
        lo, up, _ = h.bounds()
        assert_close(lo, l_ref, what=f"lower after batch {j}")
        assert_close(up, u_ref, what=f"upper after batch {j}")
    h.close()
