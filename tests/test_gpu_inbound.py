"""Inbound Katz (Sec. 2.1): omega_i(v) counts the walks of length i that end
at v, which is outbound Katz of the reverse graph.  A handle created with
inbound = 1 on a directed CSR reverses it on the device; it is compared with
the oracle run on the reverse graph (built on the host), statically, through
update batches (which name arcs of the graph as given), and through a
checkpoint round trip."""
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


def _opts(**kw):
    base = dict(undirected=0, inbound=1, keep_history=1, r_max=256)
    base.update(kw)
    return K.katz_default_opts(**base)


@pytest.mark.parametrize("on_device,locality", [(True, 0), (False, 0), (True, 1), (False, 1)])
def test_inbound_static_matches_oracle_on_the_reverse_graph(on_device, locality):
    g = gg.orient(gg.rmat(14, 16, seed=71), seed=3)
    rev = gg.reverse(g)
    assert not np.array_equal(rev.col, g.col)
    k, eps = 200, 1e-9
    ref = oracle.katz_static(rev.rowptr, rev.col, 0.0, k, eps, undirected=False, r_max=256)
    conv = _dev if on_device else np.ascontiguousarray
    h = K.Katz(conv(g.rowptr), conv(g.col), _opts(locality=locality))  # 1: anchor order of the reverse graph
    info = h.rank(0.0, k, eps)
    assert info.r == ref["r"] and info.converged == 1
    lo, up, _ = h.bounds()
    assert_close(lo, ref["l"], what="lower")
    assert_close(up, ref["u"], what="upper")
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"])
    # D is the largest in-degree of the graph as given
    assert abs(info.alpha - 1.0 / (rev.deg_max() + 1)) < 1e-15
    s = oracle.Session(rev.rowptr, rev.col, False)
    assert s.run_fixed(info.alpha, 4) == oracle.OK
    for i in range(1, 5):
        assert_close(h.walk(i), s.alpha_pow(i) * s.omega(i), what=f"s_{i}")
    h.close()


def test_inbound_fp32_certified_and_outbound_differ():
    g = gg.orient(gg.rmat(13, 16, seed=72), seed=5)
    rev = gg.reverse(g)
    k, eps = 100, 1e-9
    ref = oracle.katz_static(rev.rowptr, rev.col, 0.0, k, eps, undirected=False, r_max=256)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(precision=K.KATZ_FP32_CERT, keep_history=0))
    info = h.rank(0.0, k, eps)
    assert info.converged == 1
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"], atol=eps)
    out = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, undirected=False, r_max=256)
    assert list(out["ranking"]) != list(ref["ranking"])
    h.close()


def test_inbound_is_ignored_on_undirected_handles():
    g = gg.rmat(12, 16, seed=73)
    a = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(inbound=1))
    b = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts())
    a.rank(0.0, 50, 1e-9)
    b.rank(0.0, 50, 1e-9)
    np.testing.assert_array_equal(a.ranking(50), b.ranking(50))
    np.testing.assert_array_equal(a.bounds()[0], b.bounds()[0])


def test_inbound_updates_name_arcs_of_the_given_graph():
    g = gg.orient(gg.rmat(12, 16, seed=74), seed=6)
    rev = gg.reverse(g)
    D = rev.deg_max() + 16  # a bound on in-degrees of g
    k, eps = 50, 1e-9
    h = K.Katz(_dev(g.rowptr), _dev(g.col), _opts(deg_bound=D))
    h.rank(0.0, k, eps)
    s = oracle.Session(rev.rowptr, rev.col, False, D)
    assert s.rank_static(0.0, k, eps, 256) == oracle.OK
    cur = g
    for b, m in enumerate([1, 40, 800]):
        # drawn against the reverse graph (its out-degrees are g's in-degrees)
        rsrc, rdst, ins = gg.directed_update_batch(gg.reverse(cur), m, seed=300 + b, deg_bound=D)
        src, dst = rdst, rsrc  # the same arcs, as arcs of g
        assert s.apply_update(rsrc, rdst, ins) == oracle.OK
        info = h.update(src, dst, ins)
        cur = gg.apply_directed_batch(cur, src, dst, ins)
        assert info.r == s.info()["r"] and info.nnz == cur.nnz
        c, l, u = s.bounds()
        lo, up, _ = h.bounds()
        assert_close(lo, l, what="lower")
        assert_close(up, u, what="upper")
        assert_same_ranking(h.ranking(k), s.ranking(), l)
    # the handle's graph is the reverse of the updated graph
    t = oracle.Session(gg.reverse(cur).rowptr, gg.reverse(cur).col, False, D)
    assert t.run_fixed(s.info()["alpha"], s.info()["r"]) == oracle.OK
    assert_close(h.bounds()[0], t.bounds()[1], what="lower vs recompute")
    # a checkpoint keeps the orientation
    h2 = K.Katz.restore(h.checkpoint())
    rsrc, rdst, ins = gg.directed_update_batch(gg.reverse(cur), 30, seed=399, deg_bound=D)
    i1 = h.update(rdst, rsrc, ins)
    i2 = h2.update(rdst, rsrc, ins)
    assert i1.r == i2.r
    np.testing.assert_array_equal(h.ranking(k), h2.ranking(k))
    np.testing.assert_array_equal(h.bounds()[1], h2.bounds()[1])


def test_inbound_create_rejects_a_bad_column_entry():
    g = gg.orient(gg.rmat(10, 8, seed=75), seed=7)
    col = g.col.copy()
    col[len(col) // 2] = g.n  # out of range: caught before the reverse scatter
    with pytest.raises(K.KatzError) as e:
        K.Katz(_dev(g.rowptr), _dev(col), _opts())
    assert e.value.name == "KATZ_EINVAL"
    rp = g.rowptr.copy()
    rp[5] = rp[6] + 1  # offsets not monotone (host arrays this time)
    with pytest.raises(K.KatzError) as e:
        K.Katz(rp, g.col, _opts())
    assert e.value.name == "KATZ_EINVAL"
