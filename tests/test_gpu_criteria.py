"""The ranking, score and pair criteria of Sec. 3.1 (katz_rank) against the
oracle: same r, same certified order (ranking: all n nodes, up to ties closer
than eps; pair: the two nodes), bounds within 1e-12."""
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


def _pair_up(g, criterion, eps, pair=None, r_max=256):
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(r_max=r_max))
    info = h.rank_by(criterion, eps=eps, pair=pair)
    s = oracle.Session(g.rowptr, g.col)
    assert s.rank(0.0, criterion, eps, pair=pair if pair is not None else (0, 1), r_max=r_max) == oracle.OK
    assert info.r == s.info()["r"], (info.r, s.info()["r"])
    assert info.converged == 1
    lo, up, _ = h.bounds()
    c, l, u = s.bounds()
    assert_close(lo, l, what="lower")
    assert_close(up, u, what="upper")
    return h, info, s, l


@pytest.mark.parametrize("graph", ["er", "rmat12", "rmat15"])
def test_ranking_criterion_orders_every_node_like_the_oracle(graph):
    g = {"er": lambda: gg.erdos_renyi(3000, 12000, seed=71), "rmat12": lambda: gg.rmat(12, 16, seed=72),
         "rmat15": lambda: gg.rmat(15, 16, seed=73)}[graph]()
    eps = 1e-7
    h, info, s, l = _pair_up(g, K.KATZ_CRIT_RANKING, eps)
    assert info.k == g.n
    full = h.ranking(g.n)
    assert sorted(full.tolist()) == list(range(g.n))   # a permutation
    assert_same_ranking(full, s.ranking(), l, atol=eps)
    h.close()


@pytest.mark.parametrize("seed", range(3))
def test_score_criterion_like_the_oracle(seed):
    g = gg.rmat(13, 8, seed=80 + seed)
    h, info, s, l = _pair_up(g, K.KATZ_CRIT_SCORE, 1e-8)
    lo, up, _ = h.bounds()
    assert np.all(up - lo < 1e-8)
    with pytest.raises(K.KatzError) as e:
        h.ranking(1)
    assert e.value.name == "KATZ_ESTATE"
    h.close()


@pytest.mark.parametrize("seed", range(4))
def test_pair_criterion_like_the_oracle(seed):
    g = gg.rmat(13, 16, seed=90 + seed)
    rng = np.random.default_rng(seed)
    deg = np.diff(g.rowptr)
    cand = np.nonzero(deg > 0)[0]
    a, b = (int(x) for x in rng.choice(cand, 2, replace=False))
    h, info, s, l = _pair_up(g, K.KATZ_CRIT_PAIR, 1e-9, pair=(a, b))
    assert list(h.ranking(2)) == list(s.ranking())
    h.close()


def test_criterion_argument_errors():
    g = gg.rmat(10, 8, seed=3)
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    for bad in [dict(criterion=7), dict(criterion=K.KATZ_CRIT_PAIR, pair=(1, 1)),
                dict(criterion=K.KATZ_CRIT_PAIR, pair=(0, g.n))]:
        with pytest.raises(K.KatzError) as e:
            h.rank_by(bad.pop("criterion"), **bad)
        assert e.value.name == "KATZ_EINVAL"
    h.rank_by(K.KATZ_CRIT_RANKING, eps=1e-6)
    with pytest.raises(K.KatzError) as e:  # updates continue the top-k criterion only
        h.update(np.array([0], np.int32), np.array([1], np.int32), np.array([1], np.uint8))
    assert e.value.name == "KATZ_ESTATE"
    h.close()
    h32 = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(precision=K.KATZ_FP32_CERT))
    with pytest.raises(K.KatzError) as e:
        h32.rank_by(K.KATZ_CRIT_SCORE, eps=1e-6)
    assert e.value.name == "KATZ_ESTATE"
    h32.close()
