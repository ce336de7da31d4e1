"""Checkpoint and restore (katz_checkpoint / katz_restore): a restored handle
holds the same ranking, bounds and walk history and continues exactly like
the original through later update batches and rankings."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(a, b, k, walks=()):
    np.testing.assert_array_equal(a.ranking(k), b.ranking(k))
    la, ua, _ = a.bounds()
    lb, ub, _ = b.bounds()
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(ua, ub)
    for i in walks:
        np.testing.assert_array_equal(a.walk(i), b.walk(i))


def test_restored_handle_continues_like_the_original():
    g = gg.rmat(13, 16, seed=51)
    D, k = g.deg_max() + 32, 64
    st = gg.stream(g, 3, seed=52, max_size=500, deg_bound=D)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(keep_history=1, deg_bound=D))
    info = h.rank(0.0, k, 1e-9)
    h.update(*st.batch(0))
    image = h.checkpoint()
    h2 = K.Katz.restore(image)
    assert h2.n == g.n
    _same(h, h2, k, walks=range(1, info.r + 1))
    for j in (1, 2):  # the same later batches on both
        i1 = h.update(*st.batch(j))
        i2 = h2.update(*st.batch(j))
        assert i1.r == i2.r
        _same(h, h2, k)
    h.close()
    h2.rank(0.0, k, 1e-9)  # and it ranks from scratch on its own
    h2.close()


def test_checkpoint_of_fp32_and_ranking_criterion_handles():
    g = gg.rmat(12, 16, seed=53)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(precision=K.KATZ_FP32_CERT))
    h.rank(0.0, 50, 1e-9)
    h2 = K.Katz.restore(h.checkpoint())
    _same(h, h2, 50)
    h.close()
    h2.close()
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    h.rank_by(K.KATZ_CRIT_RANKING, eps=1e-7)
    h2 = K.Katz.restore(h.checkpoint())
    _same(h, h2, g.n)
    h.close()
    h2.close()


def test_bad_images_are_rejected():
    g = gg.rmat(10, 8, seed=54)
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    with pytest.raises(K.KatzError) as e:  # nothing ranked yet
        h.checkpoint()
    assert e.value.name == "KATZ_ESTATE"
    h.rank(0.0, 10, 1e-9)
    image = h.checkpoint()
    for bad in (image[:-1], image[:100], np.concatenate([image, np.zeros(1, np.uint8)])):
        with pytest.raises(K.KatzError) as e:
            K.Katz.restore(bad)
        assert e.value.name == "KATZ_EINVAL"
    broken = image.copy()
    broken[0] ^= 1  # magic
    with pytest.raises(K.KatzError):
        K.Katz.restore(broken)
    h.close()
