"""Checkpoint and restore (katz_checkpoint / katz_restore): a restored handle
holds the same ranking, bounds and walk history, continues exactly like the
original through later update batches and rankings, and after each batch
agrees with the oracle session fed the same batches (Sec. 4: the state kept
between batches).  Corrupted images are refused before any kernel runs."""
from __future__ import annotations

import ctypes

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
    s = oracle.Session(g.rowptr, g.col, True, D)  # the oracle session, fed the same batches
    assert s.rank_static(0.0, k, 1e-9, 256) == oracle.OK
    assert s.apply_update(*st.batch(0)) == oracle.OK
    for j in (1, 2):  # the same later batches on both
        i1 = h.update(*st.batch(j))
        i2 = h2.update(*st.batch(j))
        assert i1.r == i2.r
        _same(h, h2, k)
        assert s.apply_update(*st.batch(j)) == oracle.OK
        assert i2.r == s.info()["r"]
        _, l_ref, u_ref = s.bounds()
        assert_same_ranking(h2.ranking(k), s.ranking(), l_ref)
        lo, up, _ = h2.bounds()
        assert_close(lo, l_ref, what=f"lower after batch {j}")
        assert_close(up, u_ref, what=f"upper after batch {j}")
    s.close()
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


def _rowptr_offset(image, n, nnz):
    """Byte offset of the int32 row offsets in an image (header and trace come
    first): the first place where n + 1 monotone int32 values run from 0 to nnz."""
    for o in range(0, 8192, 4):
        rp = image[o:o + 4 * (n + 1)].view(np.int32)
        if rp.shape[0] == n + 1 and rp[0] == 0 and rp[-1] == nnz and np.all(np.diff(rp) >= 0):
            return o
    raise AssertionError("row offsets not found")


def test_corrupted_images_are_refused():
    """A bit-flipped image of the right length is refused with KATZ_EINVAL, as
    katz_create_csr refuses the same input: a column entry out of range, a
    row offset out of order, and header fields that disagree with the arrays."""
    g = gg.rmat(11, 8, seed=55)
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    h.rank(0.0, 20, 1e-9)
    image = h.checkpoint()
    h.close()
    K.Katz.restore(image).close()  # the intact image restores
    o_rp = _rowptr_offset(image, g.n, g.nnz)
    o_col = o_rp + 4 * (g.n + 1)
    hdr = 16 + ctypes.sizeof(K.katz_opts)  # magic, version, sizes, the creation options; then the int64 fields
    fields = {"n": 0, "nnz": 1, "D": 2, "deg_max": 3, "stride": 4, "k_eff": 5, "row_warp": 6, "row_octet": 7,
              "row_thread": 8, "chunks": 9}
    assert image[hdr:hdr + 8].view(np.int64)[0] == g.n
    bad = []
    b = image.copy()
    b[o_col:o_col + 4] = np.array([g.n], np.int32).view(np.uint8)  # col[0] = n
    bad.append(b)
    b = image.copy()
    b[o_col + 40:o_col + 44] = np.array([-1], np.int32).view(np.uint8)  # a negative column id
    bad.append(b)
    b = image.copy()
    mid = o_rp + 4 * (g.n // 2)
    b[mid:mid + 4] = np.array([g.nnz + 5], np.int32).view(np.uint8)  # offsets out of order
    bad.append(b)
    for name, val in (("k_eff", g.n + 1), ("D", 0), ("row_octet", g.n + 1), ("stride", g.n)):
        b = image.copy()
        o = hdr + 8 * fields[name]
        b[o:o + 8] = np.array([val], np.int64).view(np.uint8)
        bad.append(b)
    for b in bad:
        with pytest.raises(K.KatzError) as e:
            K.Katz.restore(b)
        assert e.value.name == "KATZ_EINVAL"
