"""The seeded generators produce valid symmetric CSR graphs (CPU only)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check(g):
    n = g.n
    assert g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) >= 0) and g.rowptr[-1] == g.nnz
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    assert np.all(g.col >= 0) and np.all(g.col < n)
    assert not np.any(rows == g.col), "self-loop"
    key = rows.astype(np.int64) * n + g.col
    assert np.all(np.diff(key) > 0), "rows sorted, no duplicates"
    rkey = g.col.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(rkey), key), "symmetric"


def test_er_exact_edge_count():
    g = gg.erdos_renyi(16384, 131072, seed=gg.SEED_BASE)
    _check(g)
    assert g.nnz == 2 * 131072


@pytest.mark.parametrize("scale", [8, 12])
def test_rmat_valid(scale):
    g = gg.rmat(scale, 16, seed=3)
    _check(g)
    assert g.nnz <= 2 * 16 * (1 << scale)
    d = g.degrees()
    assert d.max() > 5 * max(1.0, d.mean())  # skewed


def test_chung_lu_valid():
    g = gg.chung_lu(1 << 14, 16.0, 2.1, seed=5)
    _check(g)
    assert 4.0 < g.nnz / g.n < 40.0


def test_generators_independent_of_thread_count():
    code = ("import graphgen as gg, hashlib; g = gg.rmat(12, 16, seed=9); c = gg.chung_lu(4096, seed=9);"
            "print(hashlib.sha1(g.col.tobytes() + c.col.tobytes()).hexdigest())")
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t, PYTHONPATH=ROOT)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=ROOT).strip())
    assert outs[0] == outs[1]


def test_update_batch_preconditions():
    g = gg.rmat(10, 8, seed=1)
    src, dst, ins = gg.update_batch(g, 200, seed=2)
    assert len(src) == 200
    for a, b, i in zip(src, dst, ins):
        present = b in g.col[g.rowptr[a]:g.rowptr[a + 1]]
        assert present != bool(i) and a != b
    pairs = {(min(a, b), max(a, b)) for a, b in zip(src, dst)}
    assert len(pairs) == 200
    g2 = gg.apply_batch(g, src, dst, ins)
    _check(g2)
    assert g2.nnz == g.nnz + 2 * int(ins.sum()) - 2 * int((1 - ins).sum())


def test_stream_batches_are_valid_against_the_evolving_graph():
    g = gg.rmat(10, 8, seed=3)
    D = g.deg_max() + 4
    st = gg.stream(g, 40, seed=7, max_size=300, rate=200.0, deg_bound=D)
    sizes = st.sizes()
    assert len(st) == 40 and sizes.min() >= 1 and sizes.max() <= 300
    assert np.all(np.diff(st.arrival) > 0) and st.arrival[0] > 0
    again = gg.stream(g, 40, seed=7, max_size=300, rate=200.0, deg_bound=D)
    assert np.array_equal(st.src, again.src) and np.array_equal(st.is_insert, again.is_insert)
    cur = g
    for j in range(len(st)):
        src, dst, ins = st.batch(j)
        pairs = set()
        for a, b, i in zip(src.tolist(), dst.tolist(), ins.tolist()):
            assert a != b
            key = (min(a, b), max(a, b))
            assert key not in pairs
            pairs.add(key)
            present = b in cur.col[cur.rowptr[a]:cur.rowptr[a + 1]]
            assert present != bool(i), (j, a, b, i)
        cur = gg.apply_batch(cur, src, dst, ins)
        assert cur.deg_max() <= D
    # both kinds of update occur, and the mean gap matches the rate
    assert 0 < st.is_insert.mean() < 1
    assert 0.002 < st.arrival[-1] / len(st) < 0.01


def test_directed_helpers_make_valid_graphs_and_batches():
    g = gg.orient(gg.rmat(10, 8, seed=4), seed=9)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    arcs = set(zip(rows.tolist(), g.col.tolist()))
    assert all(a != b for a, b in arcs) and len(arcs) == g.nnz
    assert any((b, a) not in arcs for a, b in arcs)  # not symmetric
    assert any((b, a) in arcs for a, b in arcs)      # some edges reciprocal
    for r in range(g.n):
        row = g.col[g.rowptr[r]:g.rowptr[r + 1]]
        assert np.all(np.diff(row) > 0)
    D = g.deg_max() + 2
    cur = g
    for j in range(5):
        src, dst, ins = gg.directed_update_batch(cur, 200, seed=j, deg_bound=D)
        assert len(src) == 200 and 0 < ins.mean() < 1
        seen = set()
        cur_rows = np.repeat(np.arange(cur.n), np.diff(cur.rowptr))
        cur_arcs = set(zip(cur_rows.tolist(), cur.col.tolist()))
        for a, b, i in zip(src.tolist(), dst.tolist(), ins.tolist()):
            assert a != b and (a, b) not in seen
            seen.add((a, b))
            assert ((a, b) in cur_arcs) != bool(i)
        nxt = gg.apply_directed_batch(cur, src, dst, ins)
        assert nxt.nnz == cur.nnz + int(ins.sum()) - int((1 - ins).sum())
        assert nxt.deg_max() <= max(D, cur.deg_max())
        cur = nxt


def test_band_union_pads_to_an_exact_size():
    """The padding graph is symmetric, sorted, free of self-loops and
    duplicates, leaves the base graph's rows unchanged, and lands n + nnz on
    the requested total."""
    base = gg.chung_lu(2000, 8.0, 2.1, seed=9)
    for extra, d in ((7, 4), (5000, 4), (123457, 16)):
        g = gg.padded_to(base, base.n + base.nnz + extra, d=d)
        assert g.n + g.nnz == base.n + base.nnz + extra
        assert np.array_equal(g.rowptr[:base.n + 1], base.rowptr)
        assert np.array_equal(g.col[:base.nnz], base.col)
        rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        assert np.all(rows != g.col)
        keys = rows.astype(np.int64) * g.n + g.col
        assert np.all(np.diff(keys) > 0)  # rows sorted, no duplicates
        rev = g.col.astype(np.int64) * g.n + rows
        assert np.array_equal(np.sort(rev), keys)  # symmetric
        assert int(np.diff(g.rowptr)[base.n:].max(initial=0)) <= 2 * d
