"""Parity of the CUDA static path (Algorithm 1) with the CPU oracle, through
the C ABI.  FP64 mode: same iteration count r, same certified ranking (up to
rounding-level ties), and omega_i, l_r, u_r within 1e-12 relative."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.parity import REL_TOL, assert_close, assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(g, alpha, k, eps, *, undirected=True, keep_history=True, r_max=256, on_device=True, use_graph=1,
            precision=0, profile=0, locality=0):
    opts = K.katz_default_opts(undirected=1 if undirected else 0, keep_history=1 if keep_history else 0,
                               r_max=r_max, use_graph=use_graph, precision=precision, profile=profile,
                               locality=locality)
    rp, cl = (_dev(g.rowptr), _dev(g.col)) if on_device else (g.rowptr, g.col)
    h = K.Katz(rp, cl, opts)
    info = h.rank(alpha, k, eps)
    kk = min(k, g.n)
    out = dict(info=info, ranking=h.ranking(kk))
    out["l"], out["u"], out["err"] = h.bounds()
    if keep_history:
        out["walks"] = [h.walk(i) for i in range(1, info.r + 1)]
    out["trace"] = h.trace()[: info.r]
    h.close()
    return out


def run_oracle(g, alpha, k, eps, undirected=True):
    return oracle.katz_static(g.rowptr, g.col, alpha, k, eps, undirected=undirected, r_max=256)


def check_parity(g, alpha, k, eps, undirected=True, walks=True, **kw):
    ref = run_oracle(g, alpha, k, eps, undirected)
    got = run_gpu(g, alpha, k, eps, undirected=undirected, keep_history=walks, **kw)
    assert got["info"].r == ref["r"], (got["info"].r, ref["r"])
    assert got["info"].converged == 1
    assert got["info"].alpha == ref["alpha"]
    assert_same_ranking(got["ranking"], ref["ranking"], ref["l"])
    assert_close(got["l"], ref["l"], what="lower")
    assert_close(got["u"], ref["u"], what="upper")
    if walks:
        s = ref["session"]
        for i in range(1, ref["r"] + 1):
            expect = s.alpha_pow(i) * s.omega(i)
            assert_close(got["walks"][i - 1], expect, what=f"s_{i}")
    # |M| after each iteration matches the oracle's active set size at the end
    assert got["trace"][-1] == ref["active"]
    return got, ref


def test_er_16k_top100():
    g = gg.workload("er16k")
    got, ref = check_parity(g, 0.0, 100, 1e-9)
    assert ref["r"] > 5


@pytest.mark.parametrize("scale,k", [(12, 10), (14, 100), (16, 1000), (16, 1)])
def test_rmat_parity(scale, k):
    g = gg.rmat(scale, 16, seed=scale)
    check_parity(g, 0.0, k, 1e-9)


def test_rmat_alpha_half_inverse_degree():
    g = gg.rmat(14, 16, seed=5)
    check_parity(g, 0.5 / g.deg_max(), 100, 1e-9)


@pytest.mark.parametrize("graph", ["complete", "star", "path", "isolated", "single"])
def test_small_and_degenerate_graphs(graph):
    if graph == "complete":
        g = gg.complete(9)        # every node ties (Lemma 3)
        k = 4
    elif graph == "star":
        g = gg.star(5000)         # centre row spans several merge-path tiles
        k = 3
    elif graph == "path":
        g = gg.path(1000)
        k = 20
    elif graph == "isolated":
        g = gg.from_edges(300, np.array([0, 1, 2]), np.array([1, 2, 3]))
        k = 10
    else:
        g = gg.Graph(np.zeros(2, np.int64), np.zeros(0, np.int32), "single")
        k = 1
    check_parity(g, 0.0, k, 1e-6)


@pytest.mark.parametrize("k,use_graph", [(50, 1), (50, 0), (3000, 1), (K.KATZ_MAX_K, 0)])
def test_many_ties_take_the_large_candidate_path(k, use_graph):
    # every node has the same bounds: the candidate set is V, larger than the
    # one-CTA sort holds, and the select kernel narrows it on the device
    g = gg.cycle(20000)
    check_parity(g, 0.0, k, 1e-6, walks=False, use_graph=use_graph)


def test_k_at_least_n():
    g = gg.erdos_renyi(500, 2000, seed=3)
    check_parity(g, 0.0, 5000, 1e-9)


def test_directed_graph():
    rng = np.random.default_rng(11)
    n = 3000
    src = rng.integers(0, n, 20000)
    dst = rng.integers(0, n, 20000)
    keep = src != dst
    key = np.unique(src[keep].astype(np.int64) * n + dst[keep])
    s, d = key // n, key % n
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, s + 1, 1)
    rowptr = np.cumsum(rowptr)
    g = gg.Graph(rowptr, d.astype(np.int32), "directed")
    check_parity(g, 0.0, 30, 1e-9, undirected=False)


def test_host_pointers_and_host_loop():
    g = gg.rmat(12, 16, seed=21)
    check_parity(g, 0.0, 50, 1e-9, on_device=False, use_graph=0)


def test_r_max_reports_not_converged():
    g = gg.rmat(12, 16, seed=4)
    opts = K.katz_default_opts(r_max=2)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(0.0, 100, 1e-12, check=False)
    assert info.status == 5 and info.r == 2 and info.converged == 0  # KATZ_ENOTCONV
    s = oracle.Session(g.rowptr, g.col)
    s.run_fixed(info.alpha, 2)
    _, l, u = s.bounds()
    lo, up, _ = h.bounds()
    assert_close(lo, l, what="lower at r_max")
    assert_close(up, u, what="upper at r_max")


def test_argument_errors():
    g = gg.star(10)
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    with pytest.raises(K.KatzError) as e:
        h.rank(0.1, 3, 1e-9)  # alpha * deg_max = 1
    assert e.value.name == "KATZ_EALPHA"
    for alpha, k, eps in [(0.0, 0, 1e-9), (0.0, 3, 0.0), (0.0, 3, -1.0), (0.0, K.KATZ_MAX_K + 1, 1e-9)]:
        gg_big = g if k <= g.n else gg.cycle(K.KATZ_MAX_K + 10)
        hh = h if gg_big is g else K.Katz(_dev(gg_big.rowptr), _dev(gg_big.col))
        with pytest.raises(K.KatzError) as e:
            hh.rank(alpha, k, eps)
        assert e.value.name == "KATZ_EINVAL"
    with pytest.raises(K.KatzError) as e:
        h.ranking(5)  # no successful ranking yet
    assert e.value.name == "KATZ_ESTATE"
    bad = g.col.copy()
    bad[3] = 99
    with pytest.raises(K.KatzError) as e:
        K.Katz(_dev(g.rowptr), _dev(bad))
    assert e.value.name == "KATZ_EINVAL"


def test_repeat_call_is_deterministic():
    g = gg.rmat(14, 16, seed=8)
    h = K.Katz(_dev(g.rowptr), _dev(g.col))
    h.rank(0.0, 200, 1e-9)
    a = (h.ranking(200), *h.bounds()[:2])
    h.rank(0.0, 200, 1e-9)
    b = (h.ranking(200), *h.bounds()[:2])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.slow
def test_rmat22_top1000_full_size():
    """The benchmark workload at full size (R-MAT scale 22, top-1000, eps 1e-9)
    in the configuration bench.py times (profiled host loop, two walk slots),
    against a complete oracle run: same r, same ranking, every node's bounds."""
    g = gg.workload("rmat22")
    oracle.set_threads(0)
    check_parity(g, 0.0, 1000, 1e-9, walks=False, profile=1)



def test_large_host_csr_is_copied_in_slices_and_matches_device_input():
    # a host CSR of >= 2^22 arcs is copied slice by slice and renamed as it
    # arrives: the handle must equal one created from device arrays
    g = gg.rmat(18, 16, seed=61)
    assert g.nnz >= 1 << 22
    a = run_gpu(g, 0.0, 200, 1e-9, keep_history=False, on_device=False)
    b = run_gpu(g, 0.0, 200, 1e-9, keep_history=False, on_device=True)
    assert a["info"].r == b["info"].r
    np.testing.assert_array_equal(a["ranking"], b["ranking"])
    np.testing.assert_array_equal(a["l"], b["l"])
    np.testing.assert_array_equal(a["u"], b["u"])


def test_host_slices_hub_chunks_and_anchor_order_give_the_same_bits():
    # a host CSR is renamed slice by slice as it arrives, hub rows (more than
    # 2048 arcs, chunk by chunk) with the slice that holds them, and the anchor
    # order then permutes the low-degree rows: host or device input, anchor
    # order on or off, the results are the same bits
    g = gg.chung_lu(1 << 19, 16.0, 2.1, seed=63)
    assert g.nnz >= 1 << 22 and g.deg_max() > 2048
    runs = [run_gpu(g, 0.0, 200, 1e-9, keep_history=False, on_device=dev, locality=loc)
            for loc in (1, -1) for dev in (False, True)]
    for b in runs[1:]:
        assert b["info"].r == runs[0]["info"].r
        np.testing.assert_array_equal(b["ranking"], runs[0]["ranking"])
        np.testing.assert_array_equal(b["l"], runs[0]["l"])
        np.testing.assert_array_equal(b["u"], runs[0]["u"])


def test_large_host_csr_with_a_bad_column_entry_in_a_late_slice_is_rejected():
    g = gg.rmat(18, 16, seed=62)
    col = g.col.copy()
    col[-3] = g.n  # out of range, in the last slice
    with pytest.raises(K.KatzError) as e:
        K.Katz(g.rowptr, col)
    assert e.value.name == "KATZ_EINVAL"
    rp = g.rowptr.copy()
    rp[g.n // 2] = rp[g.n // 2 + 1] + 5  # not monotone
    with pytest.raises(K.KatzError) as e:
        K.Katz(rp, g.col)
    assert e.value.name == "KATZ_EINVAL"


def test_directed_graph_with_anchor_order_matches_the_oracle():
    # the anchor order on a directed graph (rows ordered by out-degree class,
    # anchors among out-neighbours): oracle parity and the bits of the plain order
    g = gg.orient(gg.chung_lu(1 << 15, 16.0, 2.1, seed=97), seed=98)
    got, _ = check_parity(g, 0.0, 100, 1e-9, undirected=False, locality=1)
    plain = run_gpu(g, 0.0, 100, 1e-9, undirected=False, locality=-1)
    np.testing.assert_array_equal(got["ranking"], plain["ranking"])
    np.testing.assert_array_equal(got["l"], plain["l"])
    np.testing.assert_array_equal(got["u"], plain["u"])


def test_l2_fetch_option_keeps_the_bits_and_restores_the_limit():
    """katz_opts.l2_fetch_bytes changes the context's maximum L2 fetch
    granularity only during the call: the ranking and bounds are the same
    bits, and the limit reads as before afterwards."""
    import ctypes

    cu = ctypes.CDLL("libcuda.so.1")

    def limit():
        out = ctypes.c_size_t(0)
        assert cu.cuCtxGetLimit(ctypes.byref(out), ctypes.c_int(5)) == 0  # CU_LIMIT_MAX_L2_FETCH_GRANULARITY
        return int(out.value)

    g = gg.rmat(14, 16, seed=9)
    torch.zeros(1, device="cuda")
    before = limit()
    out = []
    for fetch in (0, 64, 32):
        h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(l2_fetch_bytes=fetch))
        h.rank(0.0, 200, 1e-9)
        out.append((h.ranking(200), *h.bounds()[:2]))
        h.close()
        assert limit() == before
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_locality_order_gives_the_same_bits(precision):
    """katz_opts.locality = 1 reorders the low-degree rows by anchor (the
    internal order only): ranking, bounds and every walk level are the same
    bits as in the plain degree-class order, also after update batches, and
    the FP64 path still matches the oracle."""
    g = gg.chung_lu(1 << 15, 16.0, 2.1, seed=95)
    D, k, eps = g.deg_max() + 32, 100, 1e-9
    st = gg.stream(g, 3, seed=96, max_size=400, deg_bound=D)
    res = []
    for loc in (-1, 1):
        h = K.Katz(_dev(g.rowptr), _dev(g.col),
                   K.katz_default_opts(locality=loc, precision=precision, keep_history=1, deg_bound=D))
        info = h.rank(0.0, k, eps)
        out = [h.ranking(k), *h.bounds()[:2], *[h.walk(i) for i in range(1, info.r + 1)]]
        for j in range(len(st)):
            h.update(*st.batch(j))
            out += [h.ranking(k), *h.bounds()[:2]]
        res.append(out)
        h.close()
    assert len(res[0]) == len(res[1])
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    if precision == 0:
        check_parity(g, 0.0, k, eps, locality=1)
