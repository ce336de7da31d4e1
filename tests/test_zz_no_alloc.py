"""katz_certify_topk_noalloc through the C ABI.

The entry point is for callers that cannot let a library allocate device
memory; it keeps its working memory in a fixed array inside the library.
These tests check its output against the oracle's converged() on the same
bounds (Algorithm 1's top-k criterion with M = V) and against the static
path (katz_rank_static / katz_get_ranking), on calls in a row that share the
fixed array, and check that a call allocates no device memory.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.parity import assert_same_ranking

torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _static(g, alpha, k, eps, r_max=256):
    """Existing entry points: rank, then read the ranking and the bounds."""
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(r_max=r_max))
    info = h.rank(alpha, k, eps, check=False)
    ranking = h.ranking(min(k, g.n)) if info.converged else None
    lower = torch.empty(g.n, dtype=torch.float64, device="cuda")
    upper = torch.empty(g.n, dtype=torch.float64, device="cuda")
    K.katz_get_bounds(h.h, lower=lower, upper=upper)
    torch.cuda.synchronize()
    h.close()
    return info, ranking, lower, upper


def _noalloc(lower, upper, k, eps):
    ids = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    cert = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    K.katz_certify_topk_noalloc(lower, upper, k, eps, ids, cert, stream)
    stream.synchronize()
    return ids.cpu().numpy(), int(cert.item())


def _against_oracle(lower, upper, k, eps):
    """The entry point's ids and verdict equal the oracle's converged() on the
    same bounds: the top-k order (l desc, id asc) is unique, so ids compare
    exactly."""
    ids, cert = _noalloc(lower, upper, k, eps)
    ok, top = oracle.converged_bounds(lower.cpu().numpy(), upper.cpu().numpy(), k, eps)
    assert cert == int(ok)
    assert np.array_equal(ids, top)
    return ids, cert


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_oracle_and_the_static_path():
    cases = [(gg.rmat(15, 16, seed=41), 0.0, 600, 1e-9),      # several radix passes, k > one warp's worth
             (gg.erdos_renyi(3000, 12000, seed=42), 0.0, 16, 1e-7)]  # smaller n and k after a larger call
    for g, alpha, k, eps in cases:
        info, ranking, lower, upper = _static(g, alpha, k, eps)
        assert info.converged == 1
        ids, cert = _against_oracle(lower, upper, k, eps)
        assert cert == 1
        assert_same_ranking(ids, ranking, lower.cpu().numpy())


@pytest.mark.gpu
def test_ties_and_uncertified_bounds_match_the_oracle():
    # bounds of a ranking stopped after one iteration: not certified
    g = gg.rmat(13, 16, seed=43)
    info, _, lower, upper = _static(g, 0.0, 64, 1e-9, r_max=1)
    assert info.converged == 0
    _, cert = _against_oracle(lower, upper, 64, 1e-9)
    assert cert == 0
    # a cycle: every node has the same bounds; the top-k is the k smallest ids
    g = gg.cycle(5000)
    _, _, lower, upper = _static(g, 0.0, 10, 1e-9, r_max=3)
    ids, cert = _against_oracle(lower, upper, 10, 1e-9)
    assert cert == 0 and list(ids) == list(range(10))


@pytest.mark.gpu
def test_each_failing_test_is_seen_alone():
    """One array where only an adjacent top-k pair overlaps within eps, one
    where only a node outside the top-k crosses the k-th lower bound."""
    rng = np.random.default_rng(7)
    n, k, eps = 20000, 50, 0.25
    l = rng.permutation(n).astype(np.float64)  # distinct lower bounds
    u = l.copy()
    top = np.argsort(-l)[:k]
    _, cert = _against_oracle(_dev(l), _dev(u), k, eps)
    assert cert == 1
    u_pair = u.copy()
    u_pair[top[5]] = l[top[4]] + eps  # ranks 5 and 6 not separated; everything else is
    _, cert = _against_oracle(_dev(l), _dev(u_pair), k, eps)
    assert cert == 0
    u_cross = u.copy()
    outside = int(np.argsort(-l)[k + 100])
    u_cross[outside] = l[top[-1]] + eps  # a node outside the top-k reaches theta
    _, cert = _against_oracle(_dev(l), _dev(u_cross), k, eps)
    assert cert == 0


@pytest.mark.gpu
def test_a_call_allocates_no_device_memory():
    g = gg.rmat(14, 16, seed=44)
    _, _, lower, upper = _static(g, 0.0, 100, 1e-9)
    ids = torch.full((100,), -1, dtype=torch.int32, device="cuda")
    cert = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    K.katz_certify_topk_noalloc(lower, upper, 100, 1e-9, ids, cert, stream)  # first call: per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        K.katz_certify_topk_noalloc(lower, upper, 100, 1e-9, ids, cert, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(cert.item()) == 1


def test_sizes_beyond_the_limits_are_rejected():
    # rejected by the library on the host before any device work: no GPU needed
    import ctypes

    lib = K._load()
    for n, k in [(10000, K.KATZ_MAX_K + 1), (100, 0), (10, 11), (0, 1)]:
        buf = np.zeros(max(n, 1))
        ids = np.zeros(max(k, 1), np.int32)
        cert = np.zeros(1, np.int32)
        st = lib.katz_certify_topk_noalloc(buf.ctypes.data, buf.ctypes.data, n, k, 1e-9, ids.ctypes.data,
                                           cert.ctypes.data, ctypes.c_void_p(0))
        assert K.STATUS[st] == "KATZ_EINVAL"


def test_the_binding_refuses_buffers_the_kernels_cannot_use():
    # checked in the binding before the library is called: no GPU needed
    lo = np.zeros(100)
    with pytest.raises(ValueError):  # host numpy arrays
        K.katz_certify_topk_noalloc(lo, lo, 10, 1e-9, np.zeros(10, np.int32), np.zeros(1, np.int32))
    t = torch.zeros(100, dtype=torch.float64)
    with pytest.raises(ValueError):  # CPU tensors
        K.katz_certify_topk_noalloc(t, t, 10, 1e-9, torch.zeros(10, dtype=torch.int32),
                                    torch.zeros(1, dtype=torch.int32))


@pytest.mark.gpu
def test_the_binding_refuses_wrong_dtypes_and_sizes():
    lo = torch.zeros(100, dtype=torch.float64, device="cuda")
    ids = torch.zeros(10, dtype=torch.int32, device="cuda")
    cert = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = [
        (lo.float(), lo, ids, cert),                       # float32 bounds
        (lo, lo[:99], ids, cert),                          # upper shorter than lower
        (lo, lo, ids[:9], cert),                           # ids_out shorter than k
        (lo, lo, ids.long(), cert),                        # int64 ids
        (lo, lo, ids, torch.zeros(0, dtype=torch.int32, device="cuda")),  # no room for the verdict
    ]
    for a, b, i, c in bad:
        with pytest.raises(ValueError):
            K.katz_certify_topk_noalloc(a, b, 10, 1e-9, i, c)
