"""katz_certify_topk_noalloc against katz_rank_static / katz_get_ranking,
through the C ABI: the same top-k and the same verdict from the bounds the
static path leaves behind, on two calls in a row that share the entry
point's fixed working memory."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
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


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_static_path():
    cases = [(gg.rmat(15, 16, seed=41), 0.0, 600, 1e-9),      # several radix passes, k > one warp's worth
             (gg.erdos_renyi(3000, 12000, seed=42), 0.0, 16, 1e-7)]  # smaller n and k after a larger call
    for g, alpha, k, eps in cases:
        info, ranking, lower, upper = _static(g, alpha, k, eps)
        assert info.converged == 1
        ids, cert = _noalloc(lower, upper, k, eps)
        assert cert == 1
        assert_same_ranking(ids, ranking, lower.cpu().numpy())


@pytest.mark.gpu
def test_uncertified_bounds_are_reported_as_such():
    g = gg.rmat(13, 16, seed=43)
    info, _, lower, upper = _static(g, 0.0, 64, 1e-9, r_max=1)
    assert info.converged == 0
    ids, cert = _noalloc(lower, upper, 64, 1e-9)
    assert cert == 0
    # the ids are still the 64 largest lower bounds, ties by smaller id
    l = lower.cpu().numpy()
    order = np.lexsort((np.arange(g.n), -l))[:64]
    assert np.array_equal(ids, order)


def test_sizes_beyond_the_limits_are_rejected():
    # rejected on the host before any device work: no GPU needed
    for n, k in [(10000, K.KATZ_MAX_K + 1), (100, 0), (10, 11)]:
        lower = np.zeros(n)
        with pytest.raises(K.KatzError) as e:
            K.katz_certify_topk_noalloc(lower, lower, k, 1e-9, np.zeros(max(k, 1), np.int32),
                                        np.zeros(1, np.int32))
        assert e.value.name == "KATZ_EINVAL"
