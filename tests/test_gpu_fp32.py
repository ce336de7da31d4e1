"""FP32-certified mode: walk levels from Ctrl::f32_from on are carried in FP32
and the bounds are widened by a proven rounding-error bound, evaluated with
directed rounding.  Checks: the certified bounds bracket the exact Katz score
(exact rational arithmetic) at every iteration, the certified ranking agrees
with the FP64 oracle up to eps-ties, each node's deviation from the oracle's
bounds stays inside the reported widening, and FP32 levels are really used."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
import sympy

import graphgen as gg
import oracle
from tests.parity import assert_close, assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _exact_katz(rowptr, col, alpha: Fraction):
    n = len(rowptr) - 1
    A = sympy.zeros(n, n)
    for v in range(n):
        for j in range(rowptr[v], rowptr[v + 1]):
            A[v, int(col[j])] += 1
    a = sympy.Rational(alpha.numerator, alpha.denominator)
    z = (sympy.eye(n) - a * A).LUsolve(sympy.ones(n, 1))
    return [Fraction(int(sympy.fraction(x)[0]), int(sympy.fraction(x)[1])) for x in a * A * z]


def _cert(g, k, eps, fp32_from=0, r_max=256, alpha=0.0, check=True):
    opts = K.katz_default_opts(precision=K.KATZ_FP32_CERT, fp32_from=fp32_from, r_max=r_max, keep_history=1)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(alpha, k, eps, check=check)
    out = dict(info=info, ranking=h.ranking(min(k, g.n)) if info.status in (0,) else None)
    out["l"], out["u"], out["err"] = h.bounds()
    h.close()
    return out


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("fp32_from", [2, 3])
def test_certified_bounds_bracket_exact_katz(seed, fp32_from):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(6, 12))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.4] or [(0, 1)]
    u, v = zip(*pairs)
    g = gg.from_edges(n, np.array(u), np.array(v))
    D = g.deg_max()
    alpha = Fraction(1, D + 1)
    cx = np.array([float(x) for x in _exact_katz(g.rowptr, g.col, alpha)])
    for r_max in (fp32_from, fp32_from + 1, fp32_from + 4, 40):
        got = _cert(g, n, 1e-300, fp32_from=fp32_from, r_max=r_max, alpha=float(alpha), check=False)
        assert got["info"].r <= r_max
        assert np.all(got["l"] <= cx) and np.all(got["u"] >= cx), (r_max, got["l"] - cx, got["u"] - cx)


@pytest.mark.parametrize("wl,k", [("er16k", 100), ("rmat14", 200)])
def test_fp32_certified_ranking_matches_oracle(wl, k):
    g = gg.workload("er16k") if wl == "er16k" else gg.rmat(14, 16, seed=77)
    eps = 1e-9
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, r_max=256)
    got = _cert(g, k, eps)
    info = got["info"]
    assert info.converged == 1 and info.r >= ref["r"]
    # identical certified order up to pairs closer than eps (both are certified)
    assert_same_ranking(got["ranking"], ref["ranking"], ref["l"], atol=eps)
    # per-node deviation from the FP64 oracle's bounds at the same r lies
    # within the reported rounding widening (plus the oracle's own FP64
    # rounding); where the FP32 run stopped at another r, the oracle runs
    # Algorithm 1's loop body to that r without a convergence check
    l_ref, u_ref = ref["l"], ref["u"]
    if info.r != ref["r"]:
        s = oracle.Session(g.rowptr, g.col, True)
        assert s.run_fixed(0.0, info.r) == oracle.OK
        _, l_ref, u_ref = s.bounds()
        s.close()
    assert np.all(np.abs(got["l"] - l_ref) <= got["err"] + 1e-12 * np.abs(l_ref) + 1e-300)
    assert np.all(np.abs(got["u"] - u_ref) <= got["err"] + 1e-12 * np.abs(u_ref) + 1e-300)
    assert np.all(got["l"] <= got["u"])


def test_fp32_levels_are_used_and_certify():
    g = gg.rmat(16, 16, seed=16)
    got = _cert(g, 1000, 1e-9)
    assert got["info"].converged == 1
    assert got["info"].fp32_levels >= 1
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, 1000, 1e-9, r_max=256)
    assert_same_ranking(got["ranking"], ref["ranking"], ref["l"], atol=1e-9)


def test_stall_reports_precision_error():
    # all levels in FP32 and an eps far below what FP32 can separate on a
    # graph with near-ties: the widening overtakes the tail, EPRECISION
    g = gg.rmat(12, 16, seed=3)
    got = _cert(g, 400, 1e-15, fp32_from=2, check=False)
    assert got["info"].status == 6  # KATZ_EPRECISION
    assert np.all(got["l"] <= got["u"])


def test_certified_bounds_monotone_across_the_fp32_switch():
    """Lemma 2 must hold for the certified bounds (the candidate filter and
    permanent deactivation rely on it), also where the widening grows at the
    switch to FP32 levels."""
    g = gg.rmat(15, 16, seed=5)
    k, eps = 300, 1e-9
    full = _cert(g, k, eps, fp32_from=3)
    assert full["info"].converged == 1 and len(full["ranking"]) == k
    top = full["ranking"]
    prev_l = prev_u = None
    for R in range(1, full["info"].r + 1):
        got = _cert(g, k, eps, fp32_from=3, r_max=R, check=False)
        l, u = got["l"][top], got["u"][top]
        if prev_l is not None:
            assert np.all(l >= prev_l) and np.all(u <= prev_u), R
        prev_l, prev_u = l, u


def test_fp32_switch_keeps_k_candidates_on_a_larger_graph():
    g = gg.rmat(18, 16, seed=18)
    got = _cert(g, 1000, 1e-9)
    assert got["info"].converged == 1 and got["info"].k == 1000 and len(got["ranking"]) == 1000


def test_auto_precision_escalates_a_stalled_ranking_to_fp64():
    # the stall case above, under KATZ_FP32_CERT_AUTO: the ranking is
    # recomputed with FP64 levels and matches the FP64 oracle
    g = gg.rmat(12, 16, seed=3)
    k, eps = 400, 1e-15
    opts = K.katz_default_opts(precision=K.KATZ_FP32_CERT_AUTO, fp32_from=2, r_max=256)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(0.0, k, eps)
    assert info.escalated == 1 and info.converged == 1 and info.fp32_levels == 0
    ref = oracle.katz_static(g.rowptr, g.col, 0.0, k, eps, r_max=256)
    assert info.r == ref["r"]
    lo, up, err = h.bounds()
    assert_close(lo, ref["l"], what="lower")
    assert_close(up, ref["u"], what="upper")
    assert_same_ranking(h.ranking(k), ref["ranking"], ref["l"])
    # a ranking that certifies in FP32 is not escalated
    info2 = h.rank(0.0, 50, 1e-4)
    assert info2.escalated == 0 and info2.converged == 1 and info2.fp32_levels > 0
    h.close()


def test_subnormal_fp32_levels_stay_certified():
    # alpha = 1e-13 (deg_bound 5 10^12, so alpha gamma = 1): level 2 is ~1e-26, level 3 lies around
    # the smallest normal binary32 (1.2e-38), where a rounding loses up to
    # 2^-150 absolutely instead of 2^-24 relatively.  Hubs a and b have equal
    # degree and differ in omega_2 by 1, a gap of alpha^2 that level 3
    # certifies; the bounds must bracket the exact Katz score.
    leaves = iter(range(3, 40))
    pairs = []
    a, b, c = 0, 1, 2
    for hub, extra_deg in ((a, 2), (b, 3)):  # 4 leaves + one node of degree extra_deg
        for _ in range(4):
            pairs.append((hub, next(leaves)))
        x = next(leaves)
        pairs.append((hub, x))
        for _ in range(extra_deg - 1):
            pairs.append((x, next(leaves)))
    for _ in range(4):
        pairs.append((c, next(leaves)))
    u, v = zip(*pairs)
    g = gg.from_edges(40, np.array(u), np.array(v))
    alpha = 1e-13
    opts = K.katz_default_opts(precision=K.KATZ_FP32_CERT, fp32_from=2, keep_history=1, deg_bound=5 * 10**12)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), opts)
    info = h.rank(alpha, 1, 1e-40)
    assert info.converged == 1 and info.r == 3 and info.fp32_levels == 2
    assert list(h.ranking(1)) == [b]
    s3 = h.walk(3)
    assert np.any((s3 > 0) & (s3 < 2.0 ** -126))  # subnormal FP32 values at level 3
    # exact Katz: sum over i <= 12 of alpha^i omega_i, the rest below
    # 2 (alpha deg_max)^13
    af = Fraction(alpha)
    n = g.n
    w = [1] * n
    y = [Fraction(0)] * n
    p = Fraction(1)
    for _ in range(12):
        w = [sum(w[int(x)] for x in g.col[g.rowptr[t]:g.rowptr[t + 1]]) for t in range(n)]
        p *= af
        y = [y[t] + p * w[t] for t in range(n)]
    rest = 2 * (af * g.deg_max()) ** 13
    lo, up, _ = h.bounds()
    deg = np.diff(g.rowptr)
    for t in range(n):  # an isolated node has Katz score 0 exactly
        assert Fraction(float(lo[t])) <= y[t], t
        assert Fraction(float(up[t])) >= y[t] + (rest if deg[t] else 0), t
    h.close()
