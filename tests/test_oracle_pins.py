"""Pins of the CPU oracle against things other than itself (CPU only).

* Eq. (1)/(5): exact walk counts against brute-force walk enumeration.
* Eq. (2): the closed form c = alpha A (I - alpha A)^{-1} 1 solved in exact
  rational arithmetic; Theorem 1 (l_r <= c <= u_r) at every r, and l_r, u_r
  converge to c.
* Lemma 2: l_r non-decreasing, u_r non-increasing.
* Lemma 3 (complete graph): omega_i = (n-1)^i, u_i = Katz = delta/(1-delta),
  and the closed form of l_i that follows from it (tests/golden).
* Star graph: closed form of Katz from the two geometric series (tests/golden).
* Theorem 1's precondition alpha * deg_max < 1 is enforced.
* Algorithm 1's converged(): the final ranking meets the top-k criterion of
  Sec. 3.1 checked over all pairs by brute force, one iteration earlier it
  does not, and it agrees with the exact Katz order up to eps.
* Algorithm 2 taken literally (exact arithmetic) reproduces the static walk
  counts of the modified graph (Sec. 4 correctness statement), and the
  dynamic session equals a static recomputation.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


def _random_graph(n, p, rng, directed=False):
    if directed:
        pairs = [(a, b) for a in range(n) for b in range(n) if a != b and rng.random() < p]
        rowptr = np.zeros(n + 1, np.int64)
        col = []
        for a in range(n):
            row = sorted(b for (x, b) in pairs if x == a)
            col.extend(row)
            rowptr[a + 1] = len(col)
        return rowptr, np.array(col, np.int32)
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    if not pairs:
        pairs = [(0, 1)]
    u, v = zip(*pairs)
    g = gg.from_edges(n, np.array(u), np.array(v))
    return g.rowptr, g.col


def _brute_walks(rowptr, col, r):
    """omega_i(v) by enumerating every walk of length i from v explicitly."""
    n = len(rowptr) - 1
    nbr = [list(col[rowptr[v]:rowptr[v + 1]]) for v in range(n)]
    out = [[0] * n for _ in range(r)]
    for v in range(n):
        stack = [(v, 0)]
        while stack:
            x, length = stack.pop()
            if length >= 1:
                out[length - 1][v] += 1
            if length < r:
                for y in nbr[x]:
                    stack.append((y, length + 1))
    return out


def _exact_katz(rowptr, col, alpha: Fraction):
    """c = alpha A (I - alpha A)^{-1} 1 in exact rational arithmetic (Eq. 2)."""
    n = len(rowptr) - 1
    A = sympy.zeros(n, n)
    for v in range(n):
        for j in range(rowptr[v], rowptr[v + 1]):
            A[v, int(col[j])] += 1
    a = sympy.Rational(alpha.numerator, alpha.denominator)
    z = (sympy.eye(n) - a * A).LUsolve(sympy.ones(n, 1))
    c = a * A * z
    return [Fraction(int(sympy.fraction(x)[0]), int(sympy.fraction(x)[1])) for x in c]


def _bounds_at(rowptr, col, alpha, k, eps, R, undirected=True):
    """Oracle state after exactly R iterations of Algorithm 1's loop body."""
    s = oracle.Session(rowptr, col, undirected)
    assert s.run_fixed(alpha, R) == oracle.OK
    info = s.info()
    c, l, u = s.bounds()
    return info, c, l, u, s


# ---------------------------------------------------------------------------
# Eq. (5) against brute-force enumeration
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("directed", [False, True])
def test_walk_counts_match_bruteforce(seed, directed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 8))
    rowptr, col = _random_graph(n, 0.5, rng, directed)
    r = 6
    brute = _brute_walks(rowptr, col, r)
    exact = oracle.walks_exact(rowptr, col, r)
    assert exact == brute
    # the FP64 walk counts of the session are exact while below 2^53
    s = oracle.Session(rowptr, col, not directed)
    assert s.run_fixed(0.0, r) == oracle.OK
    for i in range(1, r + 1):
        assert [int(x) for x in s.omega(i)] == brute[i - 1]


def test_walks_exact_overflow_is_reported():
    g = gg.complete(40)
    with pytest.raises(oracle.OracleError):
        oracle.walks_exact(g.rowptr, g.col, 30)  # 39^30 > 2^128


# ---------------------------------------------------------------------------
# Theorem 1 and Lemma 2 against the exact closed form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("directed", [False, True])
def test_bounds_bracket_exact_katz_every_iteration(seed, directed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 12))
    rowptr, col = _random_graph(n, 0.35, rng, directed)
    D = int(np.diff(rowptr).max())
    alpha = Fraction(1, D + 1) if seed % 2 == 0 else Fraction(1, 2 * D)
    cx = _exact_katz(rowptr, col, alpha)
    cf = np.array([float(x) for x in cx])
    prev_l, prev_u = None, None
    for R in range(1, 25):
        info, c, l, u, _ = _bounds_at(rowptr, col, float(alpha), n, 1e-300, R, not directed)
        assert info["r"] == R
        tol = 4e-16 * np.maximum(cf, 1e-300) + 1e-300
        assert np.all(l <= cf + tol), (R, l - cf)
        assert np.all(u >= cf - tol), (R, u - cf)
        if prev_l is not None:  # Lemma 2
            assert np.all(l >= prev_l - 4e-16 * np.abs(l))
            assert np.all(u <= prev_u + 4e-16 * np.abs(u))
        prev_l, prev_u = l, u
    # both bounds converge to Katz (a wrong power of alpha would not)
    # (unscaled FP64 walk counts stay finite while D^R < 1e300)
    R = min(280, int(290 / np.log10(D + 1)))
    _, _, l, u, _ = _bounds_at(rowptr, col, float(alpha), n, 1e-300, R, not directed)
    assert np.allclose(l, cf, rtol=1e-9, atol=1e-15)
    assert np.allclose(u, cf, rtol=1e-9, atol=1e-15)


def test_alpha_at_or_above_inverse_degree_is_rejected():
    g = gg.star(4)
    s = oracle.Session(g.rowptr, g.col)
    assert s.rank_static(0.25, 1, 1e-6) == oracle.EALPHA  # alpha * deg_max = 1
    assert s.rank_static(0.3, 1, 1e-6) == oracle.EALPHA
    assert s.rank_static(0.2499, 1, 1e-6) == oracle.OK


# ---------------------------------------------------------------------------
# Lemma 3 and the star graph (tests/golden)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("row", _read_golden("lemma3_complete_graph.txt"))
def test_lemma3_complete_graph(row):
    n, dn, dd, kn, kd = row
    delta = Fraction(dn, dd)
    katz = Fraction(kn, kd)
    assert katz == delta / (1 - delta)
    g = gg.complete(n)
    alpha = float(delta / (n - 1))
    cx = _exact_katz(g.rowptr, g.col, delta / (n - 1))
    assert all(x == katz for x in cx)
    assert oracle.walks_exact(g.rowptr, g.col, 5) == [[(n - 1) ** i] * n for i in range(1, 6)]
    for R in range(1, 12):
        info, c, l, u, _ = _bounds_at(g.rowptr, g.col, alpha, 1, 1e-300, R)
        assert np.allclose(u, float(katz), rtol=2e-15, atol=0)
        c_R = sum(delta ** i for i in range(1, R + 1))
        l_R = c_R + delta ** (R + 1) / (n - 1)   # alpha^{R+1} omega_R = delta^{R+1}/(n-1)
        assert np.allclose(c, float(c_R), rtol=2e-15, atol=0)
        assert np.allclose(l, float(l_R), rtol=2e-15, atol=0)


@pytest.mark.parametrize("row", _read_golden("star_closed_form.txt"))
def test_star_closed_form(row):
    L, an, ad, cn, cd, ln, ld = row
    alpha = Fraction(an, ad)
    g = gg.star(L)
    cx = _exact_katz(g.rowptr, g.col, alpha)
    assert cx[0] == Fraction(cn, cd)
    assert all(x == Fraction(ln, ld) for x in cx[1:])
    info, c, l, u, _ = _bounds_at(g.rowptr, g.col, float(alpha), L + 1, 1e-300, 60)
    assert np.isclose(l[0], cn / cd, rtol=1e-12) and np.isclose(u[0], cn / cd, rtol=1e-12)
    assert np.allclose(l[1:], ln / ld, rtol=1e-12) and np.allclose(u[1:], ln / ld, rtol=1e-12)
    # the centre outranks every leaf, certified after the first iteration
    res = oracle.katz_static(g.rowptr, g.col, float(alpha), 1, 1e-9)
    assert list(res["ranking"]) == [0]


# ---------------------------------------------------------------------------
# Algorithm 1's converged(): brute-force top-k criterion and exact order
# ---------------------------------------------------------------------------
def _criterion(l, u, k, eps):
    """Top-k criterion of Sec. 3.1 over all pairs: the k nodes with highest l
    (ties by id) are eps-separated (Eq. 3) from each other and from all others."""
    n = len(l)
    order = sorted(range(n), key=lambda v: (-l[v], v))
    top, rest = order[:k], order[k:]
    for i, j in itertools.combinations(range(len(top)), 2):
        if not (l[top[i]] > u[top[j]] - eps):
            return False, order
    lk = min(l[v] for v in top)
    for v in rest:
        if not (lk > u[v] - eps):
            return False, order
    return True, order


@pytest.mark.parametrize("seed", range(10))
def test_converged_meets_topk_criterion_first_time(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(20, 120))
    rowptr, col = _random_graph(n, float(rng.uniform(0.04, 0.2)), rng)
    k = int(rng.integers(1, min(n, 15)))
    eps = 1e-9
    res = oracle.katz_static(rowptr, col, 0.0, k, eps)
    r = res["r"]
    ok, order = _criterion(res["l"], res["u"], k, eps)
    assert ok
    assert list(res["ranking"]) == order[:k]
    if r > 1:
        _, _, l1, u1, _ = _bounds_at(rowptr, col, 0.0, k, eps, r - 1)
        assert not _criterion(l1, u1, k, eps)[0]


@pytest.mark.parametrize("seed", range(12))
def test_converged_on_given_bounds_is_the_pairwise_criterion(seed):
    """converged() on caller-given bounds (M = V) against the all-pairs
    criterion of Eq. 3; the bounds are drawn so that some arrays separate
    and some fail either at an adjacent top-k pair or at a node outside the
    top-k, and with many exact ties in l."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(5, 60))
    k = int(rng.integers(1, n + 1))
    eps = 1e-3
    base = rng.integers(0, 6 if seed % 3 == 0 else 1000, n).astype(np.float64)  # seed % 3 == 0: heavy ties
    width = rng.choice([0.0, 5e-4, 2e-3, 0.5], n, p=[0.4, 0.3, 0.2, 0.1]) * (seed % 2)
    l = base.copy()
    u = base + width
    ok, top = oracle.converged_bounds(l, u, k, eps)
    want_ok, order = _criterion(l, u, k, eps)
    assert ok == want_ok
    assert list(top) == order[:k]


def test_converged_on_given_bounds_fails_at_each_test_alone():
    """One array where only an adjacent top-k pair overlaps, one where only a
    node outside the top-k crosses the k-th lower bound."""
    eps = 0.25  # exact in binary: u - eps lands exactly on the compared lower bound
    l = np.array([10.0, 9.0, 8.0, 1.0, 0.5])
    u = l + 0.0
    assert oracle.converged_bounds(l, u, 3, eps)[0]
    u_pair = u.copy()
    u_pair[1] = 10.0 + eps  # node 1 reaches node 0 within eps: adjacent pair not separated
    assert not _criterion(l, u_pair, 3, eps)[0]
    assert not oracle.converged_bounds(l, u_pair, 3, eps)[0]
    u_cross = u.copy()
    u_cross[3] = 8.0 + eps  # node 3 (rank 4) reaches the k-th lower bound
    assert not _criterion(l, u_cross, 3, eps)[0]
    assert not oracle.converged_bounds(l, u_cross, 3, eps)[0]


@pytest.mark.parametrize("seed", range(6))
def test_certified_ranking_matches_exact_katz(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(8, 13))
    rowptr, col = _random_graph(n, 0.35, rng)
    D = int(np.diff(rowptr).max())
    alpha = Fraction(1, D + 1)
    cx = _exact_katz(rowptr, col, alpha)
    eps = 1e-9
    for k in (1, 3, n):
        res = oracle.katz_static(rowptr, col, float(alpha), k, eps)
        R = [int(v) for v in res["ranking"]]
        assert len(R) == min(k, n)
        for a, b in zip(R, R[1:]):  # consecutive ranked nodes: order correct up to eps
            assert cx[a] >= cx[b] - Fraction(eps)
        rest = set(range(n)) - set(R)
        for v in rest:
            assert cx[v] <= cx[R[-1]] + Fraction(eps)


def test_isolated_nodes_and_k_above_n():
    g = gg.from_edges(6, np.array([0, 1]), np.array([1, 2]))  # path 0-1-2, nodes 3..5 isolated
    res = oracle.katz_static(g.rowptr, g.col, 0.0, 10, 1e-9)
    assert list(res["ranking"][:3]) == [1, 0, 2]
    assert np.all(res["l"][3:] == 0) and np.all(res["u"][3:] == 0)


# ---------------------------------------------------------------------------
# Algorithm 2 against static recomputation (Sec. 4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_alg2_literal_equals_static_recompute(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(6, 14))
    g = gg.from_edges(n, *zip(*[(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.3] or [(0, 1)]))
    r = 5
    omega = oracle.walks_exact(g.rowptr, g.col, r)
    src, dst, ins = gg.update_batch(g, int(rng.integers(1, 5)), seed=seed)
    # undirected batch -> both arcs
    s2 = np.concatenate([src, dst])
    d2 = np.concatenate([dst, src])
    i2 = np.concatenate([ins, ins])
    new = oracle.alg2_update_exact(g.rowptr, g.col, omega, s2, d2, i2)
    g2 = gg.apply_batch(g, src, dst, ins)
    assert new == oracle.walks_exact(g2.rowptr, g2.col, r)


@pytest.mark.parametrize("seed", range(5))
def test_dynamic_session_equals_static_recompute(seed):
    g = gg.rmat(9, 8, seed=500 + seed)
    k, eps = 20, 1e-9
    D = g.deg_max() + 8
    s = oracle.Session(g.rowptr, g.col, True, D)
    assert s.rank_static(0.0, k, eps) == oracle.OK
    cur = g
    for b in range(3):
        src, dst, ins = gg.update_batch(cur, 8 + 10 * b, seed=1000 * seed + b)
        st = s.apply_update(src, dst, ins)
        if st == oracle.EALPHA:
            continue
        assert st == oracle.OK
        cur = gg.apply_batch(cur, src, dst, ins)
        info = s.info()
        t = oracle.Session(cur.rowptr, cur.col, True, D)
        assert t.run_fixed(info["alpha"], info["r"]) == oracle.OK  # same r
        for i in range(1, info["r"] + 1):
            assert np.array_equal(s.omega(i), t.omega(i))
        c, l, u = s.bounds()
        c2, l2, u2 = t.bounds()
        assert np.array_equal(c, c2) and np.array_equal(l, l2) and np.array_equal(u, u2)
        ok, order = _criterion(l, u, k, eps)
        assert ok and list(s.ranking()) == order[:k]


def test_dynamic_batch_validation_is_atomic():
    g = gg.cycle(8)
    s = oracle.Session(g.rowptr, g.col, True, 3)
    assert s.rank_static(0.0, 2, 1e-6) == oracle.OK
    before = s.bounds()
    cases = [
        ([0], [1], [1]),         # insert an existing edge
        ([0], [2], [0]),         # delete an absent edge
        ([0, 2], [2, 0], [1, 1]),  # the same pair twice
        ([3], [3], [1]),         # self-loop
    ]
    for src, dst, ins in cases:
        assert s.apply_update(src, dst, ins) == oracle.EINVAL
    # degree bound 3: a node of degree 2 may take one more edge, not two
    assert s.apply_update([0, 0], [2, 4], [1, 1]) == oracle.EALPHA
    after = s.bounds()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    assert s.apply_update([0], [4], [1]) == oracle.OK


# Directed graphs (Sec. 2.1: edges are ordered pairs; an update changes the
# source's row only)
@pytest.mark.parametrize("seed", range(6))
def test_alg2_literal_directed_equals_static_recompute(seed):
    rng = np.random.default_rng(450 + seed)
    n = int(rng.integers(6, 14))
    g = gg.orient(gg.from_edges(n, *zip(*[(a, b) for a in range(n) for b in range(a + 1, n)
                                          if rng.random() < 0.4] or [(0, 1)])), seed)
    r = 5
    assert oracle.walks_exact(g.rowptr, g.col, r) == [list(x) for x in _brute_walks(g.rowptr, g.col, r)]
    omega = oracle.walks_exact(g.rowptr, g.col, r)
    src, dst, ins = gg.directed_update_batch(g, int(rng.integers(1, 6)), seed=seed)
    new = oracle.alg2_update_exact(g.rowptr, g.col, omega, src, dst, ins)
    g2 = gg.apply_directed_batch(g, src, dst, ins)
    assert new == [list(x) for x in _brute_walks(g2.rowptr, g2.col, r)]


def _brute_inbound_walks(rowptr, col, r):
    """Walks of length i that END at v, by enumerating every walk from every
    start and crediting its last node (Sec. 2.1, inbound Katz)."""
    n = len(rowptr) - 1
    nbr = [list(col[rowptr[v]:rowptr[v + 1]]) for v in range(n)]
    out = [[0] * n for _ in range(r)]
    for v in range(n):
        stack = [(v, 0)]
        while stack:
            x, length = stack.pop()
            if length >= 1:
                out[length - 1][x] += 1
            if length < r:
                for y in nbr[x]:
                    stack.append((y, length + 1))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_inbound_walks_are_outbound_walks_of_the_reverse_graph(seed):
    rng = np.random.default_rng(470 + seed)
    n = int(rng.integers(5, 9))
    rowptr, col = _random_graph(n, 0.35, rng, directed=True)
    g = gg.Graph(rowptr, col)
    rev = gg.reverse(g)
    assert rev.nnz == g.nnz
    assert oracle.walks_exact(rev.rowptr, rev.col, 5) == _brute_inbound_walks(rowptr, col, 5)
    assert np.array_equal(gg.reverse(rev).rowptr, g.rowptr) and np.array_equal(gg.reverse(rev).col, g.col)


@pytest.mark.parametrize("seed", range(4))
def test_dynamic_session_directed_equals_static_recompute(seed):
    g = gg.orient(gg.rmat(9, 8, seed=520 + seed), seed)
    k, eps = 20, 1e-9
    D = g.deg_max() + 8
    s = oracle.Session(g.rowptr, g.col, False, D)
    assert s.rank_static(0.0, k, eps) == oracle.OK
    cur = g
    for b in range(3):
        src, dst, ins = gg.directed_update_batch(cur, 8 + 10 * b, seed=1000 * seed + b, deg_bound=D)
        assert s.apply_update(src, dst, ins) == oracle.OK
        cur = gg.apply_directed_batch(cur, src, dst, ins)
        info = s.info()
        t = oracle.Session(cur.rowptr, cur.col, False, D)
        assert t.run_fixed(info["alpha"], info["r"]) == oracle.OK
        for i in range(1, info["r"] + 1):
            assert np.array_equal(s.omega(i), t.omega(i))
        c, l, u = s.bounds()
        c2, l2, u2 = t.bounds()
        assert np.array_equal(c, c2) and np.array_equal(l, l2) and np.array_equal(u, u2)
        assert np.array_equal(l, c)  # directed: l_r = c_r (Theorem 1)
        ok, order = _criterion(l, u, k, eps)
        assert ok and list(s.ranking()) == order[:k]


def test_directed_batch_validation_uses_ordered_pairs():
    # 0 -> 1 -> 2 -> 0 and 0 -> 2
    g = gg.directed_from_arcs(4, [0, 1, 2, 0], [1, 2, 0, 2])
    s = oracle.Session(g.rowptr, g.col, False, 3)
    assert s.rank_static(0.0, 2, 1e-6) == oracle.OK
    before = s.bounds()
    cases = [
        ([1], [2], [1]),            # insert an existing arc
        ([2], [1], [0]),            # delete an absent arc (its reverse exists)
        ([3, 3], [0, 0], [1, 1]),   # the same ordered pair twice
        ([0, 0, 0], [3, 3, 1], [1, 1, 0]),
    ]
    for src, dst, ins in cases:
        assert s.apply_update(src, dst, ins) == oracle.EINVAL
    assert all(np.array_equal(a, b) for a, b in zip(before, s.bounds()))
    # the degree bound applies to out-degrees: with D = 2, node 0 (out-degree
    # 2) takes no further out-arc but any number of in-arcs
    s3 = oracle.Session(g.rowptr, g.col, False, 2)
    assert s3.rank_static(0.0, 2, 1e-6) == oracle.OK
    assert s3.apply_update([0], [3], [1]) == oracle.EALPHA
    assert s3.apply_update([3], [0], [1]) == oracle.OK
    assert s.apply_update([0, 1], [3, 3], [1, 1]) == oracle.OK
    assert s.apply_update([0], [3], [0]) == oracle.OK
    assert s.apply_update([3, 0], [0, 3], [1, 1]) == oracle.OK  # a -> b and b -> a in one batch
    g2 = gg.directed_from_arcs(4, [0, 1, 2, 0, 1, 3, 0], [1, 2, 0, 2, 3, 0, 3])
    t = oracle.Session(g2.rowptr, g2.col, False, 3)
    assert t.run_fixed(s.info()["alpha"], s.info()["r"]) == oracle.OK
    assert all(np.array_equal(a, b) for a, b in zip(s.bounds(), t.bounds()))
    s2 = oracle.Session(g.rowptr, g.col, False, 3)
    assert s2.rank_static(0.0, 2, 1e-6) == oracle.OK
    assert s2.apply_update([0, 0], [3, 1], [1, 0]) == oracle.OK
    assert s2.apply_update([0], [1], [1]) == oracle.OK
    assert s2.apply_update([0, 0], [3, 1], [0, 1]) == oracle.EINVAL  # 0 -> 1 present again


# ---------------------------------------------------------------------------
# The other stopping criteria of Sec. 3.1, each against a brute-force check
# of its definition at every iteration
# ---------------------------------------------------------------------------
def _bounds_fixed(rowptr, col, R):
    s = oracle.Session(rowptr, col)
    assert s.run_fixed(0.0, R) == oracle.OK
    c, l, u = s.bounds()
    return l, u


def _all_pairs_separated(l, u, eps):
    """Ranking criterion: every pair eps-separated (Eq. 3), w the node the
    order (l desc, id asc) puts first."""
    order = sorted(range(len(l)), key=lambda v: (-l[v], v))
    for i, j in itertools.combinations(range(len(order)), 2):
        if not (l[order[i]] > u[order[j]] - eps):
            return False, order
    return True, order


def _first_r(rowptr, col, test, r_max=60):
    for R in range(1, r_max + 1):
        l, u = _bounds_fixed(rowptr, col, R)
        if test(l, u):
            return R
    return None


@pytest.mark.parametrize("seed", range(6))
def test_ranking_criterion_is_all_pairs_separated_first_time(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(10, 40))
    rowptr, col = _random_graph(n, float(rng.uniform(0.08, 0.3)), rng)
    eps = 1e-6
    s = oracle.Session(rowptr, col)
    assert s.rank(0.0, oracle.RANKING, eps) == oracle.OK
    r = s.info()["r"]
    assert r == _first_r(rowptr, col, lambda l, u: _all_pairs_separated(l, u, eps)[0])
    c, l, u = s.bounds()
    assert list(s.ranking()) == _all_pairs_separated(l, u, eps)[1]
    # the ranking is the exact Katz order wherever two nodes differ by more than eps
    D = int(np.diff(rowptr).max())
    cx = _exact_katz(rowptr, col, Fraction(1, D + 1))
    R = [int(v) for v in s.ranking()]
    for i, j in itertools.combinations(range(n), 2):
        assert cx[R[i]] >= cx[R[j]] - Fraction(eps)


@pytest.mark.parametrize("seed", range(6))
def test_score_criterion_bounds_within_eps_first_time(seed):
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(10, 60))
    rowptr, col = _random_graph(n, float(rng.uniform(0.05, 0.3)), rng)
    eps = 1e-7
    s = oracle.Session(rowptr, col)
    assert s.rank(0.0, oracle.SCORE, eps) == oracle.OK
    r = s.info()["r"]
    assert r == _first_r(rowptr, col, lambda l, u: bool(np.all(u - l < eps)))
    assert len(s.ranking()) == 0
    # every score is then known to within eps
    D = int(np.diff(rowptr).max())
    cx = _exact_katz(rowptr, col, Fraction(1, D + 1))
    c, l, u = s.bounds()
    for v in range(n):
        assert abs(Fraction(float(l[v])) - cx[v]) < Fraction(eps)


@pytest.mark.parametrize("seed", range(6))
def test_pair_criterion_first_time(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(10, 60))
    rowptr, col = _random_graph(n, float(rng.uniform(0.05, 0.3)), rng)
    a, b = (int(x) for x in rng.choice(n, 2, replace=False))
    eps = 1e-8

    def separated(l, u):
        w, v = (a, b) if (l[a], -a) > (l[b], -b) else (b, a)
        return l[w] > u[v] - eps

    s = oracle.Session(rowptr, col)
    assert s.rank(0.0, oracle.PAIR, eps, pair=(a, b)) == oracle.OK
    r = s.info()["r"]
    assert r == _first_r(rowptr, col, separated)
    c, l, u = s.bounds()
    w, v = (a, b) if (l[a], -a) > (l[b], -b) else (b, a)
    assert list(s.ranking()) == [w, v]
