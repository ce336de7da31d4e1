"""Helpers comparing the CUDA path with the CPU oracle (test-only)."""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-12  # FP64 mode: omega, l, u within 1e-12 relative of the oracle


def tie_groups(ranking, l_ref, tol=REL_TOL, atol=0.0):
    """Split a ranking into runs of nodes whose reference lower bounds agree
    to within tol (relative) + atol; the order inside a run is not unique."""
    groups, cur = [], [int(ranking[0])] if len(ranking) else []
    for a, b in zip(ranking, ranking[1:]):
        la, lb = l_ref[a], l_ref[b]
        if abs(la - lb) <= tol * max(abs(la), abs(lb)) + atol:
            cur.append(int(b))
        else:
            groups.append(cur)
            cur = [int(b)]
    if cur:
        groups.append(cur)
    return groups


def assert_same_ranking(got, ref, l_ref, tol=REL_TOL, atol=0.0):
    """Identical certified order, up to permutations inside runs of
    rounding-level ties (compared as sets); the last run may be cut by k, so
    there the GPU's members must be tied with the oracle's k-th node."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if np.array_equal(got, ref):
        return 0
    gref = tie_groups(ref, l_ref, tol, atol)
    pos = 0
    for gi, grp in enumerate(gref):
        seg = got[pos:pos + len(grp)]
        if gi < len(gref) - 1:
            assert set(seg.tolist()) == set(grp), f"rank {pos}: {sorted(seg.tolist())} vs {sorted(grp)}"
        else:
            lk = l_ref[grp[0]]
            for v in seg:
                assert abs(l_ref[v] - lk) <= tol * abs(lk) + atol, f"rank {pos}: node {v} not tied with {grp[0]}"
        pos += len(grp)
    return sum(len(g) > 1 for g in gref)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.maximum(np.abs(b), np.finfo(np.float64).tiny)
    d = np.abs(a - b)
    d[(a == b)] = 0.0
    return d / den


def assert_close(a, b, tol=REL_TOL, what=""):
    e = rel_err(a, b)
    i = int(np.argmax(e)) if e.size else 0
    assert e.size == 0 or e[i] <= tol, f"{what}: max rel err {e[i]:.3e} at {i}: {a[i]!r} vs {b[i]!r}"
