"""The float32 pre-screen of the kNN query never rejects a true neighbour.

The query compares a float32 squared distance d2f (float32 coordinates,
float32 arithmetic, possibly contracted into FMAs) against a bound derived
from the current k-th exact key kth:

    bound(kth) = f32( kth (1 + 1e-6) + 4 delta sqrt(kth) + 4 delta^2 ) (1 + 1e-6),
    delta = 4 * 1.5 * M * 2^-24,  M = largest |coordinate| of the bounding box,

and skips a candidate only when d2f > bound(kth).  A candidate that belongs in
the list has exact key d2 <= kth, and the bound grows with kth, so it is never
skipped if d2f <= bound(d2) for every pair.  This test checks that inequality
on adversarial pairs -- near-coincident points far from the origin (where
float32 rounding of the coordinates dominates), points at the box corners,
and random pairs -- for the three ways the compiler may contract
fx*fx + fy*fy + fz*fz.  Host-side check of the margin's derivation; no GPU.
"""
import numpy as np

f32 = np.float32


def _bound(d2, M):
    delta = 4.0 * 1.5 * M * 2.0 ** -24
    b = (d2 * (1.0 + 1e-6) + 4.0 * delta * np.sqrt(d2) + 4.0 * delta * delta).astype(np.float32)
    return b * f32(1.0 + 1e-6)


def _fma32(a, b, c):
    # a*b is exact in float64 for float32 a, b; one more rounding to float32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _d2f_variants(q, p):
    qf, pf = q.astype(np.float32), p.astype(np.float32)
    fx, fy, fz = (pf[:, a] - qf[:, a] for a in range(3))
    plain = (fx * fx + fy * fy) + fz * fz
    fused = _fma32(fz, fz, _fma32(fy, fy, fx * fx))
    mixed = _fma32(fy, fy, fx * fx) + fz * fz
    return plain, fused, mixed


def _exact_key(q, p):
    # the float64 key of the query, (dx dx + dy dy) + dz dz without contraction
    d = p - q
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def _check(q, p, M):
    d2 = _exact_key(q, p)
    b = _bound(d2, M)
    for v in _d2f_variants(q, p):
        assert np.all(v <= b), float(np.max(v.astype(np.float64) - b.astype(np.float64)))


def test_screen_keeps_every_true_neighbour():
    rng = np.random.default_rng(11)
    for M in (1.0, 1.3, 37.0, 1e-3):
        n = 200_000
        # random pairs in the box
        q = rng.uniform(-M, M, (n, 3))
        p = rng.uniform(-M, M, (n, 3))
        _check(q, p, M)
        # near-coincident pairs far from the origin (relative offsets 1e-9 .. 1e-3)
        q = rng.choice([-1.0, 1.0], (n, 3)) * rng.uniform(0.5 * M, M, (n, 3))
        scale = M * 10.0 ** rng.uniform(-9, -3, (n, 1))
        p = np.clip(q + scale * rng.standard_normal((n, 3)), -M, M)
        _check(q, p, M)
        # pairs on the sphere of radius M (the benchmark's surfaces), spacing ~1e-3 M
        v = rng.standard_normal((n, 3))
        q = M * v / np.linalg.norm(v, axis=1, keepdims=True)
        w = q + 1e-3 * M * rng.standard_normal((n, 3))
        p = M * w / np.linalg.norm(w, axis=1, keepdims=True)
        _check(q, p, M)


def test_screen_bound_is_not_vacuous():
    """The bound stays within a few float32 ulps of the key for pairs at the
    stencil scale (it prunes: a candidate twice as far is rejected)."""
    rng = np.random.default_rng(3)
    M = 1.0
    v = rng.standard_normal((10_000, 3))
    q = v / np.linalg.norm(v, axis=1, keepdims=True)
    p = q + 0.01 * rng.standard_normal((10_000, 3))
    d2 = _exact_key(q, p)
    b = _bound(d2, M).astype(np.float64)
    assert np.all(b < 1.01 * d2 + 1e-9)
    far = _d2f_variants(q, q + 2.0 * (p - q))[0].astype(np.float64)
    assert np.all(far > b)
