"""The float prefilters of the GPU graph construction (greedy sampling,
l-bar searches) rely on one bound: for float32 coordinates, the squared
distance formed in float32 as (dx*dx + dy*dy) + dz*dz, every operation
rounded to nearest, is within a relative 4e-7 of the exact squared
distance (plus 1e-36 for subnormal results). The kernels take a margin of
1e-5 around R^2 (greedy) and around the k-th float distance (l-bar), so
no decision moves. Checked here on the host with numpy's IEEE float32
arithmetic, on random pairs over many scales and on pairs built at the
radius itself."""
import numpy as np
import pytest

BOUND = 4e-7


def _sqd_f32(a, b):
    d = (a - b).astype(np.float32)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def _sqd_exact(a, b):
    d = a.astype(np.float64) - b.astype(np.float64)   # exact: float32 inputs
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


@pytest.mark.parametrize("scale", [1e-4, 1e-2, 1.0, 1e2, 1e4])
def test_float_squared_distance_relative_error(scale):
    rng = np.random.default_rng(int(np.log10(scale) * 10 + 100))
    a = (rng.standard_normal((200000, 3)) * scale).astype(np.float32)
    # neighbours at distances from 1e-6 to 1 of the scale
    off = rng.standard_normal((200000, 3)) * scale * 10.0 ** rng.uniform(-6, 0, (200000, 1))
    b = (a.astype(np.float64) + off).astype(np.float32)
    d2f = _sqd_f32(a, b).astype(np.float64)
    d2 = _sqd_exact(a, b)
    assert np.all(np.abs(d2f - d2) <= BOUND * d2 + 1e-36)


def test_margins_keep_every_decision_at_the_radius():
    """Pairs placed within a relative 1e-4 of R: the three-way test of the
    greedy cover (float below R^2 (1 - 1e-5): inside; at or above
    R^2 (1 + 1e-5) + 1e-36: outside; else the double test) gives the
    double test's answer every time."""
    rng = np.random.default_rng(7)
    n = 400000
    a = rng.uniform(-3, 3, (n, 3)).astype(np.float32)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    R = 0.062
    dist = R * (1.0 + rng.uniform(-1e-4, 1e-4, (n, 1)))
    b = (a.astype(np.float64) + u * dist).astype(np.float32)
    R2 = R * R
    d2f = _sqd_f32(a, b)
    d2 = _sqd_exact(a, b)
    thr_in = np.float32(R2 * (1.0 - 1e-5))
    thr = np.float32(R2 * (1.0 + 1e-5) + 1e-36)
    decided = np.where(d2f < thr_in, True, np.where(d2f < thr, d2 < R2, False))
    assert np.array_equal(decided, d2 < R2)
    # the shell left to the double test is thin
    assert np.mean((d2f >= thr_in) & (d2f < thr)) < 0.25


def test_knn_filter_keeps_the_exact_nearest():
    """The l-bar filter: with t the k-th smallest float squared distance,
    every one of the k nearest by the exact distance has a float squared
    distance of at most t (1 + 1e-5) + 1e-36."""
    rng = np.random.default_rng(11)
    k = 6
    for trial in range(200):
        p = rng.uniform(-1, 1, (1, 3)).astype(np.float32)
        q = (p + rng.standard_normal((300, 3)) * 10.0 ** rng.uniform(-5, 0)).astype(np.float32)
        # ties and near-ties: duplicate some candidates, nudge others by one ulp
        q[:20] = q[20:40]
        q[40:60] = np.nextafter(q[60:80], np.float32(np.inf))
        P = np.repeat(p, len(q), axis=0)
        d2f = _sqd_f32(P, q)
        d2 = _sqd_exact(P, q)
        t = np.sort(d2f)[k - 1]
        keep = d2f <= np.float32(np.float64(t) * (1 + 1e-5) + 1e-36)
        nearest = np.argsort(d2, kind="stable")[:k]
        assert np.all(keep[nearest]), trial
        # the kept set's k smallest exact values are the exact k smallest
        assert np.array_equal(np.sort(d2[keep])[:k], np.sort(d2)[:k])
