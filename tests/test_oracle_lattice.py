"""Pins of the oracle's permutohedral lattice filter and CRF mean-field update (Sec. 3.5.3, Eq. 19-22).

Which simplex encloses a point is an integer decision taken in FP32 (fixed order), shared with any FP32
evaluation of the same order; the barycentric weights are real-valued and solved in FP64 from the FP64
elevated point, so the geometry is checked to FP64 rounding.

The simplex search is checked against the lattice's definition (vertices are lattice points of remainder
0..d, the barycentric weights are a convex combination reproducing the elevated point, and the remainder-0
vertex is the nearest remainder-0 point); for d = 1 the whole filter equals a 1-D grid filter computed here by
hand (tent splat, [1 2 1]/4 blur twice, tent slice); the filter is invariant to a shift of the features by a
lattice vector; and the normalised filter approximates a unit-std
Gaussian filter (2-3 % relative RMS in low dimension)."""
import itertools

import numpy as np
import pytest

import oracle


def basis(d):
    """Orthonormal basis of {x in R^(d+1): sum x = 0}: u_i = (1, .., 1, -i, 0, ..) / sqrt(i (i + 1))."""
    U = np.zeros((d + 1, d))
    for i in range(1, d + 1):
        U[:i, i - 1] = 1.0
        U[i, i - 1] = -i
        U[:, i - 1] /= np.sqrt(i * (i + 1))
    return U


def elevate(p):
    """Elevated points (..., d+1) of features p (..., d)."""
    d = p.shape[-1]
    return (d + 1) * np.sqrt(2.0 / 3.0) * (p @ basis(d).T)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 9])
def test_simplex_is_the_enclosing_lattice_simplex(d):
    rng = np.random.default_rng(d)
    for _ in range(300):
        p = rng.normal(size=d) * 4
        x = elevate(p)
        V, b = oracle.lattice_simplex(p)
        assert np.all(V.sum(1) == 0)
        for j in range(d + 1):
            assert np.all(np.mod(V[j], d + 1) == j)  # vertex j is a remainder-j lattice point
        # weights solved in FP64 (a point within FP32 rounding of a face may get a weight of -1e-6 or so: the
        # FP32 decision picked the neighbouring simplex)
        assert abs(b.sum() - 1) < 1e-12 and b.min() > -1e-5
        np.testing.assert_allclose(b @ V, x, rtol=0, atol=1e-9)
        if d <= 3:  # the remainder-0 vertex is the nearest remainder-0 point
            r0 = V[0]
            best = np.linalg.norm(x - r0)
            for delta in itertools.product((-1, 0, 1), repeat=d + 1):
                if sum(delta) == 0:
                    assert np.linalg.norm(x - (r0 + (d + 1) * np.array(delta))) >= best - 1e-3


def test_d1_filter_is_the_grid_filter():
    rng = np.random.default_rng(0)
    p = rng.uniform(-3, 3, (60, 1))
    v = rng.normal(size=(60, 2))
    out, M = oracle.lattice_filter(p, v)
    a = elevate(p)[:, 0]  # x0 of the elevated point; the lattice points are the integers along x0
    lo = np.floor(a).astype(int)
    t = a - lo
    pts = sorted(set(lo.tolist()) | set((lo + 1).tolist()))
    idx = {q: i for i, q in enumerate(pts)}
    g = np.zeros((len(pts), 2))
    for i in range(60):
        g[idx[lo[i]]] += (1 - t[i]) * v[i]
        g[idx[lo[i] + 1]] += t[i] * v[i]
    for _ in range(2):  # two lattice directions, both along the line
        h = 2 * g.copy()
        for q, i in idx.items():
            if q - 1 in idx:
                h[i] += g[idx[q - 1]]
            if q + 1 in idx:
                h[i] += g[idx[q + 1]]
        g = h / 4
    want = np.array([(1 - t[i]) * g[idx[lo[i]]] + t[i] * g[idx[lo[i] + 1]] for i in range(60)])
    assert M == len(pts)
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 5])
def test_filter_is_shift_invariant(d):
    """(The filter is not symmetric on a sparse lattice: the directional blurs commute only where every
    neighbour exists.)"""
    rng = np.random.default_rng(10 + d)
    p = rng.normal(size=(300, d)) * 2
    a = rng.normal(size=(300, 1))
    Fa, _ = oracle.lattice_filter(p, a)
    # a remainder-0 lattice vector w = (d + 1)(e_0 - e_1) pulled back to feature space
    w = np.zeros(d + 1)
    w[0], w[1] = d + 1, -(d + 1)
    delta = basis(d).T @ w / ((d + 1) * np.sqrt(2.0 / 3.0))
    Fs, _ = oracle.lattice_filter(p + delta, a)
    np.testing.assert_allclose(Fs, Fa, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("d,tol", [(2, 0.03), (3, 0.04)])
def test_normalised_filter_approximates_a_unit_gaussian(d, tol):
    rng = np.random.default_rng(0)
    p = rng.uniform(-6, 6, size=(1500, d))
    v = np.sin(0.7 * p[:, :1]) + 0.3 * p[:, 1:2]
    out, _ = oracle.lattice_filter(p, v, normalize=True)
    K = np.exp(-((p[:, None, :] - p[None, :, :]) ** 2).sum(-1) / 2)
    bf = (K @ v) / K.sum(1, keepdims=True)
    inner = np.all(np.abs(p) < 3, axis=1)
    rel = np.sqrt(((bf - out)[inner] ** 2).mean() / ((bf[inner] - bf[inner].mean()) ** 2).mean())
    assert rel < tol


def test_meanfield_update():
    rng = np.random.default_rng(3)
    n, L = 200, 5
    p = rng.normal(size=(n, 3)) * 2
    U = rng.normal(size=(n, L))
    Q = np.exp(-U)
    Q /= Q.sum(1, keepdims=True)
    Q0 = oracle.crf_meanfield(p, U, Q, 0.0)  # no pairwise term: the unaries' softmax
    np.testing.assert_allclose(Q0, Q, atol=1e-14)
    Q1 = oracle.crf_meanfield(p, U, Q, 2.0)
    np.testing.assert_allclose(Q1.sum(1), 1.0, atol=1e-12)
    assert Q1.min() > 0
    # Potts smoothing pulls each node towards its neighbours' labels: disagreement with the filtered label
    # distribution drops
    F, _ = oracle.lattice_filter(p, Q, normalize=True)
    assert np.abs(Q1 - F).mean() < np.abs(Q - F).mean()
