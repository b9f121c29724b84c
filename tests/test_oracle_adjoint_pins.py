"""Pins of the oracle's derivatives (form 3) to facts outside them: central
finite differences of losses evaluated by sparse LU, the classical identity
grad(total area) = L V (the cotangent formula for the area gradient, Pinkall
and Polthier 1993), Euler's theorem on homogeneous functions, and the rigid-
motion invariance of the operator.  A dropped term (area or cotangent part),
a wrong sign, or a swapped corner fails one of these."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import synth

EPS = 1e-6


@pytest.fixture(scope="module")
def small_disk():
    V, F, bnd = synth.disk(30, seed=4)
    h = synth.mean_edge_length(V, F)
    u = np.flatnonzero(~bnd)
    return V, F, bnd, h * h, len(u) // 3


def _dirs(shape, k, seed):
    rng = np.random.default_rng(seed)
    for _ in range(k):
        d = rng.standard_normal(shape)
        yield d / np.linalg.norm(d)


def test_area_gradient_is_cotan_laplacian_times_positions():
    for V, F in (synth.perturbed_icosphere(3, seed=2), synth.torus(30, 12, seed=1)):
        G = oracle.mass_grad(V, F, np.ones(V.shape[0]))
        LV = oracle.cotan_laplacian(V, F) @ V
        assert np.abs(G - LV).max() <= 1e-13 * np.abs(LV).max()


def test_operator_gradient_homogeneity_and_rigid_invariance():
    """lambda^T M x is homogeneous of degree 2 in V and lambda^T L x of degree 0,
    so sum_v V_v . G_v = 2 lambda^T M x; translations and rotations leave the
    operator unchanged, so sum_v G_v = 0 and sum_v V_v x G_v = 0 (closed mesh)."""
    V, F = synth.torus(40, 16, seed=5)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal((V.shape[0], 2))
    x = rng.standard_normal((V.shape[0], 2))
    t = 0.3
    G, dt = oracle.operator_grad(V, F, t, lam, x)
    m = oracle.lumped_mass(V, F)
    scale = np.abs(G).max() * np.abs(V).max()
    assert abs(np.sum(V * G) - 2.0 * np.sum(m[:, None] * lam * x)) <= 1e-12 * scale * V.shape[0]
    assert np.abs(G.sum(axis=0)).max() <= 1e-12 * np.abs(G).max() * V.shape[0]
    assert np.abs(np.cross(V, G).sum(axis=0)).max() <= 1e-12 * scale * V.shape[0]
    L = oracle.cotan_laplacian(V, F)
    assert abs(dt - np.sum(lam * (L @ x))) <= 1e-12 * abs(dt)


def test_operator_gradient_matches_finite_differences():
    """d/dV [lambda^T A(V, t) x] along random directions, A assembled afresh."""
    V, F = synth.perturbed_icosphere(2, seed=6)
    rng = np.random.default_rng(2)
    lam = rng.standard_normal(V.shape[0])
    x = rng.standard_normal(V.shape[0])
    t = 0.05
    G, _ = oracle.operator_grad(V, F, t, lam, x)
    for d in _dirs(V.shape, 6, 3):
        fp = lam @ (oracle.system_matrix(V + EPS * d, F, t) @ x)
        fm = lam @ (oracle.system_matrix(V - EPS * d, F, t) @ x)
        fd = (fp - fm) / (2 * EPS)
        assert abs(fd - np.sum(G * d)) <= 1e-7 * np.abs(G).max() * np.sqrt(G.size)


def test_heat_loss_gradient_matches_finite_differences(small_disk):
    V, F, bnd, t, s = small_disk
    r = oracle.heat_loss_grad(V, F, t, bnd, s)
    # in-plane moves of boundary vertices change areas and angles; out-of-plane moves
    # of a flat disk change neither to first order
    assert np.all(r.dV[bnd][:, :2] != 0.0) and np.all(r.dV[:, 2] == 0.0)
    for d in _dirs(V.shape, 8, 4):
        fd = (oracle.heat_loss(V + EPS * d, F, t, bnd, s) - oracle.heat_loss(V - EPS * d, F, t, bnd, s)) / (2 * EPS)
        an = np.sum(r.dV * d)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9 * r.loss, (fd, an)
    et = EPS * t
    fd = (oracle.heat_loss(V, F, t + et, bnd, s) - oracle.heat_loss(V, F, t - et, bnd, s)) / (2 * et)
    assert abs(fd - r.dt) <= 1e-6 * abs(r.dt)


def test_heat_loss_gradient_in_b_is_adjoint_solution(small_disk):
    """dl/db = lambda: perturb b alone (A and M fixed) and difference l = x^T M x."""
    V, F, bnd, t, s = small_disk
    r = oracle.heat_loss_grad(V, F, t, bnd, s)
    u = np.flatnonzero(~bnd)
    A = oracle.system_matrix(V, F, t).tocsr()[u][:, u].tocsc()
    m = oracle.lumped_mass(V, F)[u]
    lu = spla.splu(A)
    b = np.zeros(u.size)
    b[s] = m[s]
    for d in _dirs(b.shape, 4, 5):
        xp, xm = lu.solve(b + EPS * d), lu.solve(b - EPS * d)
        fd = (m @ (xp * xp) - m @ (xm * xm)) / (2 * EPS)
        assert abs(fd - r.db @ d) <= 1e-7 * abs(r.db @ d) + 1e-12


def test_mass_gradient_matches_finite_differences():
    V, F, bnd = synth.disk(20, seed=7)
    u = np.flatnonzero(~bnd)
    w = np.random.default_rng(8).standard_normal(u.size)
    G = oracle.mass_grad(V, F, w, u)
    for d in _dirs(V.shape, 4, 9):
        fd = (w @ oracle.lumped_mass(V + EPS * d, F)[u] - w @ oracle.lumped_mass(V - EPS * d, F)[u]) / (2 * EPS)
        assert abs(fd - np.sum(G * d)) <= 1e-7 * np.abs(G).max() * np.sqrt(G.size)
