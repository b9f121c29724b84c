"""Pins of the oracle to facts fixed outside it: closed forms, identities,
textbook special cases, a hand-worked run of Alg. 3 and independent library
routines.  A dropped term, a sign or index error, or a transposed operand in
the oracle fails at least one of these."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------
def test_laplacian_annihilates_constants_and_is_symmetric():
    V, F = synth.perturbed_icosphere(3, seed=3)
    L = oracle.cotan_laplacian(V, F)
    assert abs(L - L.T).max() == 0.0
    scale = abs(L).max()
    assert np.abs(L @ np.ones(V.shape[0])).max() < 1e-12 * scale


def _dirichlet_energy(V, F, f):
    """sum_T area_T |grad f_T|^2 with grad phi_c = n x e_c / (2 area), e_c the edge
    opposite corner c taken counter-clockwise: the gradient form, not cotangents."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    dbl = np.linalg.norm(nrm, axis=1)
    nh = nrm / dbl[:, None]
    g = np.zeros_like(a)
    for k, e in ((0, c - b), (1, a - c), (2, b - a)):
        g += f[F[:, k]][:, None] * np.cross(nh, e) / dbl[:, None]
    return float(np.sum(0.5 * dbl * np.einsum("ij,ij->i", g, g)))


def test_laplacian_quadratic_form_is_dirichlet_energy():
    V, F = synth.perturbed_icosphere(3, seed=5)
    rng = np.random.default_rng(0)
    L = oracle.cotan_laplacian(V, F)
    for _ in range(3):
        f = rng.standard_normal(V.shape[0])
        e = _dirichlet_energy(V, F, f)
        assert abs(f @ (L @ f) - e) < 1e-11 * e


def test_right_triangle_grid_gives_five_point_stencil():
    N = 9
    g = np.arange(N, dtype=float)
    X, Y = np.meshgrid(g, g, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(N * N)], 1)
    F = []
    for a in range(N - 1):
        for b in range(N - 1):
            v00, v10, v11, v01 = a * N + b, (a + 1) * N + b, (a + 1) * N + b + 1, a * N + b + 1
            F += [(v00, v10, v11), (v00, v11, v01)]
    L = oracle.cotan_laplacian(V, np.array(F)).toarray()
    for a in range(1, N - 1):
        for b in range(1, N - 1):
            i = a * N + b
            expect = np.zeros(N * N)
            expect[i] = 4.0
            for j in (i - 1, i + 1, i - N, i + N):
                expect[j] = -1.0
            assert np.allclose(L[i], expect, atol=1e-14)


def test_laplacian_linear_precision_on_planar_disk():
    V, F, bnd = synth.disk(24, jitter=0.05, seed=2)
    L = oracle.cotan_laplacian(V, F)
    for k in range(2):
        r = L @ V[:, k]
        assert np.abs(r[~bnd]).max() < 1e-12


def test_lumped_mass_sums_to_area():
    V, F = synth.perturbed_icosphere(3, seed=1)
    m = oracle.lumped_mass(V, F)
    # Heron's formula, independent of the cross product used by the oracle
    la = np.linalg.norm(V[F[:, 1]] - V[F[:, 2]], axis=1)
    lb = np.linalg.norm(V[F[:, 2]] - V[F[:, 0]], axis=1)
    lc = np.linalg.norm(V[F[:, 0]] - V[F[:, 1]], axis=1)
    s = 0.5 * (la + lb + lc)
    heron = np.sqrt(s * (s - la) * (s - lb) * (s - lc))
    assert np.all(m > 0)
    assert abs(m.sum() - heron.sum()) < 1e-12 * heron.sum()
    V6, F6 = synth.icosphere(6)
    assert abs(oracle.lumped_mass(V6, F6).sum() - 4 * np.pi) < 2e-3 * 4 * np.pi


def test_system_matrix_is_spd_with_mesh_pattern():
    V, F = synth.perturbed_icosphere(2, seed=0)
    A = oracle.system_matrix(V, F, 1e-2)
    S = oracle.mesh_pattern(V.shape[0], F)
    assert (A.indptr == S.indptr).all() and (A.indices == S.indices).all()
    Ad = A.toarray()
    assert np.linalg.eigvalsh(Ad).min() > 0
    assert np.allclose(Ad, Ad.T, atol=0)


# ---------------------------------------------------------------------------
# Galerkin, colouring, Gauss-Seidel, Cholesky
# ---------------------------------------------------------------------------
def test_galerkin_brute_force_and_quadratic_form(torus_pin_hierarchy):
    V, F = synth.perturbed_icosphere(1, seed=4)          # 42 vertices
    A = oracle.system_matrix(V, F, 0.1)
    rng = np.random.default_rng(1)
    n, nc = 42, 12
    P = np.zeros((n, nc))
    for i in range(n):                                    # 3 barycentric weights per row
        cols = rng.choice(nc, 3, replace=False)
        w = rng.uniform(0.1, 1.0, 3)
        P[i, cols] = w / w.sum()
    Ac = oracle.galerkin(A, sp.csr_matrix(P)).toarray()
    Ad = A.toarray()
    brute = np.zeros((nc, nc))
    for I in range(nc):
        for J in range(nc):
            s = 0.0
            for i in range(n):
                if P[i, I] == 0:
                    continue
                for j in range(n):
                    s += P[i, I] * Ad[i, j] * P[j, J]
            brute[I, J] = s
    assert np.abs(Ac - brute).max() < 1e-14 * np.abs(brute).max()
    x = rng.standard_normal(nc)
    assert abs(x @ Ac @ x - (P @ x) @ Ad @ (P @ x)) < 1e-13 * abs(x @ Ac @ x)


def test_colouring_matches_hand_worked_alg3():
    txt = [l.split() for l in open(os.path.join(GOLDEN, "alg3_colouring_small.txt"))
           if l.strip() and not l.startswith("#")]
    d = {t[0]: [int(v) for v in t[1:]] for t in txt}
    n = d["n"][0]
    e = np.array(d["edges"]).reshape(-1, 2)
    r = np.concatenate([e[:, 0], e[:, 1], np.arange(n)])
    c = np.concatenate([e[:, 1], e[:, 0], np.arange(n)])
    S = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    assert list(oracle.greedy_colouring(S)) == d["colours"]


def test_colouring_is_proper_on_mesh_and_galerkin_patterns(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    for P in [None] + Ps:
        if P is not None:
            A = oracle.galerkin(A, P)
        col = oracle.greedy_colouring(A)
        coo = A.tocoo()
        off = coo.row != coo.col
        assert np.all(col[coo.row[off]] != col[coo.col[off]])


def test_gauss_seidel_equals_matrix_splitting():
    V, F = synth.perturbed_icosphere(2, seed=8)
    A = oracle.system_matrix(V, F, 1e-2)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((A.shape[0], 2))
    x0 = rng.standard_normal((A.shape[0], 2))
    col = oracle.greedy_colouring(A)
    for reverse in (False, True):
        order = oracle.colour_order(col, reverse)
        x = x0.copy()
        oracle.gs_sweep(A, x, b, order)
        Ap = A.toarray()[np.ix_(order, order)]
        xp = sla.solve_triangular(np.tril(Ap), b[order] - np.triu(Ap, 1) @ x0[order], lower=True)
        assert np.abs(x[order] - xp).max() < 1e-13 * np.abs(xp).max()
        x32 = x0.astype(np.float32)
        oracle.gs_sweep(A.astype(np.float32), x32, b.astype(np.float32), order)
        assert np.abs(x32[order] - xp).max() < 1e-5 * np.abs(xp).max()


def test_single_precision_sweep_within_rounding_error_bound():
    """The binary32 sweep is a triangular solve carried out in binary32:
    row i computes x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii with the newest
    x_j (earlier rows of the order) and the old x_j (later rows).  With the
    binary32 inputs taken exactly, the textbook rounding analysis of a sum of
    m products followed by a division (Higham, "Accuracy and Stability of
    Numerical Algorithms", Lemma 3.1 and Sec. 8.1) bounds the residual of
    every row componentwise by gamma_{m+2} times the sum of the magnitudes
    of its terms, gamma_k = k u / (1 - k u) with u = 2^-24.  The computed
    values are binary32 numbers, and they are not the binary64 sweep of the
    same inputs (which would leave a residual near 2^-53)."""
    V, F = synth.perturbed_icosphere(2, seed=8)
    A = oracle.system_matrix(V, F, 1e-2).astype(np.float32)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((A.shape[0], 2)).astype(np.float32)
    x0 = rng.standard_normal((A.shape[0], 2)).astype(np.float32)
    col = oracle.greedy_colouring(A)
    u = 2.0 ** -24
    for reverse in (False, True):
        order = oracle.colour_order(col, reverse)
        x = x0.copy()
        oracle.gs_sweep(A, x, b, order)
        assert x.dtype == np.float32
        Ap = A.toarray().astype(np.float64)[np.ix_(order, order)]
        lo, up = np.tril(Ap), np.triu(Ap, 1)
        xn, xo, bp = x[order].astype(np.float64), x0[order].astype(np.float64), b[order].astype(np.float64)
        res = lo @ xn - (bp - up @ xo)
        mag = np.abs(lo) @ np.abs(xn) + np.abs(up) @ np.abs(xo) + np.abs(bp)
        m = np.diff(A.indptr)[order][:, None] - 1
        gamma = (m + 2) * u / (1 - (m + 2) * u)
        assert np.all(np.abs(res) <= gamma * mag)
        assert np.max(np.abs(res) / mag) > 1e-3 * u


def test_cholesky_against_lapack_and_not_spd():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 30 * np.eye(30)
    L = oracle.cholesky(A)
    assert np.abs(L @ L.T - A).max() < 1e-13 * np.abs(A).max()
    assert np.abs(L - np.linalg.cholesky(A)).max() < 1e-12 * np.abs(L).max()
    b = rng.standard_normal((30, 3))
    assert np.abs(oracle.chol_solve(L, b) - np.linalg.solve(A, b)).max() < 1e-12
    A[5, 5] = -1.0
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(A)


# ---------------------------------------------------------------------------
# cycle and solve
# ---------------------------------------------------------------------------
def test_single_level_cycle_is_direct_solve():
    V, F = synth.perturbed_icosphere(2, seed=2)
    A = oracle.system_matrix(V, F, 1e-2)
    levels = oracle.build_levels(A, [])
    b = synth.uniform_rhs(A.shape[0], seed=4)
    x = oracle.vcycle(levels, 0, np.zeros_like(b), b, oracle.Options())
    assert oracle.rel_residual(A, x, b) < 1e-13


def test_identity_prolongation_cycle_is_exact():
    V, F = synth.perturbed_icosphere(2, seed=2)
    A = oracle.system_matrix(V, F, 1e-2)
    levels = oracle.build_levels(A, [sp.identity(A.shape[0], format="csr")])
    b = synth.uniform_rhs(A.shape[0], seed=4)
    x = oracle.vcycle(levels, 0, np.zeros_like(b), b, oracle.Options())
    assert oracle.rel_residual(A, x, b) < 1e-12


def test_two_level_without_relaxation_is_coarse_correction(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps[:1])
    rng = np.random.default_rng(5)
    b = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[0])
    opt = oracle.Options(mu_pre=0, mu_post=0)
    x = oracle.vcycle(levels, 0, x0.copy(), b, opt)
    P = Ps[0].toarray()
    Ad = A.toarray()
    expect = x0 + P @ np.linalg.solve(P.T @ Ad @ P, P.T @ (b - Ad @ x0))
    assert np.abs(x - expect).max() < 1e-12 * np.abs(expect).max()


def test_cycle_converges_to_direct_solution(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps)
    b = synth.uniform_rhs(A.shape[0], nrhs=2, seed=6)
    res = oracle.solve(levels, b, opt=oracle.Options(rtol=1e-12))
    xs = spla.splu(A.tocsc()).solve(b)
    assert res.history[-1] <= 1e-12
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-10
    rho = oracle.convergence_factor(res.history)
    assert 0 < rho < 0.5
    assert all(h1 < h0 for h0, h1 in zip(res.history, res.history[1:]))


def test_mixed_precision_reaches_direct_solution(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps)
    b = synth.uniform_rhs(A.shape[0], seed=9)
    res = oracle.solve_mixed(levels, b, opt=oracle.Options(rtol=1e-10))
    xs = spla.splu(A.tocsc()).solve(b)
    assert res.history[-1] <= 1e-10
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-9


def _binary32_exact_levels(A0, Ps):
    """A hierarchy whose operators are all binary32 numbers: every level's
    matrix is the binary32 rounding of the Galerkin product of the level
    above (the prolongations used here hold 1 and 1/2, exact in binary32), so
    the binary32 copies equal the binary64 operators and a binary32 cycle
    differs from a binary64 cycle by arithmetic alone."""
    r32 = lambda M: M.astype(np.float32).astype(np.float64).tocsr()
    A = r32(A0)
    levels = []
    for P in Ps:
        assert np.array_equal(P.data.astype(np.float32).astype(np.float64), P.data)
        col = oracle.greedy_colouring(A)
        levels.append(oracle.Level(A=A, P=P.tocsr(), colour=col, fwd=oracle.colour_order(col),
                                   rev=oracle.colour_order(col, reverse=True)))
        A = r32(oracle.galerkin(A, P))
    levels.append(oracle.Level(A=A, L=oracle.cholesky(A.toarray())))
    for lv in levels:
        lv.A32 = lv.A.astype(np.float32)
        lv.P32 = None if lv.P is None else lv.P.astype(np.float32)
    return levels


def test_single_precision_cycle_is_binary32_arithmetic(torus_pin_hierarchy):
    """One cycle with single=True returns binary32 values, and on operators
    and a right-hand side that are exact binary32 numbers it differs from the
    binary64 cycle by arithmetic rounding alone: more than 1e-9 relative
    (binary64 arithmetic anywhere in place of binary32, e.g. a binary64
    operator mixed into the sweep, would agree to ~1e-15) and less than 1e-5
    (a few hundred units of u = 2^-24; a wrong operator or a dropped term is
    O(1)); and most entries differ from the binary32 rounding of the binary64
    result, which a binary64 cycle rounded only at its end would reproduce."""
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = _binary32_exact_levels(A, Ps)
    for nrhs in (1, 3):
        b32 = synth.uniform_rhs(A.shape[0], nrhs=nrhs, seed=9).astype(np.float32)
        d32 = oracle.vcycle(levels, 0, np.zeros_like(b32), b32, oracle.Options(), single=True)
        assert d32.dtype == np.float32
        b64 = b32.astype(np.float64)
        d64 = oracle.vcycle(levels, 0, np.zeros_like(b64), b64, oracle.Options())
        diff = np.linalg.norm(d32 - d64) / np.linalg.norm(d64)
        assert 1e-9 < diff < 1e-5, diff
        # binary32 rounding of every operation, not only of the result: a
        # binary64 cycle rounded once at the end would equal round32(d64)
        assert np.mean(d32 != d64.astype(np.float32)) > 0.1


def test_mixed_refinement_tracks_binary64_cycles(torus_pin_hierarchy):
    """A V-cycle is an affine map x -> x + B (b - A x) (every Gauss-Seidel
    sweep, the coarse correction and the direct solve are linear in x and
    b, with A^-1 b as fixed point), and a cycle from zero on the residual
    r = b - A x returns B r.  So refinement step k of the mixed form,
    x_k = x_{k-1} + B32 (b - A x_{k-1}), equals binary64 cycle k of Alg. 1
    except for binary32 rounding in B32: the two iterates differ by a small
    multiple of u = 2^-24 times the size of that step's correction (the
    earlier differences are contracted by the cycle), and by more than
    binary64 rounding at the first step."""
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps)
    for nrhs in (1, 2):
        b = synth.uniform_rhs(A.shape[0], nrhs=nrhs, seed=10)
        opt = oracle.Options(rtol=1e-12)
        mx = oracle.solve_mixed(levels, b, opt=opt, keep_iterates=True)
        fp = oracle.solve(levels, b, opt=opt, keep_iterates=True)
        assert mx.cycles >= 3 and fp.cycles >= 3
        prev = np.zeros_like(b)
        for k in range(min(mx.cycles, fp.cycles)):
            step = np.abs(fp.iterates[k] - prev).max()
            gap = np.abs(mx.iterates[k] - fp.iterates[k]).max()
            assert gap <= 1e-5 * step + 1e-14 * np.abs(fp.iterates[k]).max(), k
            if k == 0:
                assert gap > 1e-9 * step
            prev = fp.iterates[k]


def test_dirichlet_reduction_solves_constrained_minimum():
    V, F, bnd = synth.disk(16, seed=1)
    n = V.shape[0]
    A = oracle.system_matrix(V, F, 1e-2)
    b = synth.uniform_rhs(n, seed=2)
    Auu, _, u, _ = oracle.dirichlet_reduce(A, [], bnd)
    xu = spla.spsolve(Auu.tocsc(), b[u])
    x = np.zeros(n)
    x[u] = xu
    g = A @ x - b                       # gradient of 1/2 x'Ax - x'b
    assert np.abs(g[u]).max() < 1e-12 * np.abs(b).max()


def test_dirichlet_drops_empty_coarse_columns():
    # fine 0..5, coarse 0..2; fine row 5 is known and is the only support of coarse 2
    P1 = sp.csr_matrix(np.array([[1, 0, 0], [0, 1, 0], [.5, .5, 0], [.25, .75, 0],
                                 [1, 0, 0], [0, 0, 1.]]))
    P2 = sp.csr_matrix(np.array([[1.0, 0], [0, 1.0], [0.5, 0.5]]))
    A = sp.identity(6, format="csr")
    known = np.array([0, 0, 0, 0, 0, 1], dtype=bool)
    Auu, Ps, u, keep = oracle.dirichlet_reduce(A, [P1, P2], known)
    assert list(keep) == [0, 1]
    assert Ps[0].shape == (5, 2) and Ps[1].shape == (2, 2)
    assert np.allclose(Ps[1].toarray(), np.eye(2))


# ---------------------------------------------------------------------------
# damped Jacobi relaxation (App. "Ablation Study")
# ---------------------------------------------------------------------------
def test_jacobi_sweep_damps_grid_eigenmodes_by_closed_form():
    """On the right-triangle grid the operator is the 5-point stencil with a
    constant diagonal 4 (times the spacing factor), so a sine mode of the
    interior is an eigenvector of D^{-1} A with eigenvalue
    1 - (cos(pi p h) + cos(pi q h)) / 2 and one damped sweep on A e = 0 scales
    the error by 1 - omega * lambda (the textbook damping factor)."""
    m = 9
    g = np.linspace(0.0, 1.0, m)
    X, Y = np.meshgrid(g, g, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(m * m)], axis=1)
    F = []
    for i in range(m - 1):
        for j in range(m - 1):
            a, b_, c, d = i * m + j, (i + 1) * m + j, (i + 1) * m + j + 1, i * m + j + 1
            F += [[a, b_, c], [a, c, d]]
    F = np.array(F)
    L = oracle.cotan_laplacian(V, F).tocsr()
    inner = np.array([i * m + j for i in range(1, m - 1) for j in range(1, m - 1)])
    Li = L[inner][:, inner].tocsr()
    h = 1.0 / (m - 1)
    omega = 2.0 / 3.0
    for p_, q_ in ((1, 1), (2, 5), (7, 7)):
        e = np.array([np.sin(np.pi * p_ * X.ravel()[k]) * np.sin(np.pi * q_ * Y.ravel()[k]) for k in inner])
        lam = 1.0 - (np.cos(np.pi * p_ * h) + np.cos(np.pi * q_ * h)) / 2.0
        x = e.copy()
        oracle.jacobi_sweep(Li, x, np.zeros_like(e), omega)
        assert np.abs(x - (1.0 - omega * lam) * e).max() <= 1e-12


def test_jacobi_cycle_keeps_the_solution_fixed_and_converges(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps)
    b = synth.uniform_rhs(A.shape[0], nrhs=2, seed=31)
    xs = spla.splu(A.tocsc()).solve(b)
    opt = oracle.Options(smoother="jacobi", rtol=1e-10, max_cycles=200)
    x1 = oracle.vcycle(levels, 0, xs.copy(), b, opt)
    assert np.abs(x1 - xs).max() <= 1e-12 * np.abs(xs).max()   # the solution is a fixed point
    res = oracle.solve(levels, b, opt=opt)
    assert oracle.rel_residual(A, res.x, b) <= 1e-10
    assert oracle.convergence_factor(res.history) < 1.0
    gs = oracle.solve(levels, b, opt=oracle.Options(rtol=1e-10))
    assert gs.cycles <= res.cycles   # Gauss-Seidel smooths better per sweep


# ---------------------------------------------------------------------------
# 2-ring systems (Sec. 6: Bilaplacian)
# ---------------------------------------------------------------------------
def test_two_ring_pattern_is_graph_distance_two():
    V, F = synth.torus(12, 6, seed=2)
    n = V.shape[0]
    S2 = oracle.mesh_pattern2(n, F)
    nb = [set() for _ in range(n)]
    for f in F:
        for a in range(3):
            nb[f[a]].add(f[(a + 1) % 3])
            nb[f[(a + 1) % 3]].add(f[a])
    for i in range(n):
        ring2 = {i} | nb[i] | set().union(*(nb[j] for j in nb[i]))
        assert set(S2.indices[S2.indptr[i]:S2.indptr[i + 1]]) == ring2


def test_bilaplacian_system_identities():
    """M + t L M^{-1} L: symmetric, A 1 = M 1 (L 1 = 0), x^T A x = x^T M x +
    t |M^{-1/2} L x|^2 (its energy), positive definite."""
    V, F = synth.perturbed_icosphere(2, seed=4)
    t = 0.03
    A = oracle.bilaplacian_system(V, F, t)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    m = oracle.lumped_mass(V, F)
    assert np.abs(A @ np.ones(V.shape[0]) - m).max() <= 1e-13 * m.max()
    x = np.random.default_rng(1).standard_normal(V.shape[0])
    L = oracle.cotan_laplacian(V, F)
    e = x @ (m * x) + t * np.sum((L @ x) ** 2 / m)
    assert abs(x @ (A @ x) - e) <= 1e-12 * e
    assert np.linalg.eigvalsh(A.toarray()).min() > 0


def test_block_colouring_sweeps_vertices_component_by_component():
    """3|V| systems: the colour of unknown (v, c) is 3 C(v) + c with C Alg. 3 on
    the vertex pattern (pinned by the hand-worked run and the properness
    tests above), so (i) it is a proper colouring of the block pattern (no two
    coupled unknowns share a colour), (ii) it restricted to one component is
    the vertex colouring, and (iii) the sweep in its colour order equals the
    sweep that visits the vertex classes in order and, inside a class, the
    components 0, 1, 2 of all its vertices (the triangular solve of the
    permuted system)."""
    V, F = synth.perturbed_icosphere(2, seed=4)
    S = oracle.mesh_pattern(V.shape[0], F)
    S3 = oracle.block_pattern(S, 3)
    col = oracle.block_colouring(S3, 3)
    vc = oracle.greedy_colouring(S)
    assert np.array_equal(col[0::3], 3 * vc) and np.array_equal(col[2::3], 3 * vc + 2)
    r, c = S3.nonzero()
    off = r != c
    assert not np.any(col[r[off]] == col[c[off]])
    A = oracle.expand_blocks(oracle.system_matrix(V, F, 1e-2), 3) + \
        0.001 * sp.kron(oracle.cotan_laplacian(V, F), np.ones((3, 3)))
    A = oracle.on_pattern(S3, A.tocsr())
    rng = np.random.default_rng(8)
    b = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[0])
    x = x0.copy()
    oracle.gs_sweep(A, x, b, oracle.colour_order(col))
    order = np.concatenate([3 * np.flatnonzero(vc == k) + comp for k in range(vc.max() + 1) for comp in range(3)])
    Ap = A.toarray()[np.ix_(order, order)]
    xp = sla.solve_triangular(np.tril(Ap), b[order] - np.triu(Ap, 1) @ x0[order], lower=True)
    assert np.abs(x[order] - xp).max() < 1e-13 * np.abs(xp).max()


def test_block_expansion_identities():
    """X (x) I_3: (A (x) I)(u (x) e_k) = (A u) (x) e_k, and a Galerkin product of
    expanded operators is the expansion of the vertex Galerkin product."""
    V, F = synth.perturbed_icosphere(2, seed=2)
    A = oracle.system_matrix(V, F, 1e-2)
    n = A.shape[0]
    rng = np.random.default_rng(3)
    u = rng.standard_normal(n)
    A3 = oracle.expand_blocks(A, 3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        assert np.abs(A3 @ np.kron(u, e) - np.kron(A @ u, e)).max() <= 1e-14 * np.abs(A @ u).max()
    P = sp.random(n, 20, density=0.1, random_state=4, format="csr")
    lhs = oracle.expand_blocks(P, 3).T @ A3 @ oracle.expand_blocks(P, 3)
    rhs = oracle.expand_blocks((P.T @ A @ P).tocsr(), 3)
    assert abs(lhs - rhs).max() <= 1e-13 * abs(rhs).max()
    S3 = oracle.block_pattern(oracle.mesh_pattern(n, F), 3)
    assert S3.nnz == 9 * oracle.mesh_pattern(n, F).nnz
