"""CPU FP64 oracle for surface multigrid (Liu, Zhang, Ben-Chen, Jacobson 2021).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The product library
never calls it and shares no code with it: the only common inputs are the
seeded meshes and vectors from `synth`, and the hierarchy of prolongations
P_1..P_H, which the method's setup stage produces from geometry alone and
which the oracle takes as given data (Alg. 1: P's are computed once, before
A and b exist).

What is computed, in the paper's order and notation:
  * A = M + t L on the mesh (Sec. 6 "cotangent Laplacian"; lumped mass).  The
    paper prints no formula: L is the positive semi-definite cotan Laplacian
    (off-diagonal -(cot a + cot b)/2), M the barycentric lumped mass.
  * Dirichlet reduction (App. "Dirichlet Boundary Conditions").
  * Galerkin coarse operators A_{h+1} = P_{h+1}^T A_h P_{h+1} (Eq. "gca" with R = P^T).
  * Greedy colouring (Alg. 3) and colour-ordered Gauss-Seidel (App. "Multi-Color
    Gauss Seidel").
  * The V-cycle of Alg. 2 and the solve loop of Alg. 1.
  * The mixed-precision form: FP32 V-cycles inside FP64 iterative refinement.

Pins (what fixes each function other than itself) live in tests/test_oracle_pins.py.
Parity unpinned: none of the functions here; the convergence *rate* of the
cycle has no printed value in the paper and is pinned only by rho < 1.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_greedy_colouring.argtypes = [i64, p, p, p]
        lib.oracle_greedy_colouring.restype = i64
        for name in ("oracle_gs_sweep_f64", "oracle_gs_sweep_f32"):
            getattr(lib, name).argtypes = [i64, p, p, p, p, i64, p, p, i64]
            getattr(lib, name).restype = i64
        lib.oracle_cholesky.argtypes = [i64, p, p]
        lib.oracle_cholesky.restype = i64
        lib.oracle_chol_solve.argtypes = [i64, p, p, p, i64]
        lib.oracle_chol_solve.restype = None
        _LIB = lib
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Assembly: A = M + t L
# ---------------------------------------------------------------------------
def mesh_pattern(n, F):
    """Structural 1-ring pattern of a mesh operator: every edge (both directions)
    plus the diagonal, as a CSR matrix of ones with sorted column indices."""
    F = np.asarray(F, dtype=np.int64)
    r = np.concatenate([F[:, 0], F[:, 1], F[:, 1], F[:, 2], F[:, 2], F[:, 0], np.arange(n)])
    c = np.concatenate([F[:, 1], F[:, 0], F[:, 2], F[:, 1], F[:, 0], F[:, 2], np.arange(n)])
    S = sp.csr_matrix((np.ones(r.shape[0]), (r, c)), shape=(n, n))
    S.sum_duplicates()
    S.data[:] = 1.0
    S.sort_indices()
    return S


def mesh_pattern2(n, F):
    """Structural 2-ring pattern (Sec. 6: Bilaplacian and squared-Hessian
    energies couple vertices joined by at most two edges): the pattern of S S
    with S the 1-ring pattern."""
    S = mesh_pattern(n, F)
    S2 = (S @ S).tocsr()
    S2.data[:] = 1.0
    S2.sort_indices()
    return S2


def bilaplacian_system(V, F, t):
    """A = M + t L M^{-1} L (data smoothing with the Bilaplacian energy, Sec. 6
    and App. "Fast Data Smoothing" with Q = L M^{-1} L), on the 2-ring pattern."""
    n = np.asarray(V).shape[0]
    L = cotan_laplacian(V, F)
    m = lumped_mass(V, F)
    A = sp.diags(m) + t * (L @ sp.diags(1.0 / m) @ L)
    return on_pattern(mesh_pattern2(n, F), A.tocsr())


def expand_blocks(X, bs):
    """bs unknowns per vertex (3|V| systems of Sec. 6, components adjacent):
    X (x) I_bs for operators and prolongations alike."""
    return sp.kron(X, sp.identity(bs), format="csr")


def block_pattern(S, bs):
    """Pattern of bs x bs blocks over the vertex pattern S."""
    B = sp.kron(S, np.ones((bs, bs)), format="csr")
    B.data[:] = 1.0
    B.sort_indices()
    return B


def on_pattern(S, C):
    """Values of C placed on the structural pattern S (pattern(C) must be a subset
    of pattern(S)); entries of S absent from C are explicit zeros."""
    S = S.tocsr()
    S.sort_indices()
    C = C.tocsr()
    C.sum_duplicates()
    ncol = S.shape[1]
    rs = np.repeat(np.arange(S.shape[0], dtype=np.int64), np.diff(S.indptr))
    rc = np.repeat(np.arange(C.shape[0], dtype=np.int64), np.diff(C.indptr))
    ks = rs * ncol + S.indices
    kc = rc * ncol + C.indices
    pos = np.searchsorted(ks, kc)
    if kc.size and (np.any(pos >= ks.size) or np.any(ks[np.minimum(pos, ks.size - 1)] != kc)):
        raise ValueError("values outside the structural pattern")
    data = np.zeros(ks.size, dtype=C.dtype)
    data[pos] = C.data
    return sp.csr_matrix((data, S.indices.copy(), S.indptr.copy()), shape=S.shape)


def face_cotangents_areas(V, F):
    """Per face (i, j, k): cot of the angle at each corner and the face area.
    cot at corner a = (e1 . e2) / |e1 x e2| with e1, e2 the two edges leaving a."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    cots = np.zeros((F.shape[0], 3))
    for c in range(3):
        a = V[F[:, c]]
        e1 = V[F[:, (c + 1) % 3]] - a
        e2 = V[F[:, (c + 2) % 3]] - a
        cots[:, c] = np.einsum("ij,ij->i", e1, e2) / np.linalg.norm(np.cross(e1, e2), axis=1)
    area = 0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)
    return cots, area


def cotan_laplacian(V, F):
    """PSD cotangent Laplacian: for each face and each corner k opposite edge (i, j),
    L_ij = L_ji -= cot(k)/2 and L_ii, L_jj += cot(k)/2.  Hence L 1 = 0."""
    n = np.asarray(V).shape[0]
    F = np.asarray(F, dtype=np.int64)
    cots, _ = face_cotangents_areas(V, F)
    rows, cols, vals = [], [], []
    for k in range(3):
        i, j = F[:, (k + 1) % 3], F[:, (k + 2) % 3]
        w = 0.5 * cots[:, k]
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-w, -w, w, w]
    L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return on_pattern(mesh_pattern(n, F), L)


def lumped_mass(V, F):
    """Barycentric lumped mass: M_ii = sum over faces at i of area / 3."""
    n = np.asarray(V).shape[0]
    F = np.asarray(F, dtype=np.int64)
    _, area = face_cotangents_areas(V, F)
    m = np.zeros(n)
    for c in range(3):
        np.add.at(m, F[:, c], area / 3.0)
    return m


def system_matrix(V, F, t):
    """A = M + t L on the 1-ring pattern (CSR, sorted columns, diagonal present)."""
    n = np.asarray(V).shape[0]
    L = cotan_laplacian(V, F)
    A = L * t + sp.diags(lumped_mass(V, F))
    return on_pattern(mesh_pattern(n, F), A)


# ---------------------------------------------------------------------------
# Dirichlet reduction (App. "Dirichlet Boundary Conditions")
# ---------------------------------------------------------------------------
def dirichlet_reduce(A, Ps, known):
    """Reduce to the unknowns: A_uu, the rows P_{u:} of the finest prolongation with
    all-zero columns removed, and the matching rows removed from the next P.
    Returns (A_uu, [P_1', P_2', ...], unknown_index, kept_coarse_columns)."""
    known = np.asarray(known, dtype=bool)
    u = np.flatnonzero(~known)
    A = A.tocsr()
    Auu = A[u][:, u].tocsr()
    Auu.sort_indices()
    Ps = [P.tocsr() for P in Ps]
    if not Ps:
        return Auu, [], u, None
    P1u = Ps[0][u].tocsr()
    colmax = np.asarray(P1u.max(axis=0).todense()).ravel()
    keep = np.flatnonzero(colmax > 0)
    out = [P1u[:, keep].tocsr()]
    if len(Ps) > 1:
        out.append(Ps[1][keep].tocsr())
        out += Ps[2:]
    return Auu, out, u, keep


# ---------------------------------------------------------------------------
# Galerkin coarse operator (Eq. gca with R = P^T)
# ---------------------------------------------------------------------------
def galerkin_pattern(S, P):
    """Structural pattern of P^T S P: products of non-negative 0/1 matrices never cancel."""
    Pb = P.tocsr().copy()
    Pb.data = np.ones_like(Pb.data)
    Sb = S.tocsr().copy()
    Sb.data = np.ones_like(Sb.data)
    C = (Pb.T @ Sb @ Pb).tocsr()
    C.data[:] = 1.0
    C.sort_indices()
    return C


def galerkin(A, P):
    """A_c = P^T A P, values on the structural pattern of P^T A P."""
    C = (P.T.tocsr() @ A.tocsr() @ P.tocsr()).tocsr()
    return on_pattern(galerkin_pattern(A, P), C)


# ---------------------------------------------------------------------------
# Colouring (Alg. 3) and Gauss-Seidel
# ---------------------------------------------------------------------------
def greedy_colouring(S):
    """Colours of the off-diagonal graph of pattern S by Alg. 3 (C loop)."""
    S = S.tocsr()
    S.sort_indices()
    n = S.shape[0]
    rp = S.indptr.astype(np.int64)
    ci = S.indices.astype(np.int64)
    colour = np.empty(n, dtype=np.int32)
    k = _lib().oracle_greedy_colouring(n, _ptr(rp), _ptr(ci), _ptr(colour))
    if k < 0:
        raise MemoryError("colouring failed")
    return colour


def block_colouring(S, bs):
    """Colours of a system with bs unknowns per vertex (3|V| systems of Sec. 6;
    unknown r is component r % bs of vertex r // bs, every level a pattern of
    bs x bs blocks).  Reading of Alg. 3 for such systems: Alg. 3 colours the
    vertices (the pattern of the blocks), and vertex colour class C is swept
    component by component, so unknown (v, c) gets colour bs * C(v) + c."""
    S = S.tocsr()
    n = S.shape[0]
    rows = np.repeat(np.arange(n) // bs, np.diff(S.indptr))
    Sv = sp.csr_matrix((np.ones(rows.size), (rows, S.indices // bs)), shape=(n // bs, n // bs))
    Sv.sum_duplicates()
    Sv.sort_indices()
    vc = greedy_colouring(Sv).astype(np.int64)
    return (bs * np.repeat(vc, bs) + np.tile(np.arange(bs), n // bs)).astype(np.int32)


def colour_order(colour, reverse=False):
    """Row order of a sweep: colour classes one after another (ascending colour
    ids, or descending when reverse), rows ascending within a class."""
    colour = np.asarray(colour)
    key = -colour if reverse else colour
    return np.lexsort((np.arange(colour.size), key)).astype(np.int64)


def gs_sweep(A, x, b, order):
    """One Gauss-Seidel pass over `order`; x (n or n x k) is updated in place."""
    A = A.tocsr()
    dt = A.dtype
    fn = _lib().oracle_gs_sweep_f64 if dt == np.float64 else _lib().oracle_gs_sweep_f32
    rp = A.indptr.astype(np.int64)
    ci = A.indices.astype(np.int64)
    val = np.ascontiguousarray(A.data)
    xb = x.reshape(x.shape[0], -1)
    bb = np.ascontiguousarray(b.reshape(b.shape[0], -1), dtype=dt)
    assert xb.flags.c_contiguous and xb.dtype == dt
    order = np.ascontiguousarray(order, dtype=np.int64)
    st = fn(A.shape[0], _ptr(rp), _ptr(ci), _ptr(val), _ptr(order), order.size,
            _ptr(bb), _ptr(xb), xb.shape[1])
    if st != 0:
        raise ZeroDivisionError("zero diagonal in row %d" % (-st - 1))
    return x


# ---------------------------------------------------------------------------
# Dense Cholesky of the coarsest operator
# ---------------------------------------------------------------------------
def cholesky(Ad):
    Ad = np.ascontiguousarray(Ad, dtype=np.float64)
    n = Ad.shape[0]
    L = np.empty_like(Ad)
    st = _lib().oracle_cholesky(n, _ptr(Ad), _ptr(L))
    if st != 0:
        raise np.linalg.LinAlgError("not SPD: pivot %d" % (-st - 1))
    return L


def chol_solve(L, b):
    L = np.ascontiguousarray(L, dtype=np.float64)
    bb = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(L.shape[0], -1))
    x = np.empty_like(bb)
    _lib().oracle_chol_solve(L.shape[0], _ptr(L), _ptr(bb), _ptr(x), bb.shape[1])
    return x.reshape(np.shape(b))


# ---------------------------------------------------------------------------
# Hierarchy, V-cycle (Alg. 2) and solve loop (Alg. 1)
# ---------------------------------------------------------------------------
@dataclass
class Level:
    A: sp.csr_matrix                 # A_h
    P: sp.csr_matrix = None          # P_{h+1}: n_h x n_{h+1} (None at the coarsest)
    colour: np.ndarray = None
    fwd: np.ndarray = None           # colour-major sweep order
    rev: np.ndarray = None           # reversed colour classes
    L: np.ndarray = None             # Cholesky factor (coarsest only)
    A32: sp.csr_matrix = None
    P32: sp.csr_matrix = None


@dataclass
class Options:
    mu_pre: int = 2
    mu_post: int = 2
    post_reverse: bool = True        # post-relaxation visits the colour classes in reverse
    rtol: float = 1e-10
    max_cycles: int = 100
    smoother: str = "gs"             # "gs" (Sec. 5) or "jacobi" (damped; App. "Ablation Study")
    omega: float = 2.0 / 3.0         # Jacobi damping (the paper gives none; 2/3 is the textbook weight)


def build_levels(A0, Ps, block=1):
    """Levels 0..H from A_0 and P_1..P_H: Galerkin products, colourings (Alg. 3;
    with block = 3 the colouring of 3|V| systems, block_colouring), the
    Cholesky factor of A_H."""
    levels = []
    A = A0.tocsr()
    A.sort_indices()
    for P in Ps:
        col = greedy_colouring(A) if block == 1 else block_colouring(A, block)
        levels.append(Level(A=A, P=P.tocsr(), colour=col, fwd=colour_order(col),
                            rev=colour_order(col, reverse=True)))
        A = galerkin(A, P)
    levels.append(Level(A=A, L=cholesky(A.toarray())))
    for lv in levels:
        lv.A32 = lv.A.astype(np.float32)
        if lv.P is not None:
            lv.P32 = lv.P.astype(np.float32)
    return levels


def jacobi_sweep(A, x, b, omega):
    """One damped Jacobi pass: x <- x + omega D^{-1} (b - A x), every row from the
    old iterate (App. "Ablation Study"); x (n or n x k) is updated in place."""
    d = A.diagonal().reshape(-1, *([1] * (x.ndim - 1)))
    r = b - A @ x
    x += (omega * r / d).astype(x.dtype)
    return x


def relax(lv, x, b, sweeps, reverse, single=False, opt=None):
    A = lv.A32 if single else lv.A
    jacobi = opt is not None and opt.smoother == "jacobi"
    for _ in range(sweeps):
        if jacobi:
            jacobi_sweep(A, x, b, np.float32(opt.omega) if single else opt.omega)
        else:
            gs_sweep(A, x, b, lv.rev if reverse else lv.fwd)
    return x


def vcycle(levels, h, x, b, opt, single=False):
    """Alg. 2.  x_old is updated and returned.  Coarser levels start from 0.
    Reading of the update step: the correction is added to the pre-relaxed
    iterate x_old' (the printed x_old would discard the pre-relaxation)."""
    lv = levels[h]
    if h == len(levels) - 1:
        if single:                   # coarsest factor stays in FP64
            return chol_solve(lv.L, b.astype(np.float64)).astype(np.float32)
        return chol_solve(lv.L, b)
    A = lv.A32 if single else lv.A
    P = lv.P32 if single else lv.P
    x = relax(lv, x, b, opt.mu_pre, False, single, opt)               # pre-relaxation
    r = P.T @ (b - A @ x)                                             # restrict residual
    nc = levels[h + 1].A.shape[0]
    zero = np.zeros((nc,) + b.shape[1:], dtype=b.dtype)
    c = vcycle(levels, h + 1, zero, r, opt, single)                   # coarse correction
    x = x + P @ c                                                     # prolong and add
    x = np.ascontiguousarray(x)
    x = relax(lv, x, b, opt.mu_post, opt.post_reverse, single, opt)   # post-relaxation
    return x


def rel_residual(A, x, b):
    """max over right-hand sides of ||b - A x||_2 / ||b||_2 (absolute when b = 0)."""
    r = (b - A @ x).reshape(b.shape[0], -1)
    bn = np.linalg.norm(b.reshape(b.shape[0], -1), axis=0)
    rn = np.linalg.norm(r, axis=0)
    return float(np.max(np.where(bn > 0, rn / np.where(bn > 0, bn, 1.0), rn)))


@dataclass
class SolveResult:
    x: np.ndarray
    cycles: int
    history: list = field(default_factory=list)    # relative residual before cycle 1, after each cycle
    iterates: list = field(default_factory=list)


def solve(levels, b, x0=None, opt=None, keep_iterates=False):
    """Alg. 1: repeat V-cycles while the relative residual exceeds rtol."""
    opt = opt or Options()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    A = levels[0].A
    hist = [rel_residual(A, x, b)]
    its = []
    k = 0
    while hist[-1] > opt.rtol and k < opt.max_cycles:
        x = vcycle(levels, 0, x, b, opt)
        k += 1
        hist.append(rel_residual(A, x, b))
        if keep_iterates:
            its.append(x.copy())
        if not np.isfinite(hist[-1]):
            break
    return SolveResult(x=x, cycles=k, history=hist, iterates=its)


def solve_mixed(levels, b, x0=None, opt=None, keep_iterates=False):
    """Mixed precision: x_{k+1} = x_k + Vcycle_FP32(b - A x_k), with the residual and
    the update in FP64 and the coarsest Cholesky in FP64."""
    opt = opt or Options()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    A = levels[0].A
    hist = [rel_residual(A, x, b)]
    its = []
    k = 0
    while hist[-1] > opt.rtol and k < opt.max_cycles:
        r = (b - A @ x).astype(np.float32)
        d = vcycle(levels, 0, np.zeros_like(r), r, opt, single=True)
        x = x + d.astype(np.float64)
        k += 1
        hist.append(rel_residual(A, x, b))
        if keep_iterates:
            its.append(x.copy())
        if not np.isfinite(hist[-1]):
            break
    return SolveResult(x=x, cycles=k, history=hist, iterates=its)


def convergence_factor(history):
    """rho = (r_k / r_0)^(1/k) over the recorded cycles."""
    k = len(history) - 1
    if k <= 0 or history[0] == 0:
        return 0.0
    return float((history[-1] / history[0]) ** (1.0 / k))


# ---------------------------------------------------------------------------
# Derivatives for the differentiable solve (form 3; the paper has no adjoint)
# ---------------------------------------------------------------------------
# x = A(V, t)^{-1} b.  For a loss l(x): lambda = A^{-1} dl/dx (A symmetric), and
#   dl/db = lambda,  dl/dt = -lambda^T L x,  dl/dV = -d/dV [lambda^T A(V) x].
# The position derivatives here are per-face complex-step derivatives
# (Squire and Trapp 1998: f'(a) = Im f(a + i h) / h, exact to rounding for
# real-analytic f), so they share no formula with any closed-form derivative
# of cot or area.  The per-face terms sum over faces because
#   lambda^T M x = sum_f area_f / 3 * sum_{c in f} lambda_c x_c
#   lambda^T L x = sum_f sum_k cot_k / 2 * (lambda_i - lambda_j)(x_i - x_j)
# with edge (i, j) opposite corner k.
_CS_STEP = 1e-30


def _face_energy(P, lv, xv, w, t):
    """Per-face energy from corner positions P (nf, 3, 3), complex allowed.
    Operator form (w is None): area/3 sum_c lv_c.xv_c + t sum_k cot_k/2 (dlv).(dxv);
    mass form: area/3 sum_c w_c.  No abs() anywhere, so complex steps propagate."""
    def cross(a, b):
        return np.stack([a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1],
                         a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2],
                         a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]], axis=1)

    def norm(a):
        return np.sqrt(np.sum(a * a, axis=1))

    area = 0.5 * norm(cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]))
    if w is not None:
        return area / 3.0 * w.sum(axis=1)
    e = area / 3.0 * np.einsum("fcq,fcq->f", lv, xv)
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        u = P[:, i] - P[:, k]
        v = P[:, j] - P[:, k]
        cot = np.sum(u * v, axis=1) / norm(cross(u, v))
        e = e + t * 0.5 * cot * np.einsum("fq,fq->f", lv[:, i] - lv[:, j], xv[:, i] - xv[:, j])
    return e


def _faces_complex_step(V, F, lv, xv, w, t):
    """d(face energy)/d(corner coordinate) for every face, gathered per vertex."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    P = V[F]
    G = np.zeros_like(V)
    for c in range(3):
        for d in range(3):
            Pc = P.astype(np.complex128)
            Pc[:, c, d] += 1j * _CS_STEP
            g = _face_energy(Pc, lv, xv, w, t).imag / _CS_STEP
            np.add.at(G[:, d], F[:, c], g)
    return G


def _per_vertex(a, n, unknowns):
    """Values on the unknowns (n_u x K) -> per-vertex (n x K), zero on known vertices."""
    a = np.asarray(a, dtype=np.float64)
    a = a.reshape(a.shape[0], -1)
    out = np.zeros((n, a.shape[1]))
    out[unknowns] = a
    return out


def operator_grad(V, F, t, lam, x, unknowns=None):
    """(d/dV [lambda^T A(V, t) x] as n x 3, lambda^T L x) with lambda, x given on
    the unknowns (all vertices when `unknowns` is None); known vertices carry 0."""
    n = np.asarray(V).shape[0]
    u = np.arange(n) if unknowns is None else np.asarray(unknowns)
    lv = _per_vertex(lam, n, u)
    xv = _per_vertex(x, n, u)
    F64 = np.asarray(F, dtype=np.int64)
    G = _faces_complex_step(V, F64, lv[F64], xv[F64], None, t)
    L = cotan_laplacian(V, F)
    dt = float(np.sum(lv * (L @ xv)))
    return G, dt


def mass_grad(V, F, w, unknowns=None):
    """d/dV [w^T m(V)] (n x 3) with m the lumped mass of the unknowns."""
    n = np.asarray(V).shape[0]
    u = np.arange(n) if unknowns is None else np.asarray(unknowns)
    wv = _per_vertex(w, n, u)[:, 0]
    F64 = np.asarray(F, dtype=np.int64)
    return _faces_complex_step(V, F64, None, None, wv[F64], 0.0)


@dataclass
class HeatLossResult:
    loss: float
    x: np.ndarray
    lam: np.ndarray
    dV: np.ndarray       # n x 3
    dt: float
    db: np.ndarray       # on the unknowns


def heat_loss_grad(V, F, t, known, s):
    """l = x^T M x with A x = b, b = M e_s (unit impulse at unknown s), all on the
    Dirichlet-reduced unknowns (zero values on the known vertices).  Exact solves
    by sparse LU.  Gradient in V (t held fixed), in t, and in b."""
    import scipy.sparse.linalg as spla
    n = np.asarray(V).shape[0]
    known = np.asarray(known, dtype=bool)
    u = np.flatnonzero(~known)
    A = system_matrix(V, F, t).tocsr()[u][:, u].tocsc()
    m = lumped_mass(V, F)[u]
    b = np.zeros(u.size)
    b[s] = m[s]
    lu = spla.splu(A)
    x = lu.solve(b)
    lam = lu.solve(2.0 * m * x)
    w = x * x
    w[s] += lam[s]                 # dl/dm through l = sum m x^2 and through b_s = m_s
    Gop, dt = operator_grad(V, F, t, lam, x, u)
    dV = mass_grad(V, F, w, u) - Gop
    return HeatLossResult(loss=float(m @ (x * x)), x=x, lam=lam, dV=dV, dt=-dt, db=lam)


def heat_loss(V, F, t, known, s):
    """The loss of heat_loss_grad alone (for finite differences)."""
    import scipy.sparse.linalg as spla
    known = np.asarray(known, dtype=bool)
    u = np.flatnonzero(~known)
    A = system_matrix(V, F, t).tocsr()[u][:, u].tocsc()
    m = lumped_mass(V, F)[u]
    b = np.zeros(u.size)
    b[s] = m[s]
    x = spla.splu(A).solve(b)
    return float(m @ (x * x))


# ---------------------------------------------------------------------------
# The V-cycle as a preconditioner for conjugate gradients (Sec. "Limitations &
# Future Work" names it as a direction; the paper gives no algorithm).
# ---------------------------------------------------------------------------
def _coldot(a, b):
    return np.sum(a * b, axis=0)


def pcg(levels, b, x0=None, opt=None, single=False, keep_iterates=False, trace=None, precond=True):
    """Preconditioned conjugate gradients on A x = b, each column on its own.
    The preconditioner is one V-cycle of Alg. 2 from a zero start with r as the
    right-hand side (binary32 when `single`); with mu_pre = mu_post and the
    post-relaxation in reverse colour order the cycle is a symmetric positive
    definite operator.  `precond=False` gives plain CG (identity).  Stops like
    Alg. 1: while max over columns of ||r|| / ||b|| > rtol, r the recurrence
    residual.  `trace`, if a list, receives (r, z, p) of every iteration."""
    opt = opt or Options()
    A = levels[0].A
    b2 = np.ascontiguousarray(b, dtype=np.float64).reshape(b.shape[0], -1)
    x = np.zeros_like(b2) if x0 is None else np.array(x0, dtype=np.float64, copy=True).reshape(b2.shape)
    r = b2 - A @ x
    bn = np.linalg.norm(b2, axis=0)

    def rel(res):
        rn = np.linalg.norm(res, axis=0)
        return float(np.max(np.where(bn > 0, rn / np.where(bn > 0, bn, 1.0), rn)))

    hist = [rel(r)]
    its = []
    k = 0
    p = None
    rho_old = None
    while hist[-1] > opt.rtol and k < opt.max_cycles:
        if not precond:
            z = r.copy()
        elif single:
            r32 = r.astype(np.float32).reshape(b.shape)
            z = vcycle(levels, 0, np.zeros_like(r32), r32, opt, single=True).astype(np.float64).reshape(b2.shape)
        else:
            z = vcycle(levels, 0, np.zeros_like(r).reshape(b.shape), np.ascontiguousarray(r.reshape(b.shape)),
                       opt).reshape(b2.shape)
        rho = _coldot(r, z)
        if p is None:
            p = z.copy()
        else:
            beta = np.where(rho_old != 0, rho / np.where(rho_old != 0, rho_old, 1.0), 0.0)
            p = z + beta * p
        q = A @ p
        pq = _coldot(p, q)
        alpha = np.where(pq != 0, rho / np.where(pq != 0, pq, 1.0), 0.0)
        if trace is not None:
            trace.append((r.copy(), z.copy(), p.copy()))
        x = x + alpha * p
        r = r - alpha * q
        rho_old = rho
        k += 1
        hist.append(rel(r))
        if keep_iterates:
            its.append(x.reshape(b.shape).copy())
        if not np.isfinite(hist[-1]):
            break
    return SolveResult(x=x.reshape(b.shape), cycles=k, history=hist, iterates=its)
