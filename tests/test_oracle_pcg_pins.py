"""Pins of the oracle's preconditioned conjugate gradients to facts outside it:
the textbook CG iterates of scipy (identity preconditioner), one-step
convergence with an exact preconditioner (single-level hierarchy), the
mutual orthogonality of CG (r_i . z_j = 0 and p_i . A p_j = 0 for i != j),
symmetry of the V-cycle operator that makes it a valid preconditioner, and the
direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import synth
import paper_2104_13755_gb300 as smg  # host-only setup (plan), no GPU


@pytest.fixture(scope="module")
def torus_levels():
    V, F = synth.torus(40, 16, seed=3)
    plan = smg.Plan(V, F, min_coarse=40)
    A = oracle.system_matrix(V, F, 1e-2)
    Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
    return oracle.build_levels(A, Ps)


def test_identity_preconditioner_gives_scipy_cg_iterates(torus_levels):
    A = torus_levels[0].A
    b = synth.uniform_rhs(A.shape[0], seed=1)
    for k in (1, 3, 6):
        ours = oracle.pcg(torus_levels, b, opt=oracle.Options(rtol=0.0, max_cycles=k), precond=False)
        ref, _ = spla.cg(A, b, x0=np.zeros_like(b), maxiter=k, rtol=0.0, atol=0.0)
        assert np.linalg.norm(ours.x - ref) <= 1e-10 * np.linalg.norm(ref), k


def test_exact_preconditioner_converges_in_one_step():
    V, F = synth.perturbed_icosphere(2, seed=1)
    A = oracle.system_matrix(V, F, 1e-2)
    levels = oracle.build_levels(A, [])
    b = synth.uniform_rhs(A.shape[0], nrhs=2, seed=2)
    res = oracle.pcg(levels, b, opt=oracle.Options(rtol=1e-12))
    assert res.cycles == 1
    assert oracle.rel_residual(A, res.x, b) <= 1e-13


def test_vcycle_is_symmetric_operator(torus_levels):
    """<u, B v> = <B u, v> for the cycle from zero, B = the preconditioner."""
    n = torus_levels[0].A.shape[0]
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    Bu = oracle.vcycle(torus_levels, 0, np.zeros(n), u, oracle.Options())
    Bv = oracle.vcycle(torus_levels, 0, np.zeros(n), v, oracle.Options())
    assert abs(u @ Bv - Bu @ v) <= 1e-12 * abs(u @ Bv)
    assert u @ Bu > 0 and v @ Bv > 0


def test_orthogonality_and_direct_solution(torus_levels):
    A = torus_levels[0].A
    b = synth.uniform_rhs(A.shape[0], seed=5)
    tr = []
    res = oracle.pcg(torus_levels, b, opt=oracle.Options(rtol=1e-12), trace=tr)
    xs = spla.splu(A.tocsc()).solve(b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)
    k = min(len(tr), 5)
    for i in range(k):
        for j in range(k):
            if i == j:
                continue
            ri, zi, pi = (a.ravel() for a in tr[i])
            rj, zj, pj = (a.ravel() for a in tr[j])
            assert abs(ri @ zj) <= 1e-8 * np.sqrt(abs(ri @ zi) * abs(rj @ zj)), (i, j)
            assert abs(pi @ (A @ pj)) <= 1e-8 * np.sqrt(abs(pi @ (A @ pi)) * abs(pj @ (A @ pj))), (i, j)


def test_pcg_needs_fewer_cycles_than_plain_iteration(torus_levels):
    A = torus_levels[0].A
    b = synth.uniform_rhs(A.shape[0], nrhs=3, seed=6)
    opt = oracle.Options(rtol=1e-10)
    it = oracle.solve(torus_levels, b, opt=opt)
    cg = oracle.pcg(torus_levels, b, opt=opt)
    assert cg.cycles <= it.cycles
    assert oracle.rel_residual(A, cg.x, b) <= 1e-9
    mixed = oracle.pcg(torus_levels, b, opt=opt, single=True)
    assert oracle.rel_residual(A, mixed.x, b) <= 1e-9
