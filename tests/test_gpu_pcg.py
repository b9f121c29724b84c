"""Conjugate gradients preconditioned by one V-cycle on the GPU against the
oracle's PCG (same hierarchy, same cycle), through the C ABI.

CG is a short recurrence on top of the cycle, so the GPU iterate after k
iterations matches the oracle's to the cycle's 1e-12 times a modest growth
from the recurrences: held to 1e-11 relative for the first iterations."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2104_13755_gb300 as smg  # noqa: E402


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    def __init__(self, V, F, t, mask=None, **opts):
        self.plan = smg.Plan(V, F, dirichlet=mask, **opts)
        self.h = smg.Hierarchy(self.plan, **opts)
        A = oracle.system_matrix(V, F, t)
        Ps = [self.plan.prolongation_csr(l) for l in range(1, self.plan.num_levels)]
        known = mask if mask is not None else np.zeros(V.shape[0], dtype=bool)
        self.A, Ps, _, _ = oracle.dirichlet_reduce(A, Ps, known)
        self.levels = oracle.build_levels(self.A, Ps)
        self.h.update_positions(to_dev(V), t)
        self.n = self.A.shape[0]


@pytest.fixture(scope="module")
def torus():
    V, F = synth.torus(120, 40, seed=2)
    return Case(V, F, 1e-3, min_coarse=100)


@pytest.fixture(scope="module")
def disk():
    V, F, bnd = synth.disk(80, seed=4)
    h = synth.mean_edge_length(V, F)
    return Case(V, F, h * h, mask=bnd, min_coarse=150)


@pytest.mark.parametrize("name", ["torus", "disk"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_pcg_iterates_match_oracle(name, nrhs, request):
    c = request.getfixturevalue(name)
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=21)
    bd = to_dev(b)
    for k in (1, 2, 4):
        c.h.set_options(rtol=1e-30, max_cycles=k, solver=smg.PCG)
        x, info = c.h.solve(bd, check=False)
        assert info["cycles"] == k
        ref = oracle.pcg(c.levels, b, opt=oracle.Options(rtol=1e-30, max_cycles=k))
        assert rel(x.cpu().numpy(), ref.x) <= 1e-11, k
    c.h.set_options(rtol=1e-10)


@pytest.mark.parametrize("name", ["torus", "disk"])
def test_pcg_solve_matches_oracle_and_direct(name, request):
    c = request.getfixturevalue(name)
    b = synth.uniform_rhs(c.n, nrhs=2, seed=22)
    c.h.set_options(rtol=1e-10, solver=smg.PCG)
    x, info = c.h.solve(to_dev(b))
    ref = oracle.pcg(c.levels, b, opt=oracle.Options(rtol=1e-10))
    assert info["return"] == 0 and info["cycles"] == ref.cycles
    xs = spla.splu(c.A.tocsc()).solve(b)
    xg = x.cpu().numpy()
    assert rel(xg, xs) <= 1e-9
    assert oracle.rel_residual(c.A, xg, b) <= 1e-9
    c.h.set_options(rtol=1e-10, solver=smg.VCYCLE)
    _, vinfo = c.h.solve(to_dev(b))
    assert info["cycles"] <= vinfo["cycles"]


def test_pcg_mixed_precision(torus):
    c = torus
    b = synth.uniform_rhs(c.n, nrhs=1, seed=23)
    c.h.set_options(rtol=1e-10, solver=smg.PCG, precision=smg.MIXED)
    x, info = c.h.solve(to_dev(b))
    c.h.set_options(rtol=1e-10)
    assert info["return"] == 0
    assert oracle.rel_residual(c.A, x.cpu().numpy(), b) <= 1e-10
    ref = oracle.pcg(c.levels, b, opt=oracle.Options(rtol=1e-10), single=True)
    assert abs(info["cycles"] - ref.cycles) <= 1


@pytest.mark.parametrize("name", ["torus", "disk"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_pcg_mixed_iterates_match_oracle(name, nrhs, request):
    """CG with the binary32 cycle as preconditioner: the GPU and the oracle
    compute z = B32 r with binary32 cycles that differ only in summation
    order (a few units of 2^-24 relative); CG's binary64 recurrences carry
    that difference on with modest growth over the first iterations, so the
    iterates are held to 5e-6 (~80 u) relative, entry by entry against the
    largest (measured on GB300: at most 2.7e-7 after one iteration, less
    after more)."""
    c = request.getfixturevalue(name)
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=24)
    bd = to_dev(b)
    for k in (1, 2, 4):
        c.h.set_options(rtol=1e-30, max_cycles=k, solver=smg.PCG, precision=smg.MIXED)
        x, info = c.h.solve(bd, check=False)
        assert info["cycles"] == k
        ref = oracle.pcg(c.levels, b, opt=oracle.Options(rtol=1e-30, max_cycles=k), single=True)
        xg = x.cpu().numpy()
        assert np.abs(xg - ref.x).max() <= 5e-6 * np.abs(ref.x).max(), k
    c.h.set_options(rtol=1e-10, solver=smg.VCYCLE, precision=smg.FP64)


def test_pcg_single_level_is_one_step():
    V, F = synth.perturbed_icosphere(2, seed=1)
    c = Case(V, F, 1e-2, max_levels=1)
    b = synth.uniform_rhs(c.n, seed=3)
    c.h.set_options(rtol=1e-12, solver=smg.PCG)
    x, info = c.h.solve(to_dev(b))
    assert info["cycles"] == 1
    assert oracle.rel_residual(c.A, x.cpu().numpy(), b) <= 1e-13
