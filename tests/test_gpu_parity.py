"""CUDA path against the oracle, element by element, through the C ABI.

Tolerances: binary64 kernels differ from the oracle only in summation order,
so the assembled and Galerkin operators agree to 1e-13 relative and each V-cycle
iterate to 1e-12 relative, both in norm (||x_gpu - x_oracle|| / ||x_oracle||)
and entry by entry (max |x_gpu - x_oracle| / max |x_oracle|).  The mixed form
is held to the oracle's binary32 refinement step by step (MIXED_STEP_TOL) and
to 1e-9 relative error against a direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2104_13755_gb300 as smg  # noqa: E402

CYCLE_TOL = 1e-12


class Case:
    def __init__(self, V, F, t, mask=None, **opts):
        self.V, self.F, self.t = V, F, t
        self.plan = smg.Plan(V, F, dirichlet=mask, **opts)
        self.h = smg.Hierarchy(self.plan, **opts)
        A = oracle.system_matrix(V, F, t)
        Ps = [self.plan.prolongation_csr(l) for l in range(1, self.plan.num_levels)]
        known = mask if mask is not None else np.zeros(V.shape[0], dtype=bool)
        A, Ps, self.u, _ = oracle.dirichlet_reduce(A, Ps, known)
        self.A = A
        self.levels = oracle.build_levels(A, Ps)
        self.Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        self.h.update_positions(self.Vd, t)
        self.n = A.shape[0]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """Entry-wise: max |a - b| over max |b| (a wrong value in a few rows
    cannot hide under the norm of a large vector)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ico():
    V, F = synth.perturbed_icosphere(4, seed=0)
    return Case(V, F, 1e-3, max_levels=3, min_coarse=0)


@pytest.fixture(scope="module")
def torus():
    V, F = synth.torus(120, 40, seed=2)
    return Case(V, F, 1e-3, min_coarse=100)


@pytest.fixture(scope="module")
def disk():
    V, F, bnd = synth.disk(80, seed=4)
    h = synth.mean_edge_length(V, F)
    return Case(V, F, h * h, mask=bnd, min_coarse=150)


def test_assembly_matches_oracle(ico, disk):
    for c in (ico, disk):
        got = c.h.level_matrix(0)
        ref = c.levels[0].A.data
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def test_galerkin_matches_oracle(ico, torus, disk):
    for c in (ico, torus, disk):
        for l in range(1, c.plan.num_levels):
            got = c.h.level_matrix(l)
            ref = c.levels[l].A.data
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), l


@pytest.mark.parametrize("name", ["ico", "torus", "disk"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_vcycle_parity_every_cycle(name, nrhs, request):
    c = request.getfixturevalue(name)
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=11)
    rng = np.random.default_rng(3)
    x_or = rng.uniform(-1, 1, b.shape)
    x_gpu = to_dev(x_or.copy())
    bd = to_dev(b)
    for k in range(5):
        x_or = oracle.vcycle(c.levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
        c.h.vcycle(bd, x_gpu)
        xg = x_gpu.cpu().numpy()
        assert rel(xg, x_or) <= CYCLE_TOL, k
        assert maxrel(xg, x_or) <= CYCLE_TOL, k


@pytest.mark.parametrize("nrhs", [1, 2, 4])
def test_solve_matches_oracle_and_direct(torus, nrhs):
    c = torus
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=5)
    ref = oracle.solve(c.levels, b, opt=oracle.Options(rtol=1e-10))
    c.h.set_options(rtol=1e-10)
    x, info = c.h.solve(to_dev(b))
    assert info["return"] == 0 and info["status"] == 0
    assert info["cycles"] == ref.cycles
    assert abs(info["rel_residual"] - ref.history[-1]) <= 1e-6 * ref.history[-1]
    assert rel(x.cpu().numpy(), ref.x) <= CYCLE_TOL
    assert maxrel(x.cpu().numpy(), ref.x) <= CYCLE_TOL
    xs = spla.splu(c.A.tocsc()).solve(b)
    assert rel(x.cpu().numpy(), xs) <= 1e-9


def test_mixed_precision_reaches_direct_solution(torus, disk):
    for c in (torus, disk):
        b = synth.uniform_rhs(c.n, nrhs=2, seed=8)
        c.h.set_options(rtol=1e-10, precision=smg.MIXED)
        x, info = c.h.solve(to_dev(b))
        c.h.set_options(rtol=1e-10, precision=smg.FP64)
        assert info["return"] == 0
        xs = spla.splu(c.A.tocsc()).solve(b)
        xg = x.cpu().numpy()
        assert rel(xg, xs) <= 1e-9
        assert oracle.rel_residual(c.A, xg, b) <= 1e-10
        ref = oracle.solve_mixed(c.levels, b, opt=oracle.Options(rtol=1e-10))
        assert abs(info["cycles"] - ref.cycles) <= 1


# Mixed precision step by step.  Refinement step k of the GPU and of the
# oracle computes x_k = x_{k-1} + B32 (b - A x_{k-1}) with a binary32 cycle B32
# on both sides; the two binary32 cycles differ only in the order of their
# sums, by a few units of u = 2^-24 times the correction they compute, and an
# earlier difference is contracted by the next cycle.  So every iterate is
# held, entry by entry, to MIXED_STEP_TOL times the size of that step's
# correction, plus a binary64 floor for the last steps, where the correction
# is down at the residual's binary64 rounding.  Measured on GB300: at most
# 3.4e-7 of the step (torus and disk, 1 and 3 RHS, steps 1-6); the bound is
# ~80 u.
MIXED_STEP_TOL = 5e-6


@pytest.mark.parametrize("name", ["torus", "disk"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_mixed_precision_every_refinement_step(name, nrhs, request):
    c = request.getfixturevalue(name)
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=12)
    bd = to_dev(b)
    ref = oracle.solve_mixed(c.levels, b, opt=oracle.Options(rtol=1e-30, max_cycles=6), keep_iterates=True)
    prev = np.zeros_like(b)
    for k in range(1, 7):
        c.h.set_options(rtol=1e-30, max_cycles=k, precision=smg.MIXED)
        x, info = c.h.solve(bd, check=False)
        assert info["cycles"] == k
        xg, xo = x.cpu().numpy(), ref.iterates[k - 1]
        step = np.abs(xo - prev).max()
        gap = np.abs(xg - xo).max()
        assert gap <= MIXED_STEP_TOL * step + 1e-13 * np.abs(xo).max(), (k, gap, step)
        prev = xo
    c.h.set_options(rtol=1e-10, max_cycles=100, precision=smg.FP64)


def test_user_matrix_and_t_updates(ico):
    c = ico
    b = synth.uniform_rhs(c.n, seed=2)
    c.h.update_matrix(to_dev(c.levels[0].A.data))
    x1, i1 = c.h.solve(to_dev(b))
    c.h.update_positions(c.Vd, c.t)
    x2, i2 = c.h.solve(to_dev(b))
    assert i1["cycles"] == i2["cycles"]
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) <= CYCLE_TOL
    c.h.update_t(10 * c.t)
    A10 = oracle.system_matrix(c.V, c.F, 10 * c.t)
    got = c.h.level_matrix(0)
    assert np.abs(got - A10.data).max() <= 1e-14 * np.abs(A10.data).max()
    c.h.update_t(c.t)


def test_warm_start_converged_runs_no_cycle(torus):
    c = torus
    b = synth.uniform_rhs(c.n, seed=4)
    xs = spla.splu(c.A.tocsc()).solve(b)
    c.h.set_options(rtol=1e-8)
    _, info = c.h.solve(to_dev(b), to_dev(xs.copy()))
    c.h.set_options(rtol=1e-10)
    assert info["cycles"] == 0 and info["return"] == 0


def test_single_level_is_direct_solve():
    V, F = synth.perturbed_icosphere(2, seed=1)
    c = Case(V, F, 1e-2, max_levels=1)
    assert c.plan.num_levels == 1
    b = synth.uniform_rhs(c.n, seed=3)
    x, info = c.h.solve(to_dev(b))
    assert info["cycles"] == 1
    assert oracle.rel_residual(c.A, x.cpu().numpy(), b) <= 1e-13


@pytest.mark.parametrize("nrhs", [1, 3])
def test_dense_factor_direct_solve_many_tiles(nrhs):
    """One level of 1,000 unknowns: the whole solve is the coarsest direct solve
    through the blocked factor (32 tiles of 32, as the bench's coarsest level)
    and its inverse, against a sparse LU solve."""
    V, F = synth.torus(40, 25, seed=6)
    c = Case(V, F, 1e-2, max_levels=1)
    assert c.plan.num_levels == 1 and c.n == 1000
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=9)
    x, info = c.h.solve(to_dev(b))
    assert info["cycles"] == 1
    xg = x.cpu().numpy()
    assert oracle.rel_residual(c.A, xg, b) <= 1e-13
    xs = spla.splu(c.A.tocsc()).solve(b)
    assert maxrel(xg, xs) <= 1e-12
    c.h.close()


def test_mass_matches_oracle(disk):
    m = disk.h.mass().cpu().numpy()
    ref = oracle.lumped_mass(disk.V, disk.F)[disk.u]
    assert np.abs(m - ref).max() <= 1e-15 * ref.max()
    x = synth.uniform_rhs(disk.n, nrhs=3, seed=1)
    y = disk.h.apply_mass(to_dev(x)).cpu().numpy()
    assert np.abs(y - ref[:, None] * x).max() <= 1e-15 * np.abs(y).max()


def test_error_statuses(ico):
    V, F = synth.perturbed_icosphere(2, seed=1)
    plan = smg.Plan(V, F, max_levels=2, min_coarse=0)
    h = smg.Hierarchy(plan)
    b = to_dev(np.ones(plan.level_info(0)[0]))
    with pytest.raises(smg.SmgError) as e:
        h.solve(b)
    assert e.value.status == 10                       # solve before any update
    h.update_positions(to_dev(V), 1e-2)
    with pytest.raises(smg.SmgError) as e:
        h.solve(to_dev(np.ones((b.shape[0], 5))))
    assert e.value.status == 1                        # nrhs out of range
    A = oracle.system_matrix(V, F, 1e-2)
    h.update_matrix(to_dev(-A.data))                  # negative definite: coarsest pivot fails
    with pytest.raises(smg.SmgError) as e:
        h.solve(b)
    assert e.value.status == 4
    h.update_matrix(to_dev(A.data))
    h.set_options(rtol=1e-30, max_cycles=2)
    _, info = h.solve(b, check=False)
    assert info["return"] == 5 and info["cycles"] == 2
    h.close()


@pytest.mark.parametrize("tail", ["0", "1", "99"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_cluster_tail_and_launch_paths_match_oracle(tail, nrhs, monkeypatch):
    """Level 0 onwards inside the cluster tail ("0"), levels >= 1 ("1"), and no
    tail ("99" clamps to H): every cycle iterate must match the oracle."""
    monkeypatch.setenv("SMG_TAIL_LEVEL", tail)
    V, F = synth.torus(64, 32, seed=3)
    c = Case(V, F, 1e-3, min_coarse=100)
    H, t64, t32, ctas = c.h.cycle_config()
    assert t64 == min(int(tail), H) or ctas == 0
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=12)
    x_or = np.zeros_like(b)
    x_gpu = to_dev(x_or.copy())
    bd = to_dev(b)
    for k in range(4):
        x_or = oracle.vcycle(c.levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
        c.h.vcycle(bd, x_gpu)
        xg = x_gpu.cpu().numpy()
        assert rel(xg, x_or) <= CYCLE_TOL, k
        assert maxrel(xg, x_or) <= CYCLE_TOL, k
    c.h.set_options(rtol=1e-10, precision=smg.MIXED)
    x, info = c.h.solve(bd)
    assert info["return"] == 0
    assert oracle.rel_residual(c.A, x.cpu().numpy(), b) <= 1e-10
    c.h.close()


def _staged_env(monkeypatch, on):
    """Every level one lane per row, its sweep staged by TMA (on) or not, no cluster tail."""
    monkeypatch.setenv("SMG_TAIL_LEVEL", "99")
    monkeypatch.setenv("SMG_LANES_PER_ROW", ",".join(["1"] * 12))
    flags = ",".join([("1" if on else "0")] * 12)
    monkeypatch.setenv("SMG_STAGED_GS", flags)
    monkeypatch.setenv("SMG_STAGED_GS_F32", flags)


@pytest.mark.parametrize("mesh", ["sphere", "disk", "torus"])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
def test_staged_sweep_matches_oracle_and_register_kernel(mesh, nrhs, monkeypatch):
    """The sweep with each warp's slice of entries brought into shared memory by
    bulk copies (gs_colour_bulk) on every level, coarse rows wider than the
    staged part taking the rest from global memory: each binary64 cycle iterate
    matches the oracle and is bitwise that of the register-prefetching kernel
    with one lane per row (the same FMA chain); the mixed-precision solve too."""
    if mesh == "sphere":
        V, F = synth.perturbed_geodesic_sphere(14, seed=7)  # valences 5 to 7
        mask = None
    elif mesh == "torus":
        V, F = synth.torus(120, 40, seed=2)  # 1,200-row colour classes: several blocks per launch
        mask = None
    else:
        V, F, mask = synth.disk(40, seed=5)
    _staged_env(monkeypatch, True)
    c = Case(V, F, 1e-2, mask=mask, min_coarse=100)
    H = c.h.cycle_config()[0]
    assert H >= 2 and all(c.h.level_staged(l) == (1, 1) for l in range(H))
    assert max(c.plan.level_info(l)[1] / c.plan.level_info(l)[0] for l in range(1, H)) > 9  # wide coarse rows
    _staged_env(monkeypatch, False)
    ref = smg.Hierarchy(c.plan)
    ref.update_positions(c.Vd, 1e-2)
    assert all(ref.level_staged(l) == (0, 0) and ref.level_config(l)[:2] == (1, 1) for l in range(H))
    b = synth.uniform_rhs(c.n, nrhs=nrhs, seed=21)
    bd = to_dev(b)
    x_or = np.zeros_like(b)
    xs, xr = to_dev(x_or.copy()), to_dev(x_or.copy())
    for k in range(3):
        x_or = oracle.vcycle(c.levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
        c.h.vcycle(bd, xs)
        ref.vcycle(bd, xr)
        xg = xs.cpu().numpy()
        assert maxrel(xg, x_or) <= CYCLE_TOL, k
        assert np.array_equal(xg, xr.cpu().numpy()), k
    for h in (c.h, ref):
        h.set_options(rtol=1e-10, precision=smg.MIXED)
    x1, i1 = c.h.solve(bd)
    x2, i2 = ref.solve(bd)
    assert i1["return"] == 0 and i1["cycles"] == i2["cycles"]
    assert torch.equal(x1, x2)
    assert oracle.rel_residual(c.A, x1.cpu().numpy(), b) <= 1e-10
    c.h.close()
    ref.close()


@pytest.fixture(scope="module")
def batch_cases():
    """Uneven meshes (spheres, tori, a Dirichlet disk) for the batched form."""
    meshes = [synth.perturbed_icosphere(3, seed=1), synth.torus(48, 20, seed=2),
              synth.perturbed_geodesic_sphere(14, seed=3), synth.torus(90, 30, seed=4)]
    Vd, Fd, bnd = synth.disk(40, seed=5)
    cases = []
    for V, F in meshes:
        cases.append(Case(V, F, 1e-2, max_coarse=300))
    cases.append(Case(Vd, Fd, 1e-2, mask=bnd, max_coarse=300))
    return cases


def _batch(cases, mode, **opts):
    """A batch of the cases' hierarchies with `opts` (the batch reads them at its
    first solve), positions uploaded and updated."""
    for c in cases:
        c.h.set_options(**opts)
    batch = smg.Batch([c.h for c in cases])
    batch.set_mode(mode)
    batch.update_positions(torch.from_numpy(np.concatenate([c.V for c in cases])).cuda(), 1e-2)
    return batch


def test_batch_matches_individual_solves_and_oracle(batch_cases):
    """a11, graph mode: uneven meshes with 3 right-hand sides each, updated and
    solved by one graph launch (a branch per mesh); every mesh must equal its
    own stand-alone solve bit for bit, and the oracle."""
    cases = batch_cases
    batch = smg.Batch([c.h for c in cases])
    Vcat = torch.from_numpy(np.concatenate([c.V for c in cases])).cuda()
    batch.update_positions(Vcat, 1e-2)
    bs = [synth.uniform_rhs(c.n, nrhs=3, seed=20 + i) for i, c in enumerate(cases)]
    for prec in (smg.FP64, smg.MIXED):
        batch.close()
        batch = _batch(cases, "graph", rtol=1e-10, precision=prec)
        x, infos = batch.solve(to_dev(np.concatenate(bs)))
        xs = x.cpu().numpy()
        u = batch.unknown_offsets
        for i, c in enumerate(cases):
            xi = xs[u[i]:u[i + 1]]
            single, info = c.h.solve(to_dev(bs[i]))
            assert infos[i]["cycles"] == info["cycles"]
            assert np.array_equal(xi, single.cpu().numpy())      # same kernels, same bits
            assert oracle.rel_residual(c.A, xi, bs[i]) <= 1e-10
            if prec == smg.FP64:
                ref = oracle.solve(c.levels, bs[i], opt=oracle.Options(rtol=1e-10))
                assert infos[i]["cycles"] == ref.cycles
                assert rel(xi, ref.x) <= CYCLE_TOL
    for c in cases:
        c.h.set_options(rtol=1e-10, precision=smg.FP64)
    batch.close()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_batch_persistent_every_cycle(batch_cases, nrhs):
    """a11, persistent mode: one kernel launch runs every cycle of every mesh
    from its own work queue; after k cycles (k = 1, 2, 4) every mesh's iterate
    equals the oracle's cycle k entry by entry (1e-12), and solved to 1e-10
    every mesh takes the oracle's cycle count."""
    cases = batch_cases
    bs = [synth.uniform_rhs(c.n, nrhs=nrhs, seed=40 + i) for i, c in enumerate(cases)]
    bcat = to_dev(np.concatenate(bs))
    refs = [oracle.solve(c.levels, b, opt=oracle.Options(rtol=1e-30, max_cycles=4), keep_iterates=True)
            for c, b in zip(cases, bs)]
    for k in (1, 2, 4):
        batch = _batch(cases, "persistent", rtol=1e-30, max_cycles=k, precision=smg.FP64)
        x, infos = batch.solve(bcat, check=False)
        xs = x.cpu().numpy()
        u = batch.unknown_offsets
        for i, c in enumerate(cases):
            assert infos[i]["cycles"] == k
            xo = refs[i].iterates[k - 1]
            assert maxrel(xs[u[i]:u[i + 1]], xo) <= CYCLE_TOL, (i, k)
        batch.close()
    batch = _batch(cases, "persistent", rtol=1e-10, max_cycles=100, precision=smg.FP64)
    x, infos = batch.solve(bcat)
    xs = x.cpu().numpy()
    u = batch.unknown_offsets
    for i, c in enumerate(cases):
        ref = oracle.solve(c.levels, bs[i], opt=oracle.Options(rtol=1e-10))
        assert infos[i]["cycles"] == ref.cycles
        assert maxrel(xs[u[i]:u[i + 1]], ref.x) <= CYCLE_TOL
    batch.close()
    for c in cases:
        c.h.set_options(rtol=1e-10, max_cycles=100, precision=smg.FP64)


def test_batch_persistent_mixed_every_step(batch_cases):
    """a11 with form 1: binary32 cycles inside binary64 refinement, every mesh
    in the persistent launch, each refinement step against the oracle's
    binary32 refinement (MIXED_STEP_TOL of the step's correction), and
    solved to 1e-10 against the graph mode's cycle counts (+-1) and a direct
    solve (1e-9)."""
    cases = batch_cases
    bs = [synth.uniform_rhs(c.n, nrhs=3, seed=60 + i) for i, c in enumerate(cases)]
    bcat = to_dev(np.concatenate(bs))
    refs = [oracle.solve_mixed(c.levels, b, opt=oracle.Options(rtol=1e-30, max_cycles=3), keep_iterates=True)
            for c, b in zip(cases, bs)]
    for k in (1, 2, 3):
        batch = _batch(cases, "persistent", rtol=1e-30, max_cycles=k, precision=smg.MIXED)
        x, infos = batch.solve(bcat, check=False)
        xs = x.cpu().numpy()
        u = batch.unknown_offsets
        for i, c in enumerate(cases):
            assert infos[i]["cycles"] == k
            xo = refs[i].iterates[k - 1]
            prev = refs[i].iterates[k - 2] if k > 1 else np.zeros_like(xo)
            gap = np.abs(xs[u[i]:u[i + 1]] - xo).max()
            assert gap <= MIXED_STEP_TOL * np.abs(xo - prev).max() + 1e-13 * np.abs(xo).max(), (i, k)
        batch.close()
    out = {}
    for mode in ("persistent", "graph"):
        batch = _batch(cases, mode, rtol=1e-10, max_cycles=100, precision=smg.MIXED)
        x, infos = batch.solve(bcat)
        out[mode] = (x.cpu().numpy(), [d["cycles"] for d in infos], batch.unknown_offsets)
        batch.close()
    xs, cyc, u = out["persistent"]
    for i, c in enumerate(cases):
        assert abs(cyc[i] - out["graph"][1][i]) <= 1
        xd = spla.splu(c.A.tocsc()).solve(bs[i])
        assert rel(xs[u[i]:u[i + 1]], xd) <= 1e-9
    for c in cases:
        c.h.set_options(rtol=1e-10, max_cycles=100, precision=smg.FP64)


def test_batch_persistent_watchdog_reports_timeout(batch_cases):
    """Failure detection without a GPU fault: with the persistent launch's idle
    limit at zero every warp gives up at its first moment without work, the
    launch ends, and the solve reports SMG_ERR_TIMEOUT; with the limit back at
    two seconds the same batch solves correctly in the same context."""
    cases = batch_cases
    bs = [synth.uniform_rhs(c.n, nrhs=1, seed=80 + i) for i, c in enumerate(cases)]
    bcat = to_dev(np.concatenate(bs))
    batch = _batch(cases, "persistent", rtol=1e-10, max_cycles=100, precision=smg.FP64)
    batch.set_wait_limit(0.0)
    st = smg.lib.smg_batch_solve(batch._h, smg._dev_ptr(bcat), smg._dev_ptr(torch.zeros_like(bcat)), 1, None,
                                 smg._stream_ptr(None))
    assert st == 7 and b"idle" in smg.lib.smg_last_error()
    batch.set_wait_limit(2.0)
    x, infos = batch.solve(bcat)
    xs = x.cpu().numpy()
    u = batch.unknown_offsets
    for i, c in enumerate(cases):
        ref = oracle.solve(c.levels, bs[i], opt=oracle.Options(rtol=1e-10))
        assert infos[i]["cycles"] == ref.cycles
        assert maxrel(xs[u[i]:u[i + 1]], ref.x) <= CYCLE_TOL
    batch.close()


def test_fast_t_updates_match_oracle_galerkin_chain():
    """App. "Fast Data Smoothing": update_t forms every level from the kept
    P^T M P and P^T L P; each level must equal the oracle's Galerkin chain of
    A = M + t L for the new t, across repeated t changes and new positions."""
    V, F = synth.perturbed_icosphere(4, seed=6)
    c = Case(V, F, 1e-3, min_coarse=100)
    Ps = [c.plan.prolongation_csr(l) for l in range(1, c.plan.num_levels)]
    for Vk, t in ((V, 3e-3), (V, 0.1), (V, 1e-4), (synth.perturbed_icosphere(4, seed=7)[0], 0.02)):
        if Vk is not V:
            c.h.update_positions(to_dev(Vk), 1e-3)
        c.h.update_t(t)
        levels = oracle.build_levels(oracle.system_matrix(Vk, F, t), Ps)
        for l in range(c.plan.num_levels):
            got = c.h.level_matrix(l)
            ref = levels[l].A.data
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (t, l)
        b = synth.uniform_rhs(c.n, seed=9)
        c.h.set_options(rtol=1e-10)
        x, info = c.h.solve(to_dev(b))
        ref = oracle.solve(levels, b, opt=oracle.Options(rtol=1e-10))
        assert info["cycles"] == ref.cycles
        assert rel(x.cpu().numpy(), ref.x) <= CYCLE_TOL
    c.h.close()


@pytest.mark.parametrize("smoother,mu,ratio", [("jacobi", 2, 0.25), ("jacobi", 1, 0.5), ("gs", 1, 0.5),
                                               ("gs", 3, 0.25)])
def test_ablation_settings_match_oracle(smoother, mu, ratio):
    """App. "Ablation Study": relaxation method (multicolour Gauss-Seidel or
    damped Jacobi), mu_pre = mu_post in {1, 2, 3}, coarsening ratio 0.25 or 0.5;
    every cycle iterate against the oracle with the same settings."""
    V, F = synth.torus(96, 32, seed=5)
    sm = smg.JACOBI if smoother == "jacobi" else smg.GS
    c = Case(V, F, 1e-3, min_coarse=100, ratio=ratio, mu_pre=mu, mu_post=mu, smoother=sm)
    opt = oracle.Options(mu_pre=mu, mu_post=mu, smoother=smoother)
    b = synth.uniform_rhs(c.n, nrhs=2, seed=13)
    x_or = np.zeros_like(b)
    x_gpu = to_dev(x_or.copy())
    bd = to_dev(b)
    for k in range(4):
        x_or = oracle.vcycle(c.levels, 0, np.ascontiguousarray(x_or), b, opt)
        c.h.vcycle(bd, x_gpu)
        assert rel(x_gpu.cpu().numpy(), x_or) <= CYCLE_TOL, k
    c.h.set_options(rtol=1e-10, max_cycles=300, mu_pre=mu, mu_post=mu, smoother=sm, precision=smg.MIXED)
    x, info = c.h.solve(bd)
    assert info["return"] == 0
    assert oracle.rel_residual(c.A, x.cpu().numpy(), b) <= 1e-10
    c.h.close()


@pytest.mark.parametrize("dirichlet", [False, True])
def test_bilaplacian_two_ring_system_matches_oracle(dirichlet):
    """Sec. 6: data smoothing with the Bilaplacian energy, A = M + t L M^{-1} L on
    the 2-ring pattern (pattern_rings = 2), supplied through smg_update_matrix:
    every cycle against the oracle, then binary64, mixed and PCG solves."""
    if dirichlet:
        V, F, known = synth.disk(40, seed=8)
    else:
        V, F = synth.torus(64, 24, seed=6)
        known = np.zeros(V.shape[0], dtype=bool)
    t = 0.5 * synth.mean_edge_length(V, F) ** 2
    plan = smg.Plan(V, F, dirichlet=known if dirichlet else None, pattern_rings=2, min_coarse=100)
    h = smg.Hierarchy(plan)
    A = oracle.bilaplacian_system(V, F, t)
    Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
    A, Ps, _, _ = oracle.dirichlet_reduce(A, Ps, known)
    levels = oracle.build_levels(A, Ps)
    h.update_matrix(to_dev(A.data))
    for l in range(1, plan.num_levels):
        ref = levels[l].A.data
        assert np.abs(h.level_matrix(l) - ref).max() <= 1e-13 * np.abs(ref).max(), l
    b = synth.uniform_rhs(A.shape[0], nrhs=2, seed=17)
    bd = to_dev(b)
    x_or = np.zeros_like(b)
    x_gpu = to_dev(x_or.copy())
    for k in range(3):
        x_or = oracle.vcycle(levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
        h.vcycle(bd, x_gpu)
        assert rel(x_gpu.cpu().numpy(), x_or) <= CYCLE_TOL, k
    xs = spla.splu(A.tocsc()).solve(b)
    for kw in (dict(), dict(precision=smg.MIXED), dict(solver=smg.PCG)):
        h.set_options(rtol=1e-10, max_cycles=300, **kw)
        x, info = h.solve(bd)
        assert info["return"] == 0, kw
        assert rel(x.cpu().numpy(), xs) <= 1e-8, kw
    h.close()


@pytest.mark.parametrize("dirichlet", [False, True])
def test_block3_systems_match_oracle(dirichlet):
    """block_size = 3 (3|V| systems, Sec. 6): update_positions assembles
    (M + t L) (x) I_3; a system with cross-component coupling,
    (M + t L) (x) I_3 + s L (x) J (J the symmetric 3 x 3 tridiagonal ones, s < t /
    sqrt 2 so the sum stays positive definite), goes through update_matrix.
    Galerkin levels, every cycle (the sweep in 3 x 3 blocks, a vertex class per
    launch) and the solves against the oracle."""
    if dirichlet:
        V, F, known = synth.disk(32, seed=9)
    else:
        V, F = synth.torus(48, 20, seed=7)
        known = np.zeros(V.shape[0], dtype=bool)
    t = 1e-3
    plan = smg.Plan(V, F, dirichlet=known if dirichlet else None, block_size=3, min_coarse=100)
    h = smg.Hierarchy(plan)
    n = V.shape[0]
    S3 = oracle.block_pattern(oracle.mesh_pattern(n, F), 3)
    Ps = [oracle.expand_blocks(plan.prolongation_csr(l), 3) for l in range(1, plan.num_levels)]
    L = oracle.cotan_laplacian(V, F)
    J = sp.csr_matrix(np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 0.0]]))
    systems = [("assembled", oracle.expand_blocks(oracle.system_matrix(V, F, t), 3)),
               ("coupled", oracle.expand_blocks(oracle.system_matrix(V, F, t), 3) + 0.3 * t * sp.kron(L, J))]
    for name, A in systems:
        A = oracle.on_pattern(S3, A.tocsr())
        Ar, Pr, _, _ = oracle.dirichlet_reduce(A, Ps, np.repeat(known, 3))
        levels = oracle.build_levels(Ar, Pr, block=3)
        if name == "assembled":
            h.update_positions(to_dev(V), t)
        else:
            h.update_matrix(to_dev(Ar.data))
        for l in range(plan.num_levels):
            ref = levels[l].A.data
            assert np.abs(h.level_matrix(l) - ref).max() <= 1e-13 * np.abs(ref).max(), (name, l)
        b = synth.uniform_rhs(Ar.shape[0], nrhs=1, seed=19)
        bd = to_dev(b)
        x_or = np.zeros_like(b)
        x_gpu = to_dev(x_or.copy())
        for k in range(3):
            x_or = oracle.vcycle(levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
            h.vcycle(bd, x_gpu)
            assert rel(x_gpu.cpu().numpy(), x_or) <= CYCLE_TOL, (name, k)
            assert maxrel(x_gpu.cpu().numpy(), x_or) <= CYCLE_TOL, (name, k)
        xs = spla.splu(Ar.tocsc()).solve(b)
        for kw in (dict(), dict(precision=smg.MIXED), dict(solver=smg.PCG)):
            h.set_options(rtol=1e-10, max_cycles=300, **kw)
            x, info = h.solve(bd)
            assert info["return"] == 0, (name, kw)
            assert rel(x.cpu().numpy(), xs) <= 1e-8, (name, kw)
    h.close()
