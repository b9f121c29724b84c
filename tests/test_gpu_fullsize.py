"""Full-size cases on the GPU, through the C ABI.

* The 1,000,000-vertex torus that bench.py times, built the same way (paper
  default hierarchy, the autotuned lanes per row and cluster tail that
  bench.py gets): every entry of the first two binary64 cycles against the
  oracle (1e-12 relative), the solve to 1e-9 against the oracle's cycle count,
  and the mixed-precision solve by its binary64 residual.
* The 2,621,442-vertex perturbed icosphere (icosphere split 9 times), t = 1e-4,
  two right-hand sides: mixed-precision refinement to 1e-10 checked by the
  binary64 residual computed on the host, and against the binary64 solve.
* The 655,362-vertex icosphere deformed frame by frame: re-assembly, Galerkin
  update and a warm-started solve to 1e-8 per frame, in both precisions, each
  frame's solution checked by its binary64 residual on the host.
The oracle builds the reference hierarchy from the same prolongations (its
levels take ~10 s at 1M); at 2.6M and 655k the checks are the residual
properties that hold at any size."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2104_13755_gb300 as smg  # noqa: E402


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def bench_case():
    w = bench.WORKLOAD
    V, F, b = bench.make_workload(w)
    plan = smg.Plan(V, F)
    h = smg.Hierarchy(plan, rtol=w["rtol"], max_cycles=200)
    h.update_positions(to_dev(V), w["t"])
    A = oracle.system_matrix(V, F, w["t"])
    Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
    levels = oracle.build_levels(A, Ps)
    yield dict(V=V, F=F, b=b, plan=plan, h=h, A=A, levels=levels, w=w)
    h.close()


def test_bench_workload_cycles_and_solve_match_oracle(bench_case):
    c = bench_case
    h, b, levels = c["h"], c["b"], c["levels"]
    assert c["plan"].num_levels == 6 and c["plan"].level_info(0)[0] == 1000000
    x_or = np.zeros_like(b)
    x_gpu = to_dev(x_or)
    bd = to_dev(b)
    for k in range(2):
        x_or = oracle.vcycle(levels, 0, np.ascontiguousarray(x_or), b, oracle.Options())
        h.vcycle(bd, x_gpu)
        assert rel(x_gpu.cpu().numpy(), x_or) <= 1e-12, k
    ref = oracle.solve(levels, b, opt=oracle.Options(rtol=c["w"]["rtol"]))
    h.set_options(rtol=c["w"]["rtol"], max_cycles=200, precision=smg.FP64)
    x, info = h.solve(bd)
    assert info["cycles"] == ref.cycles
    xg = x.cpu().numpy()
    assert rel(xg, ref.x) <= 1e-10
    assert oracle.rel_residual(c["A"], xg, b) <= c["w"]["rtol"]


def test_bench_workload_mixed_precision(bench_case):
    c = bench_case
    h = c["h"]
    h.set_options(rtol=c["w"]["rtol"], max_cycles=200, precision=smg.MIXED)
    x, info = h.solve(to_dev(c["b"]))
    h.set_options(precision=smg.FP64)
    assert info["return"] == 0
    assert oracle.rel_residual(c["A"], x.cpu().numpy(), c["b"]) <= c["w"]["rtol"]


def test_icosphere9_mixed_against_fp64_and_residual():
    V, F = synth.perturbed_icosphere(9, seed=3)
    assert V.shape[0] == 2621442
    t = 1e-4
    plan = smg.Plan(V, F)
    h = smg.Hierarchy(plan, rtol=1e-10, max_cycles=200)
    h.update_positions(to_dev(V), t)
    b = synth.uniform_rhs(V.shape[0], nrhs=2, seed=7)
    bd = to_dev(b)
    h.set_options(rtol=1e-10, precision=smg.MIXED)
    xm, im = h.solve(bd)
    h.set_options(rtol=1e-10, precision=smg.FP64)
    xd, idd = h.solve(bd)
    A = oracle.system_matrix(V, F, t)
    xm, xd = xm.cpu().numpy(), xd.cpu().numpy()
    assert oracle.rel_residual(A, xm, b) <= 1e-10
    assert oracle.rel_residual(A, xd, b) <= 1e-10
    assert im["cycles"] <= idd["cycles"] + 2
    # both within rel. residual 1e-10 of the same system; kappa(A) <= ~1e3 here
    # (t / h^2 ~ 20 times the Laplacian's ~12 / h^2 spectral bound), so the two
    # solutions agree to ~2 kappa 1e-10
    assert rel(xm, xd) <= 2e-7
    h.close()


def test_icosphere8_per_frame_warm_started_resolves():
    V0, F = synth.perturbed_icosphere(8, seed=5)
    assert V0.shape[0] == 655362
    plan = smg.Plan(V0, F)
    h = smg.Hierarchy(plan, rtol=1e-8, max_cycles=200)
    t = 1e-3
    b = synth.uniform_rhs(V0.shape[0], nrhs=1, seed=9)
    bd = to_dev(b)
    for prec in (smg.FP64, smg.MIXED):
        x = torch.zeros_like(bd)
        cycles = []
        for f in range(4):
            Vf = synth.sinusoidal_displacement(V0, f, seed=11)
            h.update_positions(to_dev(Vf), t)
            h.set_options(rtol=1e-8, precision=prec)
            x, info = h.solve(bd, x)
            cycles.append(info["cycles"])
            A = oracle.system_matrix(Vf, F, t)
            assert oracle.rel_residual(A, x.cpu().numpy(), b) <= 1e-8, (prec, f)
        assert max(cycles[1:]) <= cycles[0] + 1  # warm starts need no more than the cold one
    h.close()
