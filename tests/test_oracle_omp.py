"""The multicolour OpenMP cycle used as the all-cores CPU baseline against the
serial oracle: a Gauss-Seidel sweep updates every row with the same sum in the
same CSR order, so sweeps agree bit for bit; the transfers sum in another
order, so whole cycles agree to rounding (1e-13 relative)."""
import numpy as np

import oracle
import oracle.omp as omp
import synth


def test_parallel_sweep_is_the_serial_sweep():
    V, F = synth.perturbed_icosphere(3, seed=3)
    A = oracle.system_matrix(V, F, 1e-2)
    levels = oracle.build_levels(A, [])
    col = oracle.greedy_colouring(A)
    lv = oracle.Level(A=A, P=A, colour=col, fwd=oracle.colour_order(col), rev=oracle.colour_order(col, True))
    ol = omp.OmpLevels([lv, levels[-1]])
    rng = np.random.default_rng(1)
    b = rng.standard_normal((A.shape[0], 2))
    x0 = rng.standard_normal((A.shape[0], 2))
    for reverse in (False, True):
        xs = x0.copy()
        oracle.gs_sweep(A, xs, b, lv.rev if reverse else lv.fwd)
        xp = x0.copy()
        omp._relax(ol.levels[0], xp, b, 1, reverse, 2)
        assert np.array_equal(xs, xp)


def test_parallel_cycle_matches_oracle(torus_pin_hierarchy):
    V, F, Ps = torus_pin_hierarchy
    A = oracle.system_matrix(V, F, 1e-3)
    levels = oracle.build_levels(A, Ps)
    ol = omp.OmpLevels(levels)
    assert omp.threads() >= 1
    for nrhs in (1, 3):
        b = synth.uniform_rhs(A.shape[0], nrhs=nrhs, seed=4)
        xo = np.zeros_like(b)
        xp = np.zeros_like(b)
        for _ in range(4):
            xo = oracle.vcycle(levels, 0, np.ascontiguousarray(xo), b, oracle.Options())
            xp = omp.vcycle(ol, 0, xp, b, oracle.Options())
            assert np.abs(xp - xo).max() <= 1e-13 * np.abs(xo).max()
