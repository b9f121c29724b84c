import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def torus_refinement_P(nu, nv):
    """Linear interpolation from an nu x nv torus grid to its regular refinement
    (2nu x 2nv, same diagonal direction as synth.torus): even-even fine vertices
    copy a coarse vertex, the others sit at coarse edge midpoints (1/2, 1/2).
    A textbook geometric-multigrid prolongation used to pin the oracle."""
    import scipy.sparse as sp
    rows, cols, vals = [], [], []
    fnv = 2 * nv
    for a in range(2 * nu):
        for b in range(2 * nv):
            i = a * fnv + b
            A0, B0 = a // 2, b // 2
            A1, B1 = (A0 + (a % 2)) % nu, (B0 + (b % 2)) % nv
            c0 = A0 * nv + B0
            c1 = A1 * nv + B1
            if c0 == c1:
                rows.append(i); cols.append(c0); vals.append(1.0)
            else:
                rows += [i, i]; cols += [c0, c1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(4 * nu * nv, nu * nv))


@pytest.fixture(scope="session")
def torus_pin_hierarchy():
    """Fine torus 32 x 16 with two regular-refinement prolongations (3 levels)."""
    import synth
    V, F = synth.torus(32, 16, noise=0.0)
    return V, F, [torus_refinement_P(16, 8), torus_refinement_P(8, 4)]
