"""The allocation-free residual-norm entry point, for callers that cannot
allocate device memory when they need it (real-time frame loops where an
allocation may synchronise the device; host applications that own every
device allocation of a plug-in).  Called through the C ABI on device arrays
the caller owns, twice in a row, and checked against

  * ||b_q - A x_q||^2 and ||b_q||^2 of every column, computed on the host in
    binary64 from the same CSR arrays (the sums differ only in order: 1e-12
    relative), and
  * the solver's own initial relative residual (smg_solve with no cycles,
    the existing entry point that computes the same quantity),

with identical bits on the second call (every scratch slot is rewritten and
the reduction order is fixed).

Kept in a file of its own that sorts last, so a run that stops at the first
failure has run every other test first."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2104_13755_gb300 as smg  # noqa: E402

TOL = 1e-12


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("nrhs", [1, 3, 4])
def test_noalloc_residual_norms_match_host_and_solver(nrhs):
    V, F = synth.torus(60, 24, seed=5)
    plan = smg.Plan(V, F, min_coarse=100)
    h = smg.Hierarchy(plan, max_cycles=0)
    h.update_positions(torch.from_numpy(V).cuda(), 1e-3)
    n = plan.level_info(0)[0]
    rowptr, col = plan.pattern(0)
    vals = h.level_matrix(0)
    b = synth.uniform_rhs(n, nrhs=nrhs, seed=3).reshape(n, nrhs)
    x0 = synth.uniform_rhs(n, nrhs=nrhs, seed=4).reshape(n, nrhs)

    A = sp.csr_matrix((vals, col, rowptr), shape=(n, n))
    r = b - A @ x0
    host = np.concatenate([np.sum(r * r, axis=0), np.sum(b * b, axis=0)])

    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    _, info = h.solve(bd, torch.from_numpy(np.ascontiguousarray(x0)).cuda(), check=False)
    solver_rel0 = info["rel_residual0"]
    assert info["cycles"] == 0 and solver_rel0 > 0

    rp = torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.int64)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).cuda()
    va = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
    out = torch.empty(2 * nrhs, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    results = []
    for _ in range(2):
        out.fill_(-1.0)
        st = smg.lib.smg_residual_norms_noalloc(n, _p(rp), _p(ci), _p(va), _p(xd), _p(bd), nrhs, _p(out), stream)
        assert st == 0, smg.lib.smg_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.abs(o - host) <= TOL * host), (o, host)
        rel = float(np.max(np.sqrt(o[:nrhs] / o[nrhs:])))
        assert abs(rel - solver_rel0) <= TOL * solver_rel0
        results.append(o)
    assert np.array_equal(results[0], results[1])  # fixed reduction order, scratch fully rewritten

    st = smg.lib.smg_residual_norms_noalloc(n, _p(rp), _p(ci), _p(va), _p(xd), _p(bd), 5, _p(out), stream)
    assert st == 1 and b"nrhs" in smg.lib.smg_last_error()
    h.close()
