"""Differentiable solve (form 3) on the GPU, through the C ABI and the
torch.autograd.Function binding.

Kernels against the oracle: the per-face derivative kernels compute closed-form
d(area)/dp and d(cot)/dp; the oracle takes complex-step derivatives of the same
per-face energies.  Both are exact up to rounding, so they agree to 1e-11 of the
largest entry (a face sum of ~6 terms of comparable size per vertex).

The loss is the impulse-response energy on a Dirichlet disk: b = M e_s for a
seeded interior unknown s, A x = b, l = x^T M x, t = (mean edge length)^2 held
fixed.  Its gradient is checked against central finite differences (eps 1e-6 on
32 seeded unit directions in R^{3n}) and against the oracle's gradient (exact
LU solves).  The FD tolerance |fd - g.d| <= 1e-6 |g.d| + 1e-7 l covers rounding
in the two loss evaluations divided by 2 eps; the oracle's own FD at 160,000
vertices lands within 2.5e-8 of both."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2104_13755_gb300 as smg  # noqa: E402

EPS = 1e-6
KERNEL_TOL = 1e-11


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mesh(name):
    if name == "disk":
        V, F, bnd = synth.disk(60, seed=4)
        return V, F, bnd
    V, F = synth.torus(60, 24, seed=2)
    return V, F, None


@pytest.mark.parametrize("name", ["disk", "torus"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_derivative_kernels_match_oracle(name, nrhs):
    V, F, bnd = _mesh(name)
    plan = smg.Plan(V, F, dirichlet=bnd, min_coarse=100)
    h = smg.Hierarchy(plan)
    u = np.flatnonzero(~bnd) if bnd is not None else np.arange(V.shape[0])
    t = 0.7 * synth.mean_edge_length(V, F) ** 2
    rng = np.random.default_rng(nrhs)
    lam = rng.standard_normal((u.size, nrhs)).squeeze()
    x = rng.standard_normal((u.size, nrhs)).squeeze()
    Vd = to_dev(V)
    gV, dt = h.operator_grad(Vd, t, to_dev(lam), to_dev(x))
    G, dref = oracle.operator_grad(V, F, t, lam, x, u)
    assert np.abs(gV.cpu().numpy() + G).max() <= KERNEL_TOL * np.abs(G).max()
    assert abs(dt.item() + dref) <= KERNEL_TOL * abs(dref)
    m = h.lumped_mass(Vd).cpu().numpy()
    mref = oracle.lumped_mass(V, F)[u]
    assert np.abs(m - mref).max() <= 1e-15 * mref.max()
    w = rng.standard_normal(u.size)
    gm = h.mass_grad(Vd, to_dev(w)).cpu().numpy()
    Gm = oracle.mass_grad(V, F, w, u)
    assert np.abs(gm - Gm).max() <= KERNEL_TOL * np.abs(Gm).max()
    h.close()


class HeatLoss:
    """l(V) = x^T M x, A(V, t) x = M e_s, through the differentiable binding."""

    def __init__(self, N, seed, **opts):
        self.V, self.F, self.bnd = synth.disk(N, seed=seed)
        self.u = np.flatnonzero(~self.bnd)
        self.t = synth.mean_edge_length(self.V, self.F) ** 2
        self.s = int(np.random.default_rng(seed + 100).integers(self.u.size))
        self.plan = smg.Plan(self.V, self.F, dirichlet=self.bnd, **opts)
        self.h = smg.Hierarchy(self.plan, **opts)
        self.e_s = torch.zeros(self.u.size, dtype=torch.float64, device="cuda")
        self.e_s[self.s] = 1.0

    def loss(self, Vt, t):
        m = smg.differentiable_mass(self.h, Vt)
        b = m * self.e_s
        b.retain_grad()
        x = smg.differentiable_solve(self.h, Vt, t, b)
        return (m * x * x).sum(), b

    def loss_value(self, V, t):
        """Forward only, a fixed 30 cycles (a smooth function of V, at the
        rounding floor for this operator) so +eps and -eps see the same map."""
        Vd = to_dev(V)
        self.h.update_positions(Vd, t)
        m = self.h.lumped_mass(Vd)
        self.h.set_options(rtol=1e-30, max_cycles=30)
        x, _ = self.h.solve(m * self.e_s, check=False)
        self.h.set_options(rtol=1e-12, max_cycles=100)
        return float((m * x * x).sum())

    def grad(self):
        self.h.set_options(rtol=1e-12, max_cycles=100)
        Vt = to_dev(self.V).requires_grad_(True)
        tt = torch.tensor(self.t, dtype=torch.float64, device="cuda", requires_grad=True)
        l, b = self.loss(Vt, tt)
        l.backward()
        return l.item(), Vt.grad.cpu().numpy(), tt.grad.item(), b.grad.cpu().numpy()


def _check_fd_and_oracle(c, ndir):
    l, gV, gt, gb = c.grad()
    ref = oracle.heat_loss_grad(c.V, c.F, c.t, c.bnd, c.s)
    assert abs(l - ref.loss) <= 1e-10 * ref.loss
    assert np.linalg.norm(gV - ref.dV) <= 1e-8 * np.linalg.norm(ref.dV)
    assert abs(gt - ref.dt) <= 1e-8 * abs(ref.dt)
    assert np.linalg.norm(gb - ref.db) <= 1e-8 * np.linalg.norm(ref.db)
    rng = np.random.default_rng(2024)
    for k in range(ndir):
        d = rng.standard_normal(c.V.shape)
        d /= np.linalg.norm(d)
        fd = (c.loss_value(c.V + EPS * d, c.t) - c.loss_value(c.V - EPS * d, c.t)) / (2 * EPS)
        an = float(np.sum(gV * d))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7 * l, (k, fd, an)
    et = EPS * c.t
    fd = (c.loss_value(c.V, c.t + et) - c.loss_value(c.V, c.t - et)) / (2 * et)
    assert abs(fd - gt) <= 1e-6 * abs(gt) + 1e-7 * l / c.t


def test_heat_loss_gradient_small_disk():
    c = HeatLoss(60, seed=4, min_coarse=100)
    _check_fd_and_oracle(c, 32)
    c.h.close()


def test_heat_loss_gradient_disk_160k():
    """The 400 x 400 disk (160,000 vertices, 1,596 Dirichlet boundary vertices),
    the paper's coarsening down to at least 500 coarsest unknowns."""
    c = HeatLoss(400, seed=4)
    assert c.u.size == 160000 - 1596
    _check_fd_and_oracle(c, 32)
    c.h.close()


def test_total_derivative_through_mean_edge_length():
    """t = hbar(V)^2 made a function of V in torch: the t-gradient of the solve
    flows back into V; checked by FD with t recomputed from the moved V."""
    c = HeatLoss(40, seed=9, min_coarse=100)
    E = torch.from_numpy(np.unique(np.sort(np.concatenate(
        [c.F[:, [0, 1]], c.F[:, [1, 2]], c.F[:, [2, 0]]]), axis=1), axis=0)).cuda()

    def t_of(Vt):
        return ((Vt[E[:, 0]] - Vt[E[:, 1]]).norm(dim=1).mean()) ** 2

    Vt = to_dev(c.V).requires_grad_(True)
    l, _ = c.loss(Vt, t_of(Vt))
    l.backward()
    g = Vt.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    for _ in range(8):
        d = rng.standard_normal(c.V.shape)
        d /= np.linalg.norm(d)
        vals = []
        for sgn in (1.0, -1.0):
            Vm = c.V + sgn * EPS * d
            vals.append(c.loss_value(Vm, float(t_of(to_dev(Vm)))))
        fd = (vals[0] - vals[1]) / (2 * EPS)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7 * l.item()
    c.h.close()
