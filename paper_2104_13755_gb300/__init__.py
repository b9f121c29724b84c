"""GB300 surface multigrid: Python binding of libsmg.so (C ABI in include/smg.h).

Argument marshalling only.  Every step of setup, update and solve runs in the
native library: the host setup in C++ and the per-frame and per-solve work in
sm_103a CUDA kernels.  There is no Python or CPU fallback: if the library
cannot be built or loaded, importing this package raises.

Method: Liu, Zhang, Ben-Chen, Jacobson, "Surface Multigrid via Intrinsic
Prolongation" (ACM TOG 2021): Alg. 1 (precompute P from geometry, build A,
run V-cycles), Alg. 2 (Galerkin V-cycle), Alg. 3 (colouring).
"""
import ctypes
import os

import numpy as np

from . import _build

__all__ = ["Plan", "Hierarchy", "Batch", "differentiable_solve", "differentiable_mass", "SmgError", "Options", "Info", "FP64", "MIXED", "VCYCLE", "PCG", "GS", "JACOBI", "lib", "library_path"]

FP64, MIXED = 0, 1
VCYCLE, PCG = 0, 1  # solver: Alg. 1 V-cycle iteration, or CG preconditioned by one V-cycle
GS, JACOBI = 0, 1  # smoother: multicolour Gauss-Seidel, or damped Jacobi

STATUS = {0: "ok", 1: "invalid argument", 2: "non-manifold mesh", 3: "decimation failed",
          4: "not SPD", 5: "not converged", 6: "diverged", 7: "timeout", 8: "CUDA error",
          9: "out of memory", 10: "call out of order", 11: "plan file error"}


class Options(ctypes.Structure):
    _fields_ = [("mu_pre", ctypes.c_int32), ("mu_post", ctypes.c_int32), ("ratio", ctypes.c_double),
                ("min_coarse", ctypes.c_int64), ("max_coarse", ctypes.c_int64),
                ("max_levels", ctypes.c_int32), ("max_cycles", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("post_reverse", ctypes.c_int32), ("autotune", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("jacobi_omega", ctypes.c_double),
                ("pattern_rings", ctypes.c_int32), ("block_size", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_residual0", ctypes.c_double), ("rel_residual", ctypes.c_double),
                ("rho", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SmgError(RuntimeError):
    def __init__(self, status, where):
        msg = lib.smg_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))
        self.status = status


def _load():
    path = _build.build()
    L = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "smg_default_options": (None, [P]),
        "smg_status_string": (ctypes.c_char_p, [I32]),
        "smg_last_error": (ctypes.c_char_p, []),
        "smg_plan_build": (I32, [P, I64, P, I64, P, P, P]),
        "smg_plan_destroy": (None, [P]),
        "smg_plan_num_levels": (I32, [P]),
        "smg_plan_level_info": (I32, [P, I32, P, P, P]),
        "smg_plan_mesh": (I32, [P, I32, P, P, P, P]),
        "smg_plan_prolongation": (I32, [P, I32, P, P, P, P]),
        "smg_plan_pattern": (I32, [P, I32, P, P]),
        "smg_plan_colouring": (I32, [P, I32, P]),
        "smg_plan_unknowns": (I32, [P, P, P]),
        "smg_plan_kept_coarse": (I32, [P, P, P]),
        "smg_plan_stats": (I32, [P, I32, P]),
        "smg_plan_save": (I32, [P, ctypes.c_char_p]),
        "smg_plan_load": (I32, [ctypes.c_char_p, P]),
        "smg_create": (I32, [P, P, P]),
        "smg_setup": (I32, [P, I64, P, I64, P, P, P]),
        "smg_destroy": (None, [P]),
        "smg_set_options": (I32, [P, P]),
        "smg_update_positions": (I32, [P, P, D, P]),
        "smg_update_t": (I32, [P, D, P]),
        "smg_update_matrix": (I32, [P, P, P]),
        "smg_solve": (I32, [P, P, P, I32, P, P]),
        "smg_solve_async": (I32, [P, P, P, I32, P]),
        "smg_solve_result": (I32, [P, P]),
        "smg_vcycle": (I32, [P, P, P, I32, P]),
        "smg_mass": (I32, [P, P, P]),
        "smg_apply_mass": (I32, [P, P, P, I32, P]),
        "smg_level_matrix": (I32, [P, I32, P, P]),
        "smg_run_stage": (I32, [P, I32, I32, I32, I32, I32, P]),
        "smg_level_config": (I32, [P, I32, P]),
        "smg_level_restriction": (I32, [P, I32, P]),
        "smg_level_staged": (I32, [P, I32, P]),
        "smg_cycle_config": (I32, [P, P]),
        "smg_device_bytes": (I64, [P]),
        "smg_residual_norms_noalloc": (I32, [I64, P, P, P, P, P, I32, P, P]),
        "smg_launch_counts": (I32, [P, I32, P]),
        "smg_operator_grad": (I32, [P, P, D, P, P, I32, P, P, P]),
        "smg_lumped_mass": (I32, [P, P, P, P]),
        "smg_mass_grad": (I32, [P, P, P, P, P]),
        "smg_batch_create": (I32, [P, I32, P]),
        "smg_batch_destroy": (None, [P]),
        "smg_batch_offsets": (I32, [P, P, P]),
        "smg_batch_update_positions": (I32, [P, P, D, P]),
        "smg_batch_solve": (I32, [P, P, P, I32, P, P]),
        "smg_batch_set_mode": (I32, [P, I32]),
        "smg_batch_set_wait_limit": (I32, [P, D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L, path


lib, library_path = _load()


def _check(status, where):
    if status != 0:
        raise SmgError(status, where)


def _vp(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


_NP = {ctypes.c_double: np.float64, ctypes.c_int32: np.int32, ctypes.c_int64: np.int64}


def _ptr_array(ptr, ctype, count):
    if count == 0 or not ptr:
        return np.zeros(0, dtype=_NP[ctype])
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), (count,)).copy()


def make_options(**kw):
    o = Options()
    lib.smg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


class Plan:
    """Geometry-only setup (host): decimation, self-parameterization, P, symbolic
    coarse patterns, colourings.  Wraps smg_plan_*."""

    def __init__(self, V=None, F=None, dirichlet=None, _handle=None, **opts):
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
            return
        V = np.ascontiguousarray(V, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        mask = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
        o = make_options(**opts)
        st = lib.smg_plan_build(_vp(V), V.shape[0], _vp(F), F.shape[0], _vp(mask), ctypes.byref(o),
                                ctypes.byref(self._h))
        _check(st, "smg_plan_build")

    @classmethod
    def load(cls, path):
        h = ctypes.c_void_p()
        _check(lib.smg_plan_load(os.fsencode(path), ctypes.byref(h)), "smg_plan_load")
        return cls(_handle=h)

    def save(self, path):
        _check(lib.smg_plan_save(self._h, os.fsencode(path)), "smg_plan_save")

    def close(self):
        if self._h:
            lib.smg_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self):
        return lib.smg_plan_num_levels(self._h)

    def level_info(self, level):
        n, nnz, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib.smg_plan_level_info(self._h, level, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc)),
               "smg_plan_level_info")
        return n.value, nnz.value, nc.value

    def mesh(self, level):
        n, m = ctypes.c_int64(), ctypes.c_int64()
        V, F = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.smg_plan_mesh(self._h, level, ctypes.byref(n), ctypes.byref(m), ctypes.byref(V), ctypes.byref(F)),
               "smg_plan_mesh")
        return (_ptr_array(V, ctypes.c_double, 3 * n.value).reshape(-1, 3),
                _ptr_array(F, ctypes.c_int32, 3 * m.value).reshape(-1, 3))

    def prolongation(self, level):
        """P_level (level >= 1) before Dirichlet reduction: (idx n_f x 3, w n_f x 3, n_coarse)."""
        nf, nc = ctypes.c_int64(), ctypes.c_int64()
        ip, wp = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.smg_plan_prolongation(self._h, level, ctypes.byref(nf), ctypes.byref(nc), ctypes.byref(ip),
                                         ctypes.byref(wp)), "smg_plan_prolongation")
        return (_ptr_array(ip, ctypes.c_int32, 3 * nf.value).reshape(-1, 3),
                _ptr_array(wp, ctypes.c_double, 3 * nf.value).reshape(-1, 3), nc.value)

    def prolongation_csr(self, level):
        import scipy.sparse as sp
        idx, w, nc = self.prolongation(level)
        r = np.repeat(np.arange(idx.shape[0]), 3)
        ok = idx.ravel() >= 0
        return sp.csr_matrix((w.ravel()[ok], (r[ok], idx.ravel()[ok])), shape=(idx.shape[0], nc))

    def pattern(self, level):
        n, nnz, _ = self.level_info(level)
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.smg_plan_pattern(self._h, level, ctypes.byref(rp), ctypes.byref(ci)), "smg_plan_pattern")
        return _ptr_array(rp, ctypes.c_int64, n + 1), _ptr_array(ci, ctypes.c_int32, nnz)

    def colouring(self, level):
        n, _, _ = self.level_info(level)
        cp = ctypes.c_void_p()
        _check(lib.smg_plan_colouring(self._h, level, ctypes.byref(cp)), "smg_plan_colouring")
        return _ptr_array(cp, ctypes.c_int32, n)

    def unknowns(self):
        nu, vp = ctypes.c_int64(), ctypes.c_void_p()
        _check(lib.smg_plan_unknowns(self._h, ctypes.byref(nu), ctypes.byref(vp)), "smg_plan_unknowns")
        return _ptr_array(vp, ctypes.c_int32, nu.value)

    def kept_coarse(self):
        nk, kp = ctypes.c_int64(), ctypes.c_void_p()
        _check(lib.smg_plan_kept_coarse(self._h, ctypes.byref(nk), ctypes.byref(kp)), "smg_plan_kept_coarse")
        return _ptr_array(kp, ctypes.c_int32, nk.value)

    def stats(self, level):
        out = (ctypes.c_int64 * 9)()
        _check(lib.smg_plan_stats(self._h, level, out), "smg_plan_stats")
        keys = ["collapses", "rejected_link", "rejected_boundary", "rejected_flip", "rejected_angle",
                "rejected_quality", "rejected_solve", "clamped", "worst_negative_e15"]
        return dict(zip(keys, list(out)))


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype_name="float64"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError("expected float64, got %s" % t.dtype)
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Hierarchy:
    """Device hierarchy on the current CUDA device (smg_create / smg_setup)."""

    def __init__(self, plan=None, V=None, F=None, dirichlet=None, **opts):
        import torch  # noqa: F401  (initialises the CUDA context the library attaches to)
        self._h = ctypes.c_void_p()
        o = make_options(**opts)
        if plan is None:
            plan = Plan(V, F, dirichlet, **opts)
        self.plan = plan
        _check(lib.smg_create(plan._h, ctypes.byref(o), ctypes.byref(self._h)), "smg_create")
        self.n_unknowns = plan.level_info(0)[0]
        self.n_vertices = plan.mesh(0)[0].shape[0]

    def close(self):
        if self._h:
            lib.smg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        o = make_options(**kw)
        _check(lib.smg_set_options(self._h, ctypes.byref(o)), "smg_set_options")

    def update_positions(self, V, t, stream=None):
        _check(lib.smg_update_positions(self._h, _dev_ptr(V), float(t), _stream_ptr(stream)), "smg_update_positions")

    def update_t(self, t, stream=None):
        _check(lib.smg_update_t(self._h, float(t), _stream_ptr(stream)), "smg_update_t")

    def update_matrix(self, vals, stream=None):
        _check(lib.smg_update_matrix(self._h, _dev_ptr(vals), _stream_ptr(stream)), "smg_update_matrix")

    def solve(self, b, x=None, stream=None, check=True):
        """Solve A x = b in place of x (zeros if None); returns (x, info dict)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        info = Info()
        st = lib.smg_solve(self._h, _dev_ptr(b), _dev_ptr(x), nrhs, ctypes.byref(info), _stream_ptr(stream))
        if check and st not in (0, 5):
            _check(st, "smg_solve")
        d = info.as_dict()
        d["return"] = st
        return x, d

    def solve_async(self, b, x, stream=None):
        """Enqueue a solve without waiting; call solve_result() after synchronising."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        _check(lib.smg_solve_async(self._h, _dev_ptr(b), _dev_ptr(x), nrhs, _stream_ptr(stream)), "smg_solve_async")
        return x

    def solve_result(self, check=True):
        info = Info()
        st = lib.smg_solve_result(self._h, ctypes.byref(info))
        if check and st not in (0, 5):
            _check(st, "smg_solve_result")
        d = info.as_dict()
        d["return"] = st
        return d

    def vcycle(self, b, x, stream=None):
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        _check(lib.smg_vcycle(self._h, _dev_ptr(b), _dev_ptr(x), nrhs, _stream_ptr(stream)), "smg_vcycle")
        return x

    def mass(self, stream=None):
        import torch
        m = torch.empty(self.n_unknowns, dtype=torch.float64, device="cuda")
        _check(lib.smg_mass(self._h, _dev_ptr(m), _stream_ptr(stream)), "smg_mass")
        return m

    def apply_mass(self, x, stream=None):
        import torch
        y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        _check(lib.smg_apply_mass(self._h, _dev_ptr(x), _dev_ptr(y), nrhs, _stream_ptr(stream)), "smg_apply_mass")
        return y

    def launch_counts(self, nrhs=1):
        """(kernels per update_positions, per solve outside the loop, per loop iteration)."""
        out = (ctypes.c_int32 * 3)()
        _check(lib.smg_launch_counts(self._h, int(nrhs), out), "smg_launch_counts")
        return tuple(out)

    def operator_grad(self, V, t, lam, x, stream=None):
        """(-d/dV lam^T A(V,t) x  as n x 3,  -lam^T L x  as a 1-element tensor)."""
        import torch
        gV = torch.empty_like(V)
        dt = torch.empty(1, dtype=torch.float64, device=V.device)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        _check(lib.smg_operator_grad(self._h, _dev_ptr(V), float(t), _dev_ptr(lam), _dev_ptr(x), nrhs, _dev_ptr(gV),
                                     _dev_ptr(dt), _stream_ptr(stream)), "smg_operator_grad")
        return gV, dt

    def lumped_mass(self, V, stream=None):
        import torch
        m = torch.empty(self.n_unknowns, dtype=torch.float64, device=V.device)
        _check(lib.smg_lumped_mass(self._h, _dev_ptr(V), _dev_ptr(m), _stream_ptr(stream)), "smg_lumped_mass")
        return m

    def mass_grad(self, V, w, stream=None):
        import torch
        gV = torch.empty_like(V)
        _check(lib.smg_mass_grad(self._h, _dev_ptr(V), _dev_ptr(w), _dev_ptr(gV), _stream_ptr(stream)),
               "smg_mass_grad")
        return gV

    def level_matrix(self, level, stream=None):
        """Values of A_level aligned with plan.pattern(level)."""
        nnz = self.plan.level_info(level)[1]
        out = np.zeros(nnz)
        _check(lib.smg_level_matrix(self._h, level, _vp(out), _stream_ptr(stream)), "smg_level_matrix")
        return out

    STAGES = {"cycle": 0, "sweep": 1, "residual": 2, "galerkin": 3, "factor": 4, "update": 5}

    def run_stage(self, stage, level=0, nrhs=1, precision=FP64, count=1, stream=None):
        """Enqueue `count` repetitions of one stage (measurement hook, asynchronous)."""
        _check(lib.smg_run_stage(self._h, self.STAGES[stage], level, nrhs, precision, count, _stream_ptr(stream)),
               "smg_run_stage")

    def level_config(self, level):
        """(lanes per row binary64, lanes per row binary32, colours, slices) of a level."""
        out = (ctypes.c_int32 * 4)()
        _check(lib.smg_level_config(self._h, level, out), "smg_level_config")
        return tuple(out)

    def level_restriction(self, level):
        """(entries of Q = P^T A_l, entries of P^T, padded slots, lanes per row binary64,
        binary32) of the fused residual-restriction operator from `level` to the next."""
        out = (ctypes.c_int64 * 5)()
        _check(lib.smg_level_restriction(self._h, level, out), "smg_level_restriction")
        return tuple(out)

    def level_staged(self, level):
        """(binary64, binary32): 1 where the level's sweep runs one lane per row with
        its matrix entries staged in shared memory by bulk copies, 0 for the
        register-prefetching kernel."""
        out = (ctypes.c_int32 * 2)()
        _check(lib.smg_level_staged(self._h, level, out), "smg_level_staged")
        return tuple(out)

    def cycle_config(self):
        """(H, first cluster-tail level binary64, binary32, CTAs per cluster)."""
        out = (ctypes.c_int32 * 4)()
        _check(lib.smg_cycle_config(self._h, out), "smg_cycle_config")
        return tuple(out)

    @property
    def device_bytes(self):
        return lib.smg_device_bytes(self._h)


class Batch:
    """Several hierarchies (same device): one graph launch updates every mesh
    (a branch per mesh); one persistent kernel launch solves every mesh
    (mode "persistent", the default), or one graph launch with a branch per
    mesh (mode "graph") (smg_batch_*).  Vectors are the meshes' unknown
    vectors concatenated; positions the meshes' vertices concatenated."""

    MODES = {"persistent": 0, "graph": 1}

    def __init__(self, hierarchies):
        self.hs = list(hierarchies)
        arr = (ctypes.c_void_p * len(self.hs))(*[h._h.value for h in self.hs])
        self._h = ctypes.c_void_p()
        _check(lib.smg_batch_create(arr, len(self.hs), ctypes.byref(self._h)), "smg_batch_create")
        u = (ctypes.c_int64 * (len(self.hs) + 1))()
        v = (ctypes.c_int64 * (len(self.hs) + 1))()
        _check(lib.smg_batch_offsets(self._h, u, v), "smg_batch_offsets")
        self.unknown_offsets = list(u)
        self.vertex_offsets = list(v)

    def close(self):
        if self._h:
            lib.smg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode):
        _check(lib.smg_batch_set_mode(self._h, self.MODES[mode]), "smg_batch_set_mode")

    def set_wait_limit(self, seconds):
        """Watchdog of the persistent launch (seconds a warp may find no work)."""
        _check(lib.smg_batch_set_wait_limit(self._h, float(seconds)), "smg_batch_set_wait_limit")

    def update_positions(self, V, t, stream=None):
        _check(lib.smg_batch_update_positions(self._h, _dev_ptr(V), float(t), _stream_ptr(stream)),
               "smg_batch_update_positions")

    def solve(self, b, x=None, stream=None, check=True):
        """Solve every mesh; returns (x, list of info dicts)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        infos = (Info * len(self.hs))()
        st = lib.smg_batch_solve(self._h, _dev_ptr(b), _dev_ptr(x), nrhs, infos, _stream_ptr(stream))
        if check and st != 0:
            _check(st, "smg_batch_solve")
        return x, [i.as_dict() for i in infos]


def _autograd():
    import torch

    class SolveFn(torch.autograd.Function):
        """x = A(V, t)^{-1} b through the hierarchy; backward runs the adjoint solve
        lambda = A^{-1} dl/dx with the same hierarchy (A is symmetric) and the
        per-face derivative kernels for V and t."""

        @staticmethod
        def forward(ctx, V, t, b, h):
            tv = float(t)
            h.update_positions(V.detach().contiguous(), tv)
            x, _ = h.solve(b.detach().contiguous())
            ctx.h, ctx.t = h, tv
            ctx.save_for_backward(V, x)
            return x

        @staticmethod
        def backward(ctx, gx):
            V, x = ctx.saved_tensors
            h = ctx.h
            Vc = V.detach().contiguous()
            h.update_positions(Vc, ctx.t)  # the operator of this forward pass
            lam, _ = h.solve(gx.detach().contiguous())
            gV, dt = h.operator_grad(Vc, ctx.t, lam, x)
            return gV, dt.reshape(()), lam, None

    class MassFn(torch.autograd.Function):
        """Lumped mass diagonal of the unknowns as a function of the positions."""

        @staticmethod
        def forward(ctx, V, h):
            ctx.h = h
            ctx.save_for_backward(V)
            return h.lumped_mass(V.detach().contiguous())

        @staticmethod
        def backward(ctx, gm):
            (V,) = ctx.saved_tensors
            return ctx.h.mass_grad(V.detach().contiguous(), gm.detach().contiguous()), None

    return SolveFn, MassFn


def differentiable_solve(h, V, t, b):
    """x = A(V, t)^{-1} b, differentiable in V (n x 3), t (0-d tensor) and b."""
    import torch
    SolveFn, _ = _autograd()
    if not torch.is_tensor(t):
        t = torch.tensor(float(t), dtype=torch.float64, device=V.device)
    return SolveFn.apply(V, t, b, h)


def differentiable_mass(h, V):
    """Lumped mass diagonal (unknowns) of positions V, differentiable in V."""
    _, MassFn = _autograd()
    return MassFn.apply(V, h)
