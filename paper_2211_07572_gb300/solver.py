"""Thin PyTorch-facing wrapper over the C ABI (include/slab.h).

PyTorch provides device memory and the stream; every arithmetic step runs in
libslab.so.  Tensors passed in must be CUDA float64 and contiguous; they are
never copied to the host except for the explicit host outputs (relative
residuals, T blocks).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np
import torch

from . import _lib

_PREC = {"fp64": _lib.PREC_FP64, "fp32": _lib.PREC_FP32, "tf32": _lib.PREC_TF32, "fp64tc": _lib.PREC_FP64_TC}
_STAGE2 = {"auto": 0, "sweep": 1, "oddeven": 2}


def _dev(x, device) -> torch.Tensor:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(device=device, dtype=torch.float64)
    return x.contiguous()


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class SlabSolver:
    """Factor A for one grid/coefficient set (Algorithm 3) and solve with it (Algorithm 4).

    dim, n: grid (unit square/cube, h = 1/n); b: interface spacing (b | n);
    kind: 0 Poisson, 1 diffusion -div(kappa grad u), 2 Helmholtz -Lap u - (omega/c)^2 u;
    kappa / c: node fields with (n+1)^dim entries; beta: the velocity components (dim, (n+1)^dim)
    of the convection-diffusion kind; precision: "fp32" (FP32 factor, FP64
    refinement), "tf32" (as fp32 with single-pass TF32 tensor products in the factor) or
    "fp64" (plain FP64 path); stage2: "auto", "sweep" (Algorithm 1) or
    "oddeven"; interface_precision: precision of the interface system (default: "fp64" for
    Helmholtz with an FP32 factor, else the factor precision); krylov: 0 for plain iterative
    refinement, m > 0 for restarted FP64 GMRES(m) preconditioned by the factor; pivot: row choice of
    the Gauss-Jordan interface elimination (Helmholtz, convection-diffusion): "tournament" over all
    remaining rows, or "local" (inside each 64-row diagonal block, for diagonally dominant systems).
    """

    def __init__(self, dim: int, n: int, b: int, kind: int, kappa=None, c=None, omega: float = 0.0,
                 beta=None, precision: str = "fp32", rtol: float = 1e-10, max_refine: int = 30,
                 stream: Optional[torch.cuda.Stream] = None, device=None, profile: bool = False,
                 stage2: str = "auto", interface_precision: Optional[str] = None, krylov: int = 0,
                 pivot: str = "tournament"):
        self.lib = _lib.load()
        self.device = (torch.device(device) if device is not None
                       else torch.device("cuda", torch.cuda.current_device()))
        self.dim, self.n, self.b, self.kind = dim, n, b, kind
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._kappa = _dev(kappa, self.device)
        self._c = _dev(c, self.device)
        self._beta = _dev(beta, self.device)
        grid = _lib.SlabGrid(dim, n)
        co = _lib.SlabCoeffs(kind, _ptr(self._kappa), _ptr(self._c), float(omega), _ptr(self._beta))
        opts = _lib.SlabOpts()
        self.lib.slab_default_opts(ctypes.byref(opts))
        opts.factor_prec = _PREC[precision]
        opts.rtol = float(rtol)
        opts.max_refine = int(max_refine)
        opts.stream = ctypes.c_void_p(self.stream.cuda_stream)
        opts.profile = int(profile)
        opts.stage2 = _STAGE2[stage2]
        opts.interface_prec = -1 if interface_precision is None else _PREC[interface_precision]
        opts.krylov = int(krylov)
        opts.pivot = {"tournament": 0, "local": 1}[pivot]
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.slab_factor(ctypes.byref(grid), ctypes.byref(co), int(b), ctypes.byref(opts),
                                            ctypes.byref(h)), "slab_factor")
        self.h = h
        N = ctypes.c_int64(); s = ctypes.c_int64(); ni = ctypes.c_int()
        self.lib.slab_sizes(self.h, ctypes.byref(N), ctypes.byref(s), ctypes.byref(ni))
        self.N, self.s, self.NI = N.value, s.value, ni.value

    # ------------------------------------------------------------------ helpers
    def _vec(self, x, k=None) -> torch.Tensor:
        x = _dev(x, self.device)
        if x.dim() == 1:
            x = x.view(1, -1)
        x = x.reshape(-1, self.N)
        return x

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.slab_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable: bool = True):
        _lib.check(self.lib.slab_profile(self.h, int(enable)), "slab_profile")

    def profile_read(self):
        """(ms, launches) per kernel class since the previous read (dicts keyed by class name)."""
        n = len(_lib.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _lib.check(self.lib.slab_profile_read(self.h, ms, cnt, n), "slab_profile_read")
        return ({k: ms[i] for i, k in enumerate(_lib.KERNEL_CLASSES)},
                {k: int(cnt[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)})

    @property
    def device_bytes(self) -> int:
        return int(self.lib.slab_device_bytes(self.h))

    @property
    def stage2_order(self) -> str:
        """"sweep" or "oddeven": the Stage-2 elimination order the factor used."""
        return {1: "sweep", 2: "oddeven"}.get(int(self.lib.slab_stage2_order(self.h)), "?")

    # ------------------------------------------------------------------ API
    def solve(self, f, u: Optional[torch.Tensor] = None, allow_noconv: bool = False
              ) -> Tuple[torch.Tensor, np.ndarray, int]:
        """u = A^-1 f with refinement; returns (u, relres per rhs, refinement steps)."""
        f = self._vec(f)
        k = f.shape[0]
        if u is None:
            u = torch.empty_like(f)
        rel = (ctypes.c_double * max(k, 1))()
        it = ctypes.c_int()
        st = self.lib.slab_solve(self.h, _ptr(f), _ptr(u), k, rel, ctypes.byref(it))
        _lib.check(st, "slab_solve", allow=(_lib.SLAB_ENOCONV,) if allow_noconv else ())
        return u, np.array(rel[:k]), it.value

    def residual(self, u, f) -> torch.Tensor:
        u, f = self._vec(u), self._vec(f)
        r = torch.empty_like(f)
        _lib.check(self.lib.slab_apply_residual(self.h, _ptr(u), _ptr(f), _ptr(r), f.shape[0]), "residual")
        return r

    def apply(self, x) -> torch.Tensor:
        x = self._vec(x)
        y = torch.empty_like(x)
        _lib.check(self.lib.slab_apply(self.h, _ptr(x), _ptr(y), x.shape[0]), "apply")
        return y

    def apply_transpose(self, x) -> torch.Tensor:
        x = self._vec(x)
        y = torch.empty_like(x)
        _lib.check(self.lib.slab_apply_transpose(self.h, _ptr(x), _ptr(y), x.shape[0]), "apply_transpose")
        return y

    def boundary_lift(self, g, f=None) -> torch.Tensor:
        """f + lift(g): the load of the interior system for Dirichlet data g given on all
        (n+1)^dim nodes (rows = right-hand sides); solve() with it gives the interior solution."""
        g = _dev(g, self.device)
        g = g.reshape(-1, (self.n + 1) ** self.dim)
        k = g.shape[0]
        fo = torch.empty((k, self.N), dtype=torch.float64, device=self.device)
        fi = None if f is None else self._vec(f)
        if fi is not None and fi.shape[0] != k:
            raise ValueError("f and g need the same number of right-hand sides")
        _lib.check(self.lib.slab_boundary_lift(self.h, _ptr(g), _ptr(fi), _ptr(fo), k), "boundary_lift")
        return fo

    def adjoint(self, dLdu, u=None, allow_noconv: bool = False) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
        g = self._vec(dLdu)
        lam = torch.empty_like(g)
        grad = None
        if u is not None:
            u = self._vec(u)
            grad = torch.zeros((self.n + 1,) * self.dim, dtype=torch.float64, device=self.device)
        st = self.lib.slab_adjoint(self.h, _ptr(g), _ptr(u), _ptr(lam), _ptr(grad), g.shape[0])
        _lib.check(st, "slab_adjoint", allow=(_lib.SLAB_ENOCONV,) if allow_noconv else ())
        return lam, grad

    def reduced_rhs(self, f) -> torch.Tensor:
        f = self._vec(f)
        out = torch.empty((f.shape[0], self.NI * self.s), dtype=torch.float64, device=self.device)
        _lib.check(self.lib.slab_reduced_rhs(self.h, _ptr(f), _ptr(out), f.shape[0]), "reduced_rhs")
        return out

    def interface_solve(self, ftilde) -> torch.Tensor:
        ft = _dev(ftilde, self.device).reshape(-1, self.NI * self.s)
        out = torch.empty_like(ft)
        _lib.check(self.lib.slab_interface_solve(self.h, _ptr(ft), _ptr(out), ft.shape[0]), "interface_solve")
        return out

    def interior_solve(self, f, utilde) -> torch.Tensor:
        f = self._vec(f)
        ut = _dev(utilde, self.device).reshape(-1, self.NI * self.s)
        u = torch.empty_like(f)
        _lib.check(self.lib.slab_interior_solve(self.h, _ptr(f), _ptr(ut), _ptr(u), f.shape[0]),
                   "interior_solve")
        return u

    def apply_T(self, X) -> torch.Tensor:
        """Y = T X for k interface vectors ([k][N_I s] rows) without forming T (the sketch operation
        of Sec. 3.3): one interior solve with zero load, then the interface rows of A u."""
        X = _dev(X, self.device).reshape(-1, self.NI * self.s)
        k = X.shape[0]
        Y = torch.empty_like(X)
        work = torch.empty((2 * k, self.N), dtype=torch.float64, device=self.device)
        _lib.check(self.lib.slab_apply_T(self.h, _ptr(X), _ptr(Y), k, _ptr(work)), "apply_T")
        return Y

    def T_block(self, which: int, q: int) -> np.ndarray:
        out = np.empty((self.s, self.s), dtype=np.float64)
        _lib.check(self.lib.slab_get_T_block(self.h, which, q, out.ctypes.data_as(ctypes.c_void_p)), "T_block")
        return out


class SlabSolveFunction(torch.autograd.Function):
    """u = A(kappa)^-1 f for the diffusion operator; backward by the adjoint solve.

    dL/df = lambda and dL/dkappa = -lambda^T (dA/dkappa) u with A^T lambda = dL/du.
    """

    @staticmethod
    def forward(ctx, kappa, f, n: int, b: int, precision: str = "fp32"):
        solver = SlabSolver(2, n, b, _lib.DIFFUSION, kappa=kappa.detach(), precision=precision, rtol=1e-13)
        u, _, _ = solver.solve(f.detach(), allow_noconv=True)
        ctx.solver = solver
        ctx.save_for_backward(u)
        return u.view_as(f)

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        lam, gk = ctx.solver.adjoint(gu.contiguous(), u, allow_noconv=True)
        ctx.solver.close()
        return gk, lam.view_as(gu), None, None, None


class SlabBatch:
    """Independent problems (uneven sizes allowed) factored, solved and differentiated together:
    slab_factor_batched / slab_solve_batched / slab_adjoint_batched, each problem on a stream of
    its own, driven by up to `workers` host threads.

    problems: list of dicts with keys dim, n, b, kind and kappa / c / omega / beta as for SlabSolver.
    Vectors are lists of device tensors, one [k][N_i] tensor per problem.
    """

    def __init__(self, problems, precision: str = "fp32", rtol: float = 1e-10, max_refine: int = 30,
                 stage2: str = "sweep", krylov: int = 0, workers: int = 8):
        self.lib = _lib.load()
        self.workers = int(workers)
        cnt = len(problems)
        self.count = cnt
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._coef = []
        grids = (_lib.SlabGrid * cnt)()
        coeffs = (_lib.SlabCoeffs * cnt)()
        bs = (ctypes.c_int * cnt)()
        self.meta = []
        for i, p in enumerate(problems):
            kap = _dev(p.get("kappa"), self.device)
            cc = _dev(p.get("c"), self.device)
            bet = _dev(p.get("beta"), self.device)
            self._coef.append((kap, cc, bet))
            grids[i] = _lib.SlabGrid(p["dim"], p["n"])
            coeffs[i] = _lib.SlabCoeffs(p["kind"], _ptr(kap), _ptr(cc), float(p.get("omega", 0.0)), _ptr(bet))
            bs[i] = p["b"]
            self.meta.append((p["dim"], p["n"]))
        opts = _lib.SlabOpts()
        self.lib.slab_default_opts(ctypes.byref(opts))
        opts.factor_prec = _PREC[precision]
        opts.rtol = float(rtol)
        opts.max_refine = int(max_refine)
        opts.stage2 = _STAGE2[stage2]
        opts.interface_prec = -1
        opts.krylov = int(krylov)
        self.h = (ctypes.c_void_p * cnt)()
        torch.cuda.synchronize()
        st = self.lib.slab_factor_batched(cnt, grids, coeffs, bs, ctypes.byref(opts), self.workers, self.h)
        if st != 0:
            self.close()
            _lib.check(st, "slab_factor_batched")

    def _ptrs(self, ts):
        arr = (ctypes.c_void_p * self.count)()
        for i, t in enumerate(ts):
            arr[i] = None if t is None else t.data_ptr()
        return arr

    def solve(self, fs, allow_noconv: bool = False):
        fs = [_dev(f, self.device).reshape(-1, (n - 1) ** d) for f, (d, n) in zip(fs, self.meta)]
        us = [torch.empty_like(f) for f in fs]
        ks = (ctypes.c_int * self.count)(*[f.shape[0] for f in fs])
        rel = [np.zeros(f.shape[0]) for f in fs]
        relp = (ctypes.c_void_p * self.count)(*[r.ctypes.data for r in rel])
        its = (ctypes.c_int * self.count)()
        torch.cuda.synchronize()
        st = self.lib.slab_solve_batched(self.count, self.h, self._ptrs(fs), self._ptrs(us), ks, relp, its,
                                         self.workers)
        _lib.check(st, "slab_solve_batched", allow=(_lib.SLAB_ENOCONV,) if allow_noconv else ())
        return us, rel, list(its)

    def adjoint(self, dLdus, us, allow_noconv: bool = False):
        gs = [_dev(g, self.device).reshape(-1, (n - 1) ** d) for g, (d, n) in zip(dLdus, self.meta)]
        lams = [torch.empty_like(g) for g in gs]
        grads = [torch.zeros((n + 1,) * d, dtype=torch.float64, device=self.device) for (d, n) in self.meta]
        ks = (ctypes.c_int * self.count)(*[g.shape[0] for g in gs])
        torch.cuda.synchronize()
        st = self.lib.slab_adjoint_batched(self.count, self.h, self._ptrs(gs), self._ptrs(us), self._ptrs(lams),
                                           self._ptrs(grads), ks, self.workers)
        _lib.check(st, "slab_adjoint_batched", allow=(_lib.SLAB_ENOCONV,) if allow_noconv else ())
        return lams, grads

    def close(self):
        h = getattr(self, "h", None)
        if h is not None:
            for i in range(self.count):
                if h[i]:
                    self.lib.slab_destroy(h[i])
                    h[i] = None
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A raw device buffer of the library, presented to torch through __cuda_array_interface__
    (zero-copy: torch.as_tensor aliases it)."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class GraphBatch:
    """Independent 2-D diffusion problems with the least-squares objective L_i = ||u_i - t_i||^2,
    run as CUDA graphs (slab_batch_create / slab_batch_run / slab_batch_results).

    Every run computes, per problem, the factor, u_i = A_i^-1 f_i (one solve pass and `steps`
    refinement passes), L_i, lambda_i = A_i^-T dL_i/du_i and grad_i = dL_i/dkappa_i.  All device
    memory is allocated once at construction; the per-problem inputs (kappa, f, target) and outputs
    (u, lam, grad) are tensors aliasing the batch's own buffers (``inputs(i)`` / ``outputs(i)``).
    sizes: grid sizes n_i; b: interface spacing (int or one per problem); wave: problems per graph
    (0: all in one); branches: parallel graph branches per wave.
    """

    def __init__(self, sizes, b=16, precision: str = "fp32", rtol: float = 1e-10, steps: int = 4,
                 wave: int = 0, branches: int = 16, stage2: str = "auto"):
        self.lib = _lib.load()
        self.sizes = [int(n) for n in sizes]
        cnt = len(self.sizes)
        bs = [int(b)] * cnt if np.isscalar(b) else [int(x) for x in b]
        opts = _lib.SlabOpts()
        self.lib.slab_default_opts(ctypes.byref(opts))
        opts.factor_prec = _PREC[precision]
        opts.rtol = float(rtol)
        opts.stage2 = _STAGE2[stage2]
        self.h = ctypes.c_void_p()
        narr = (ctypes.c_int * cnt)(*self.sizes)
        barr = (ctypes.c_int * cnt)(*bs)
        torch.cuda.synchronize()
        _lib.check(self.lib.slab_batch_create(cnt, narr, barr, ctypes.byref(opts), int(steps), int(wave),
                                              int(branches), ctypes.byref(self.h)), "slab_batch_create")
        self.count = cnt
        self._bufs = []
        for i, n in enumerate(self.sizes):
            ptrs = [ctypes.c_void_p() for _ in range(6)]
            _lib.check(self.lib.slab_batch_buffers(self.h, i, *[ctypes.byref(p) for p in ptrs]), "slab_batch_buffers")
            shapes = [(n + 1, n + 1), (1, (n - 1) ** 2), (1, (n - 1) ** 2), (1, (n - 1) ** 2), (1, (n - 1) ** 2),
                      (n + 1, n + 1)]
            t = [torch.as_tensor(_DeviceArray(p.value, sh), device="cuda") for p, sh in zip(ptrs, shapes)]
            self._bufs.append(dict(zip(("kappa", "f", "target", "u", "lam", "grad"), t)))

    @property
    def device_bytes(self) -> int:
        return int(self.lib.slab_batch_device_bytes(self.h))

    def inputs(self, i: int):
        """(kappa, f, target) of problem i: tensors aliasing the batch's input buffers."""
        d = self._bufs[i]
        return d["kappa"], d["f"], d["target"]

    def outputs(self, i: int):
        """(u, lam, grad) of problem i after a run: tensors aliasing the batch's output buffers."""
        d = self._bufs[i]
        return d["u"], d["lam"], d["grad"]

    def set_inputs(self, i: int, kappa, f, target):
        k, ff, t = self.inputs(i)
        k.copy_(torch.as_tensor(kappa, dtype=torch.float64).reshape(k.shape), non_blocking=True)
        ff.copy_(torch.as_tensor(f, dtype=torch.float64).reshape(ff.shape), non_blocking=True)
        t.copy_(torch.as_tensor(target, dtype=torch.float64).reshape(t.shape), non_blocking=True)

    def run(self, stream: Optional[torch.cuda.Stream] = None):
        """Enqueue one run (one graph launch per wave) on `stream` (default: the current stream)."""
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(self.lib.slab_batch_run(self.h, ctypes.c_void_p(s.cuda_stream)), "slab_batch_run")

    def results(self, allow_noconv: bool = False):
        """Wait for the last run: (losses, relres of u, relres of lambda) as numpy arrays."""
        L = np.zeros(self.count)
        ru = np.zeros(self.count)
        rl = np.zeros(self.count)
        st = self.lib.slab_batch_results(self.h, L.ctypes.data_as(ctypes.c_void_p), ru.ctypes.data_as(ctypes.c_void_p),
                                         rl.ctypes.data_as(ctypes.c_void_p))
        _lib.check(st, "slab_batch_results", allow=(_lib.SLAB_ENOCONV,) if allow_noconv else ())
        return L, ru, rl

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._bufs = []
            self.lib.slab_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batched_adjoint_gradients(problems, fs, u_targets, wave: int = 32, workers: int = 8,
                              precision: str = "fp32", rtol: float = 1e-12):
    """Loss L_i = ||u_i - u_t,i||^2 and dL_i/dkappa_i for independent diffusion problems, processed
    in waves of `wave` problems (factor, solve, adjoint solve and gradient per wave, then free).
    Returns (losses, gradients) as lists."""
    losses, grads = [], []
    for w0 in range(0, len(problems), wave):
        sl = slice(w0, w0 + wave)
        batch = SlabBatch(problems[sl], precision=precision, rtol=rtol, max_refine=40, workers=workers)
        us, _, _ = batch.solve(fs[sl], allow_noconv=True)
        uts = [_dev(t, batch.device).reshape_as(u) for t, u in zip(u_targets[sl], us)]
        losses += [float(((u - t) ** 2).sum()) for u, t in zip(us, uts)]
        _, g = batch.adjoint([2 * (u - t) for u, t in zip(us, uts)], us, allow_noconv=True)
        grads += g
        batch.close()
    return losses, grads
