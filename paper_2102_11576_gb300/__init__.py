"""GB300 (sm_103a) solver for one implicit step of the volume-penalized 2D
Riesz space-fractional diffusion scheme, preconditioned by the sine-transform
(tau) preconditioner of Huang & Sun (arXiv 2102.11576).

This module is the thin Python binding of ``librsfde.so`` (include/rsfde.h):
argument marshalling only.  Every step of the solve runs in the library's
CUDA kernels; torch provides device memory and the stream.  There is no CPU
fallback: if the library is missing or the device is not a CUDA GPU the calls
raise.

Grid arrays are float64 torch tensors on the GPU, shape (n2, n1) (x fastest),
the ordering of u^k in Section 2.
"""
import ctypes
import os

import numpy as np

__all__ = ["Solver", "Batch", "RsfdeError", "load_library", "LIB_PATH", "FP64", "FP32", "DF32", "EXACT"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsfde.so")

FP64, FP32, DF32 = 0, 1, 2
EXACT = 5  # true residual only: exact integer Toeplitz products, rounded to FP64
_VARIANTS = {"fgmres_right": 0, "gmres_left": 1}
_PRECONDS = {"fp64": 0, "fp32": 1, "bf16x3": 3, "bf16": 4}
_MATVECS = {"fp64": FP64, "df32": DF32, "fp32": FP32}
_RESIDS = {"fp64": FP64, "df32": DF32, "exact": EXACT}
_BASES = {"fp64": FP64, "df32": DF32, "fp32": FP32}
CGS, CGS2 = 0, 1
_ERR = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOTCONV", -5: "ENONFINITE",
        -6: "ETIMEOUT"}


class RsfdeError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        self.name = _ERR.get(code, str(code))
        super().__init__(f"rsfde {what}: {self.name} ({code})")


class _Grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("ax", ctypes.c_double),
                ("bx", ctypes.c_double), ("ay", ctypes.c_double), ("by", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("precond_prec", ctypes.c_int32), ("arnoldi", ctypes.c_int32),
                ("use_precond", ctypes.c_int32), ("matvec_prec", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("resid_prec", ctypes.c_int32),
                ("basis_prec", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("t_ms", ctypes.c_double * 6), ("bytes", ctypes.c_double)]

    PHASES = ("rhs_and_control", "operator", "precond", "gram_schmidt", "least_squares",
              "update_and_residual")

    def as_dict(self):
        return {"iters": self.iters, "restarts": self.restarts, "converged": bool(self.converged),
                "status": _ERR.get(self.status, self.status), "rel_res": self.rel_res,
                "bnorm": self.bnorm, "t_ms": dict(zip(self.PHASES, list(self.t_ms))),
                "bytes": self.bytes}


_lib = None


def load_library(path=LIB_PATH):
    """Loads librsfde.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2102_11576_gb300._build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, d, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    lib.rsfde_opts_default.argtypes = [ctypes.POINTER(_Opts)]
    lib.rsfde_setup.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Grid), vp, d, d, d, d, d, d,
                                ctypes.POINTER(_Opts)]
    lib.rsfde_set_params.argtypes = [vp, d, d, d]
    lib.rsfde_set_opts.argtypes = [vp, ctypes.POINTER(_Opts)]
    lib.rsfde_set_stream.argtypes = [vp, vp]
    lib.rsfde_solve.argtypes = [vp, dp, dp, ctypes.POINTER(_Stats)]
    lib.rsfde_step.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(_Stats)]
    lib.rsfde_step_host.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(_Stats)]
    lib.rsfde_adjoint.argtypes = [vp, dp, dp, ctypes.POINTER(_Stats)]
    lib.rsfde_apply_M.argtypes = [vp, dp, dp]
    lib.rsfde_residual.argtypes = [vp, dp, dp, dp]
    lib.rsfde_apply_precond.argtypes = [vp, dp, dp]
    lib.rsfde_dst2.argtypes = [vp, dp, dp]
    lib.rsfde_rhs.argtypes = [vp, dp, dp, dp, dp, dp]
    lib.rsfde_get_tables.argtypes = [vp, dp, dp, dp, dp]
    lib.rsfde_get_params.argtypes = [vp, dp]
    lib.rsfde_profile_enable.argtypes = [vp, i32]
    lib.rsfde_profile_enable.restype = ctypes.c_int
    lib.rsfde_profile_read.argtypes = [vp, dp, dp]
    lib.rsfde_profile_read.restype = ctypes.c_int
    lib.rsfde_kernel_class_name.argtypes = [i32]
    lib.rsfde_kernel_class_name.restype = ctypes.c_char_p
    lib.rsfde_set_wait_cycles.argtypes = [vp, ctypes.c_int64]
    lib.rsfde_set_wait_cycles.restype = ctypes.c_int
    lib.rsfde_kernel_launches.argtypes = [vp]
    lib.rsfde_kernel_launches.restype = ctypes.c_int64
    lib.rsfde_destroy.argtypes = [vp]
    lib.rsfde_strerror.argtypes = [i32]
    lib.rsfde_strerror.restype = ctypes.c_char_p
    lib.rsfde_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(_Grid), ctypes.POINTER(vp),
                                       dp, dp, dp, dp, dp, dp, ctypes.POINTER(_Opts)]
    lib.rsfde_batch_set.argtypes = [vp, i32, dp, dp]
    lib.rsfde_batch_run.argtypes = [vp, i32, ctypes.POINTER(_Stats)]
    lib.rsfde_batch_get.argtypes = [vp, i32, dp]
    lib.rsfde_batch_kernel_launches.argtypes = [vp]
    lib.rsfde_batch_kernel_launches.restype = ctypes.c_int64
    lib.rsfde_batch_destroy.argtypes = [vp]
    lib.rsfde_autotune.argtypes = [vp, i32, vp]
    lib.rsfde_autotune.restype = ctypes.c_int
    lib.rsfde_batch_autotune.argtypes = [vp, i32]
    lib.rsfde_batch_autotune.restype = ctypes.c_int
    for name in ("rsfde_batch_create", "rsfde_batch_set", "rsfde_batch_run", "rsfde_batch_get"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("rsfde_setup", "rsfde_set_params", "rsfde_set_opts", "rsfde_set_stream",
                 "rsfde_solve", "rsfde_step", "rsfde_step_host", "rsfde_adjoint", "rsfde_apply_M",
                 "rsfde_apply_precond", "rsfde_dst2", "rsfde_rhs", "rsfde_get_tables",
                 "rsfde_get_params"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check(code, what):
    if code != 0:
        raise RsfdeError(code, what)


class Solver:
    """One linear system M = I - A + D (Eq. 2.17) and its preconditioner (Eq. 4.6)."""

    def __init__(self, n1, n2, box, in_omega, alpha1, alpha2, kx, ky, dt, eta, restart=20,
                 max_iter=10000, tol=1e-10, precond="fp64", arnoldi="cgs", use_precond=True,
                 matvec="fp64", variant="fgmres_right", use_graph=True, stream=None, resid="fp64",
                 basis="fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("rsfde needs a CUDA GPU; there is no CPU path")
        self._torch = torch
        lib = load_library()
        self.n1, self.n2 = int(n1), int(n2)
        self.N = self.n1 * self.n2
        self.device = torch.device("cuda", torch.cuda.current_device())
        mask = torch.as_tensor(np.ascontiguousarray(in_omega, dtype=np.uint8)
                               if not isinstance(in_omega, torch.Tensor) else in_omega)
        mask = mask.to(self.device, torch.uint8).contiguous().reshape(self.n2, self.n1)
        self.in_omega = mask
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = _Opts()
        lib.rsfde_opts_default(ctypes.byref(o))
        o.restart, o.max_iter, o.tol = int(restart), int(max_iter), float(tol)
        o.precond_prec = _PRECONDS[precond]
        o.arnoldi = {"cgs": CGS, "cgs2": CGS2}[arnoldi]
        o.use_precond = int(bool(use_precond))
        o.matvec_prec = _MATVECS[matvec]
        o.variant = _VARIANTS[variant]
        o.use_graph = int(bool(use_graph))
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        o.resid_prec = _RESIDS[resid]
        o.basis_prec = _BASES[basis]
        self._opts = o
        g = _Grid(self.n1, self.n2, *map(float, box))
        h = ctypes.c_void_p()
        _check(lib.rsfde_setup(ctypes.byref(h), ctypes.byref(g), _ptr(mask), float(alpha1),
                               float(alpha2), float(kx), float(ky), float(dt), float(eta),
                               ctypes.byref(o)), "setup")
        self._h = h
        self._lib = lib
        self.box = tuple(map(float, box))
        self.alpha1, self.alpha2, self.kx, self.ky, self.dt, self.eta = (
            alpha1, alpha2, kx, ky, dt, eta)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rsfde_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers --
    def _grid(self, t, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if t.numel() != self.N or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {self.N} elements")
        return t

    def empty(self):
        return self._torch.empty((self.n2, self.n1), dtype=self._torch.float64, device=self.device)

    def set_options(self, **kw):
        o = self._opts
        for k, v in kw.items():
            if k == "precond":
                o.precond_prec = _PRECONDS[v]
            elif k == "arnoldi":
                o.arnoldi = {"cgs": CGS, "cgs2": CGS2}[v]
            elif k == "use_precond":
                o.use_precond = int(bool(v))
            elif k == "matvec":
                o.matvec_prec = _MATVECS[v]
            elif k == "use_graph":
                o.use_graph = int(bool(v))
            elif k == "variant":
                o.variant = _VARIANTS[v]
            elif k == "resid":
                o.resid_prec = _RESIDS[v]
            elif k == "basis":
                o.basis_prec = _BASES[v]
            else:
                setattr(o, k, v)
        _check(self._lib.rsfde_set_opts(self._h, ctypes.byref(o)), "set_opts")

    def set_params(self, kx, ky, dt):
        _check(self._lib.rsfde_set_params(self._h, float(kx), float(ky), float(dt)), "set_params")
        self.kx, self.ky, self.dt = kx, ky, dt

    # -- calls of the C ABI --
    def apply_M(self, z, out=None):
        out = self.empty() if out is None else out
        _check(self._lib.rsfde_apply_M(self._h, _ptr(self._grid(z, "z")), _ptr(out)), "apply_M")
        return out

    def residual(self, x, b, out=None):
        """r = b - M x with M x in the solver's resid precision ("fp64" or "exact")."""
        out = self.empty() if out is None else out
        _check(self._lib.rsfde_residual(self._h, _ptr(self._grid(x, "x")), _ptr(self._grid(b, "b")),
                                        _ptr(out)), "residual")
        return out

    def apply_precond(self, v, out=None):
        out = self.empty() if out is None else out
        _check(self._lib.rsfde_apply_precond(self._h, _ptr(self._grid(v, "v")), _ptr(out)),
               "apply_precond")
        return out

    def dst2(self, v, out=None):
        out = self.empty() if out is None else out
        _check(self._lib.rsfde_dst2(self._h, _ptr(self._grid(v, "v")), _ptr(out)), "dst2")
        return out

    def rhs(self, u_prev, u_prevprev=None, src=None):
        b, x0 = self.empty(), self.empty()
        _check(self._lib.rsfde_rhs(self._h, _ptr(self._grid(u_prev, "u_prev")),
                                   _ptr(u_prevprev), _ptr(src), _ptr(b), _ptr(x0)), "rhs")
        return b, x0

    def solve(self, b, x=None, raise_on_error=True):
        """M x = b in place of x (initial guess; zeros if None).  Returns (x, stats)."""
        x = self._torch.zeros_like(b) if x is None else x
        st = _Stats()
        rc = self._lib.rsfde_solve(self._h, _ptr(self._grid(b, "b")), _ptr(self._grid(x, "x")),
                                   ctypes.byref(st))
        if raise_on_error:
            _check(rc, "solve")
        return x, st.as_dict()

    def adjoint(self, lam, mu=None):
        mu = self._torch.zeros_like(lam) if mu is None else mu
        st = _Stats()
        _check(self._lib.rsfde_adjoint(self._h, _ptr(self._grid(lam, "lam")), _ptr(mu),
                                       ctypes.byref(st)), "adjoint")
        return mu, st.as_dict()

    def step(self, u_prev, u_prevprev=None, src=None, out=None, raise_on_error=True):
        out = self.empty() if out is None else out
        st = _Stats()
        rc = self._lib.rsfde_step(self._h, _ptr(self._grid(u_prev, "u_prev")),
                                  _ptr(u_prevprev), _ptr(src), _ptr(out), ctypes.byref(st))
        if raise_on_error:
            _check(rc, "step")
        return out, st.as_dict()

    def step_host(self, u_prev, u_prevprev=None, src=None, out=None):
        """rsfde_step_host: numpy float64 arrays in and out, copies inside the call."""
        def arr(a):
            return None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        u, uu, s = arr(u_prev), arr(u_prevprev), arr(src)
        out = np.empty((self.n2, self.n1)) if out is None else out
        st = _Stats()
        p = (lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data))
        _check(self._lib.rsfde_step_host(self._h, p(u), p(uu), p(s), p(out), ctypes.byref(st)),
               "step_host")
        return out, st.as_dict()

    def march(self, u0, steps, src=None):
        """Eq. 2.17 for k = 1..steps; returns (u^steps, per-step stats)."""
        torch = self._torch
        bufs = [u0.clone(), self.empty(), self.empty()]
        prev, prevprev = 0, None
        stats = []
        for _ in range(steps):
            nxt = ({0, 1, 2} - {prev, prevprev}).pop()
            _, st = self.step(bufs[prev], None if prevprev is None else bufs[prevprev], src,
                              out=bufs[nxt])
            stats.append(st)
            prevprev, prev = prev, nxt
        return bufs[prev], stats

    def tables(self):
        lx, ly = np.empty(self.n1), np.empty(self.n2)
        tx, ty = np.empty(self.n1), np.empty(self.n2)
        p = (lambda a: ctypes.c_void_p(a.ctypes.data))
        _check(self._lib.rsfde_get_tables(self._h, p(lx), p(ly), p(tx), p(ty)), "get_tables")
        return {"lam_x": lx, "lam_y": ly, "t_x": tx, "t_y": ty}

    def params(self):
        out = np.empty(5)
        _check(self._lib.rsfde_get_params(self._h, ctypes.c_void_p(out.ctypes.data)), "params")
        return dict(zip(("cx", "cy", "pen", "hx", "hy"), out.tolist()))

    def profile(self, on=True):
        """Brackets every kernel launch with CUDA events on the solver's stream."""
        _check(self._lib.rsfde_profile_enable(self._h, int(bool(on))), "profile_enable")

    def profile_read(self):
        """{kernel class: (device ms, launches)} since the last read."""
        K = 13
        ms = np.zeros(K)
        n = np.zeros(K, dtype=np.int64)
        _check(self._lib.rsfde_profile_read(self._h, ctypes.c_void_p(ms.ctypes.data),
                                            ctypes.c_void_p(n.ctypes.data)), "profile_read")
        return {self._lib.rsfde_kernel_class_name(k).decode(): (float(ms[k]), int(n[k]))
                for k in range(K)}

    @property
    def kernel_launches(self):
        return int(self._lib.rsfde_kernel_launches(self._h))

    def set_wait_cycles(self, cycles=0):
        """Bound of each tensor-core pipeline wait in SM clock cycles (0: the default, ~2 s)."""
        _check(self._lib.rsfde_set_wait_cycles(self._h, int(cycles)), "set_wait_cycles")

    TUNE_NAMES = ("toeplitz_rows", "toeplitz_cols", "dst_rows", "dst_cols", "precond_cols", "precond_rows",
                  "gemm1_bn", "gemm2_bn", "gemm3_bn", "gemm4_bn")

    def autotune(self, reps=5):
        """Measures every feasible tile shape of this context's transform
        kernels (and the tensor-core GEMMs' tile widths) and records the
        fastest (rsfde_autotune); returns them."""
        out = np.zeros(10, dtype=np.int32)
        _check(self._lib.rsfde_autotune(self._h, int(reps), ctypes.c_void_p(out.ctypes.data)), "autotune")
        return {n: int(f) for n, f in zip(self.TUNE_NAMES, out) if f}


class Batch:
    """Many independent problems advanced together (rsfde_batch_*): each time
    step of every instance is one branch of a single CUDA graph.

    problems: list of dicts with n1, n2, box, in_omega, alpha1, alpha2, kx,
    ky, dt, eta; solver options as for Solver apply to all instances."""

    def __init__(self, problems, restart=20, max_iter=10000, tol=1e-10, precond="fp32", matvec="df32",
                 arnoldi="cgs", stream=None, resid="fp64", basis=None, use_graph=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("rsfde needs a CUDA GPU; there is no CPU path")
        self._torch = torch
        lib = load_library()
        self._lib = lib
        self.count = len(problems)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.shapes = [(int(p["n2"]), int(p["n1"])) for p in problems]
        self._masks = [torch.as_tensor(np.ascontiguousarray(p["in_omega"], dtype=np.uint8)).to(self.dev)
                       for p in problems]
        grids = (_Grid * self.count)(*[_Grid(int(p["n1"]), int(p["n2"]), *map(float, p["box"]))
                                       for p in problems])
        masks = (ctypes.c_void_p * self.count)(*[m.data_ptr() for m in self._masks])
        arr = lambda key: np.ascontiguousarray([float(p[key]) for p in problems], dtype=np.float64)
        self._params = {k: arr(k) for k in ("alpha1", "alpha2", "kx", "ky", "dt", "eta")}
        o = _Opts()
        lib.rsfde_opts_default(ctypes.byref(o))
        o.restart, o.max_iter, o.tol = int(restart), int(max_iter), float(tol)
        o.precond_prec = _PRECONDS[precond]
        o.matvec_prec = _MATVECS[matvec]
        o.arnoldi = {"cgs": CGS, "cgs2": CGS2}[arnoldi]
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        o.resid_prec = _RESIDS[resid]
        o.basis_prec = _BASES[basis if basis is not None else matvec]
        o.use_graph = int(bool(use_graph))
        h = ctypes.c_void_p()
        pp = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(lib.rsfde_batch_create(ctypes.byref(h), self.count, grids, masks,
                                      *[pp(self._params[k]) for k in ("alpha1", "alpha2", "kx", "ky",
                                                                      "dt", "eta")],
                                      ctypes.byref(o)), "batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rsfde_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, i, u0, src=None):
        u0 = self._torch.as_tensor(u0, dtype=self._torch.float64).to(self.dev).contiguous()
        s = None if src is None else self._torch.as_tensor(src, dtype=self._torch.float64).to(
            self.dev).contiguous()
        _check(self._lib.rsfde_batch_set(self._h, i, _ptr(u0), _ptr(s)), "batch_set")

    def run(self, steps):
        """Advances every instance by `steps` steps; per-instance stats of the last step."""
        st = (_Stats * self.count)()
        rc = self._lib.rsfde_batch_run(self._h, int(steps), st)
        _check(rc, "batch_run")
        return [x.as_dict() for x in st]

    def autotune(self, reps=3):
        _check(self._lib.rsfde_batch_autotune(self._h, int(reps)), "batch_autotune")

    def get(self, i):
        out = self._torch.empty(self.shapes[i], dtype=self._torch.float64, device=self.dev)
        _check(self._lib.rsfde_batch_get(self._h, i, _ptr(out)), "batch_get")
        return out

    @property
    def kernel_launches(self):
        return int(self._lib.rsfde_batch_kernel_launches(self._h))
