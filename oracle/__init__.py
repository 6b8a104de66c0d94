"""Oracle -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around oracle/rsfde_oracle.c, the plain FP64 CPU restatement
of the penalized Riesz space-fractional diffusion scheme (Section 2, Eq. 2.17),
its tau / sine-transform preconditioner (Section 4.1, Eq. 4.6) and textbook
GMRES (Section 5).  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the GPU library and its
Python binding never do.

Arrays are numpy float64, x-fastest: ``u[j, i]`` with j the y-index and i the
x-index (the ordering of u^k in Section 2), i.e. shape (n2, n1).
"""
import ctypes
import numpy as np

from .build import build_oracle

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_oracle())
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    lib.or_c_alpha.restype = d
    lib.or_c_alpha.argtypes = [d]
    lib.or_gl_weights.argtypes = [d, i, _dp]
    lib.or_diffusion_scale.restype = d
    lib.or_diffusion_scale.argtypes = [d, d, d, d]
    lib.or_toeplitz_column.argtypes = [d, d, i, _dp]
    lib.or_dst1.argtypes = [i, _dp, _dp]
    lib.or_tau_first_column.argtypes = [i, _dp, _dp]
    lib.or_tau_matrix.argtypes = [i, _dp, _dp]
    lib.or_tau_eigenvalues.argtypes = [i, _dp, _dp]
    lib.or_setup.restype = vp
    lib.or_setup.argtypes = [i, i, d, d, d, d, _u8p, d, d, d, d, d, d]
    lib.or_destroy.argtypes = [vp]
    lib.or_get_params.argtypes = [vp, _dp]
    lib.or_get_toeplitz.argtypes = [vp, _dp, _dp]
    lib.or_get_tau_eigs.argtypes = [vp, _dp, _dp]
    lib.or_apply_M.argtypes = [vp, _dp, _dp]
    lib.or_apply_M_points.argtypes = [vp, _dp, ctypes.c_long, ctypes.POINTER(ctypes.c_long), _dp]
    lib.or_dst2.argtypes = [vp, _dp, _dp]
    lib.or_dst2_rows_sample.argtypes = [vp, _dp, i, _dp]
    lib.or_dst2_cols_sample.argtypes = [vp, _dp, i, _dp]
    lib.or_apply_precond.argtypes = [vp, _dp, _dp]
    lib.or_fgmres.restype = i
    lib.or_fgmres.argtypes = [vp, _dp, _dp, i, d, i, i, _dp]
    lib.or_gmres_left.restype = i
    lib.or_gmres_left.argtypes = [vp, _dp, _dp, i, d, i, i, _dp]
    lib.or_rhs.argtypes = [vp, _dp, _dp, _dp]
    lib.or_initial_guess.argtypes = [ctypes.c_long, _dp, _dp, _dp]
    lib.or_step.restype = i
    lib.or_step.argtypes = [vp, _dp, _dp, _dp, _dp, i, d, i, _dp]
    lib.or_adjoint_march.restype = d
    lib.or_adjoint_march.argtypes = [vp, _dp, _dp, i, _dp, i, d, _dp, _dp, _dp, _dp]
    lib.or_assemble_dense.argtypes = [vp, _dp]
    lib.or_lu_solve.restype = i
    lib.or_lu_solve.argtypes = [ctypes.c_long, _dp, _dp]
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


# ---- scalar / 1-D pieces --------------------------------------------------
def c_alpha(alpha):
    """Section 1: c_alpha = -1/(2 cos(alpha pi/2))."""
    return _load().or_c_alpha(alpha)


def gl_weights(alpha, count):
    """Eq. 2.6: g_0 .. g_{count-1}."""
    g = np.empty(count)
    _load().or_gl_weights(alpha, count, _p(g))
    return g


def diffusion_scale(dt, k, alpha, h):
    """Section 2: c_x = dt k_x c_alpha / h_x^alpha."""
    return _load().or_diffusion_scale(dt, k, alpha, h)


def toeplitz_column(alpha, scale, n):
    """Eq. 2.16: first column of scale * G_n^(alpha)."""
    t = np.empty(n)
    _load().or_toeplitz_column(alpha, scale, n, _p(t))
    return t


def dst1(v):
    """Section 4.1: S_n v, O(n^2)."""
    v = _f64(v)
    out = np.empty_like(v)
    _load().or_dst1(v.size, _p(v), _p(out))
    return out


def tau_first_column(t):
    t = _f64(t)
    out = np.empty_like(t)
    _load().or_tau_first_column(t.size, _p(t), _p(out))
    return out


def tau_matrix(t):
    """Section 4.1: tau(T_n) = T_n - H_n, dense."""
    t = _f64(t)
    out = np.empty((t.size, t.size))
    _load().or_tau_matrix(t.size, _p(t), _p(out))
    return out


def tau_eigenvalues(t):
    """Section 4.1: eigenvalues of tau(T_n) via its first column."""
    t = _f64(t)
    out = np.empty_like(t)
    _load().or_tau_eigenvalues(t.size, _p(t), _p(out))
    return out


def lu_solve(A, b):
    """Textbook LU with partial pivoting (dense reference solve)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    if _load().or_lu_solve(x.size, _p(A), _p(x)) != 0:
        raise ZeroDivisionError("singular matrix")
    return x


# ---- problem context ------------------------------------------------------
class Problem:
    """One linear system M = I - A + D of Eq. 2.17 (and its tau preconditioner).

    box = (ax, bx, ay, by) is the rectangle Omega-bar; in_omega is a (n2, n1)
    0/1 array (1 inside Omega).
    """

    def __init__(self, n1, n2, box, in_omega, alpha1, alpha2, kx, ky, dt, eta):
        lib = _load()
        self.n1, self.n2 = int(n1), int(n2)
        self.N = self.n1 * self.n2
        m = np.ascontiguousarray(in_omega, dtype=np.uint8).reshape(self.n2, self.n1)
        self.in_omega = m.copy()
        ax, bx, ay, by = box
        self._h = lib.or_setup(self.n1, self.n2, ax, bx, ay, by, m.ctypes.data_as(_u8p),
                               alpha1, alpha2, kx, ky, dt, eta)
        self.alpha1, self.alpha2, self.kx, self.ky, self.dt, self.eta = (
            alpha1, alpha2, kx, ky, dt, eta)
        prm = np.empty(5)
        lib.or_get_params(self._h, _p(prm))
        self.hx, self.hy, self.cx, self.cy, self.pen = prm.tolist()

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_destroy(self._h)
            self._h = None

    def _grid(self, a):
        a = _f64(a).reshape(self.n2, self.n1)
        return a

    def toeplitz(self):
        tx, ty = np.empty(self.n1), np.empty(self.n2)
        _load().or_get_toeplitz(self._h, _p(tx), _p(ty))
        return tx, ty

    def tau_eigs(self):
        lx, ly = np.empty(self.n1), np.empty(self.n2)
        _load().or_get_tau_eigs(self._h, _p(lx), _p(ly))
        return lx, ly

    def apply_M(self, z):
        z = self._grid(z)
        w = np.empty_like(z)
        _load().or_apply_M(self._h, _p(z), _p(w))
        return w

    def apply_M_points(self, z, idx):
        """(M z) at flat indices idx only."""
        z = self._grid(z)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(idx.size)
        _load().or_apply_M_points(self._h, _p(z), idx.size,
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _p(out))
        return out

    def dst2(self, v):
        v = self._grid(v)
        w = np.empty_like(v)
        _load().or_dst2(self._h, _p(v), _p(w))
        return w

    def dst2_rows_sample(self, v, count):
        v = self._grid(v)
        out = np.zeros_like(v)
        _load().or_dst2_rows_sample(self._h, _p(v), int(count), _p(out))
        return out

    def dst2_cols_sample(self, v, count):
        v = self._grid(v)
        out = np.zeros_like(v)
        _load().or_dst2_cols_sample(self._h, _p(v), int(count), _p(out))
        return out

    def apply_precond(self, v):
        v = self._grid(v)
        z = np.empty_like(v)
        _load().or_apply_precond(self._h, _p(v), _p(z))
        return z

    def fgmres(self, b, x0=None, restart=20, tol=1e-10, max_iter=10000, precond=True):
        """Right-preconditioned FGMRES; returns (x, stats dict)."""
        b = self._grid(b)
        x = np.zeros_like(b) if x0 is None else self._grid(x0).copy()
        st = np.zeros(3)
        rc = _load().or_fgmres(self._h, _p(b), _p(x), restart, tol, max_iter, int(precond), _p(st))
        return x, {"converged": rc == 0, "iters": int(st[0]), "restarts": int(st[1]),
                   "rel_res": float(st[2])}

    def gmres_left(self, b, x0=None, restart=20, tol=1e-8, max_iter=10000, precond=True):
        """Left-preconditioned GMRES with the preconditioned stop test of Section 5."""
        b = self._grid(b)
        x = np.zeros_like(b) if x0 is None else self._grid(x0).copy()
        st = np.zeros(3)
        rc = _load().or_gmres_left(self._h, _p(b), _p(x), restart, tol, max_iter, int(precond),
                                   _p(st))
        return x, {"converged": rc == 0, "iters": int(st[0]), "restarts": int(st[1]),
                   "rel_res": float(st[2])}

    def rhs(self, u_prev, src=None):
        u = self._grid(u_prev)
        s = None if src is None else self._grid(src)
        b = np.empty_like(u)
        _load().or_rhs(self._h, _p(u), _p(s), _p(b))
        return b

    def initial_guess(self, u_prev, u_prevprev=None):
        u = self._grid(u_prev)
        uu = None if u_prevprev is None else self._grid(u_prevprev)
        x0 = np.empty_like(u)
        _load().or_initial_guess(self.N, _p(u), _p(uu), _p(x0))
        return x0

    def step(self, u_prev, u_prevprev=None, src=None, restart=20, tol=1e-10, max_iter=10000):
        """One implicit step of Eq. 2.17 with f(u) = u - u^3 (+ src)."""
        u = self._grid(u_prev)
        uu = None if u_prevprev is None else self._grid(u_prevprev)
        s = None if src is None else self._grid(src)
        out = np.empty_like(u)
        st = np.zeros(3)
        rc = _load().or_step(self._h, _p(u), _p(uu), _p(s), _p(out), restart, tol, max_iter,
                             _p(st))
        return out, {"converged": rc == 0, "iters": int(st[0]), "restarts": int(st[1]),
                     "rel_res": float(st[2])}

    def march(self, u0, steps, src=None, restart=20, tol=1e-10, max_iter=10000):
        """Eq. 2.17 for k = 1..steps; returns (u^steps, list of per-step stats)."""
        prev, prevprev = self._grid(u0).copy(), None
        stats = []
        for _ in range(steps):
            nxt, st = self.step(prev, prevprev, src, restart, tol, max_iter)
            stats.append(st)
            prevprev, prev = prev, nxt
        return prev, stats

    def adjoint_march(self, u0, steps, target, src=None, restart=20, tol=1e-13):
        """Loss ||u^steps - target||^2 of the march and its exact gradients
        (discrete adjoint): returns (loss, u_final, dL/du0, dL/ds, (dL/dkx, dL/dky))."""
        u = self._grid(u0)
        tg = self._grid(target)
        s = None if src is None else self._grid(src)
        uf, gu, gs = np.empty_like(u), np.empty_like(u), np.empty_like(u)
        gk = np.zeros(2)
        loss = _load().or_adjoint_march(self._h, _p(u), _p(s), int(steps), _p(tg), restart, tol, _p(uf),
                                         _p(gu), _p(gs), _p(gk))
        return loss, uf, gu, gs, (float(gk[0]), float(gk[1]))

    def dense_M(self):
        Md = np.empty((self.N, self.N))
        _load().or_assemble_dense(self._h, _p(Md))
        return Md
