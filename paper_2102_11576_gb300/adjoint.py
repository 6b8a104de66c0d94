"""Gradients of the time march through the library's discrete adjoint.

``march(solver, u0, kx, ky, src, steps)`` runs Eq. 2.17 for ``steps`` implicit
steps on the GPU and is differentiable (torch.autograd) with respect to u0,
k_x, k_y and the per-cell source s.  The backward pass is hand-written: for
k = m..1 it calls ``rsfde_adjoint_step`` (solve M mu = lambda with the same
preconditioned FGMRES -- M is symmetric by Lemma 2.3 -- then the
elementwise lambda^{k-1}, source and k-gradient kernels).  Forward states are
not all kept: every ``every`` steps (default ceil(sqrt(m))) a checkpoint
pair (u^k, u^{k-1}) is stored, and the backward pass recomputes one segment
at a time from its checkpoint.  The pair reproduces the initial guess of the
recomputed steps, and the reductions are deterministic, so recomputed states
equal the original ones bit for bit.

Everything here is orchestration of C-ABI calls; the arithmetic runs in the
library's kernels.
"""
import ctypes
import math

import torch

from . import RsfdeError, Solver, _check, _ptr, _Stats


def _adjoint_step(solver, u_prev, u_k, lam, mu, lam_prev, grad_src, grad_k):
    st = _Stats()
    lib = solver._lib
    fn = lib.rsfde_adjoint_step
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 8 + [ctypes.POINTER(_Stats)]
    _check(fn(solver._h, _ptr(u_prev), _ptr(u_k), _ptr(lam), _ptr(mu), _ptr(lam_prev), _ptr(grad_src),
              _ptr(grad_k), ctypes.byref(st)), "adjoint_step")
    return st.as_dict()


class _March(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kx, ky, src, solver, steps, every):
        solver.set_params(float(kx), float(ky), solver.dt)
        u0 = u0.detach().contiguous()
        s = None if src is None else src.detach().contiguous()
        checkpoints = {0: (u0.clone(), None)}
        prev, prevprev = u0.clone(), None
        for k in range(1, steps + 1):
            nxt, _ = solver.step(prev, prevprev, s)
            if k % every == 0 and k < steps:
                checkpoints[k] = (nxt.clone(), prev.clone())
            prevprev, prev = prev, nxt
        ctx.solver, ctx.steps, ctx.every = solver, steps, every
        ctx.checkpoints, ctx.src = checkpoints, s
        ctx.kxky = (float(kx), float(ky))
        ctx.kdev = (kx.device, ky.device)
        ctx.has_src = src is not None
        return prev

    @staticmethod
    def backward(ctx, grad_out):
        solver, steps, every = ctx.solver, ctx.steps, ctx.every
        solver.set_params(ctx.kxky[0], ctx.kxky[1], solver.dt)
        lam = grad_out.detach().contiguous().clone()
        mu = torch.zeros_like(lam)
        grad_k = torch.zeros(2, dtype=torch.float64, device=lam.device)
        grad_src = torch.zeros_like(lam) if ctx.has_src else None
        starts = sorted(ctx.checkpoints)
        for k0 in reversed(starts):
            k1 = min(k0 + every, steps)
            # recompute u^{k0..k1} from the checkpoint pair
            u_k0, u_km1 = ctx.checkpoints[k0]
            states = [u_k0]
            prev, prevprev = u_k0, u_km1
            for _ in range(k0 + 1, k1 + 1):
                nxt, _ = solver.step(prev, prevprev, ctx.src)
                states.append(nxt)
                prevprev, prev = prev, nxt
            for k in range(k1, k0, -1):
                _adjoint_step(solver, states[k - 1 - k0], states[k - k0], lam, mu, lam, grad_src, grad_k)
        gkx, gky = grad_k[0].to(ctx.kdev[0]), grad_k[1].to(ctx.kdev[1])
        return lam, gkx, gky, grad_src, None, None, None


def march(solver: Solver, u0, kx, ky, src=None, steps=1, every=None):
    """Differentiable march of ``steps`` implicit steps (see module doc).

    u0, src: float64 CUDA tensors of shape (n2, n1); kx, ky: float64 tensors
    (0-d, on any device).  The solver's grid, mask, alphas, dt and eta define
    the problem; its k_x, k_y are set from kx, ky."""
    if every is None:
        every = max(1, math.ceil(math.sqrt(steps)))
    kx = kx if isinstance(kx, torch.Tensor) else torch.tensor(float(kx), dtype=torch.float64)
    ky = ky if isinstance(ky, torch.Tensor) else torch.tensor(float(ky), dtype=torch.float64)
    return _March.apply(u0, kx, ky, src, solver, int(steps), int(every))


__all__ = ["march", "RsfdeError"]
