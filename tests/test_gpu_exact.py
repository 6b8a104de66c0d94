"""GPU parity of the exact true residual (resid_prec RSFDE_EXACT): the
Toeplitz products of M x by number-theoretic transforms and the Chinese
remainder theorem, rounded to FP64.

r = b - M x is compared element by element with the oracle's dense FP64
sums.  The exact products' own error (the scalings of x and t to integers,
2^-54 and 2^-63 of the operand scales, and the final rounding) is far below
the oracle's own rounding in its n-term sums, so the bound is the FP64
evaluation's: 1e-14 of the Toeplitz sums' scale max|x| (1 + 2|t_x|_1 +
2|t_y|_1 + dt/eta)."""
import numpy as np
import pytest

import oracle
from paper_2102_11576_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_11576_gb300 import Solver  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def pair(w, **kw):
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
            w["dt"], w["eta"])
    return oracle.Problem(*args), Solver(*args, **kw)


def scale_of(orc, x):
    tx, ty = orc.toeplitz()
    return np.abs(x).max() * (1 + 2 * np.abs(tx).sum() + 2 * np.abs(ty).sum() + orc.pen)


# lengths L = 16 .. 8192: every radix mix of the transforms (small pass 2, 4, 8)
SIZES = [(1, 1), (2, 3), (5, 7), (9, 16), (16, 16), (17, 33), (33, 20), (64, 64), (65, 127), (200, 96),
         (257, 12), (12, 513), (2048, 24), (24, 2048), (2049, 10), (10, 2049)]


@pytest.mark.parametrize("n1,n2", SIZES)
def test_residual_exact_matches_oracle(n1, n2):
    w = workloads.random_problem(21, n1, n2)
    orc, gpu = pair(w, resid="exact")
    rng = np.random.default_rng(n1 * 7919 + n2)
    x = w["field"]
    b = rng.standard_normal((n2, n1))
    ref = b - orc.apply_M(x)
    got = host(gpu.residual(dev(x), dev(b)))
    assert np.abs(got - ref).max() <= 1e-14 * scale_of(orc, x)
    # the FP64 FFT residual agrees within its own rounding
    _, g64 = pair(w, resid="fp64")
    r64 = host(g64.residual(dev(x), dev(b)))
    assert np.abs(got - r64).max() <= 1e-13 * scale_of(orc, x)


def test_residual_exact_wide_dynamic_range():
    """Rows and columns whose entries span many binades (and exact zeros):
    each vector is scaled by its own largest exponent, so small vectors keep
    their relative accuracy."""
    w = workloads.random_problem(22, 96, 80)
    orc, gpu = pair(w, resid="exact")
    rng = np.random.default_rng(5)
    x = rng.standard_normal((80, 96)) * np.exp2(rng.integers(-40, 40, size=(80, 96)))
    x[:, 7] = 0.0
    x[11, :] = 0.0
    x[3, 3] = 1e-300
    b = np.zeros_like(x)
    got = host(gpu.residual(dev(x), dev(b)))
    ref = b - orc.apply_M(x)
    assert np.abs(got - ref).max() <= 1e-14 * scale_of(orc, x)
    # a vector scaled by 2^-600 gives the scaled products
    y = x * 2.0 ** -600
    got_y = host(gpu.residual(dev(y), dev(b)))
    np.testing.assert_allclose(got_y, got * 2.0 ** -600, rtol=0, atol=1e-14 * scale_of(orc, x) * 2.0 ** -600)


def test_residual_exact_nonfinite():
    w = workloads.random_problem(23, 40, 30)
    _, gpu = pair(w, resid="exact")
    x = w["field"].copy()
    x[4, 9] = np.nan
    r = host(gpu.residual(dev(x), dev(np.zeros_like(x))))
    assert np.isnan(r[4, :]).all() and np.isnan(r[:, 9]).all()
    assert np.isfinite(np.delete(np.delete(r, 4, axis=0), 9, axis=1)).all()


@pytest.mark.parametrize("n1,n2", [(1, 1), (5, 7), (33, 20), (65, 127)])
@pytest.mark.parametrize("prec,matvec,basis", [("fp64", "fp64", "fp64"), ("bf16x3", "fp32", "fp64"),
                                               ("fp32", "fp32", "fp64"), ("fp32", "fp32", "fp32")])
def test_solve_exact_residual_matches_oracle(n1, n2, prec, matvec, basis):
    w = workloads.random_problem(24, n1, n2)
    orc, gpu = pair(w, precond=prec, tol=1e-11, restart=10, matvec=matvec, basis=basis, resid="exact")
    b = np.random.default_rng(1).standard_normal((n2, n1))
    x_ref, _ = orc.fgmres(b, restart=10, tol=1e-12)
    x, st = gpu.solve(dev(b))
    x = host(x)
    assert st["converged"] and st["rel_res"] <= 1e-11
    r = b - orc.apply_M(x)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b) * 1.01
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-9


def test_exact_graph_equals_direct_and_paper_mode():
    w = workloads.random_problem(25, 70, 46)
    b = dev(np.random.default_rng(3).standard_normal((46, 70)))
    res = []
    for use_graph in (True, False):
        _, gpu = pair(w, precond="bf16x3", matvec="fp32", restart=6, tol=1e-12, use_graph=use_graph,
                      resid="exact")
        for _ in range(2):
            x, st = gpu.solve(b)
        res.append((host(x), st))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1]["iters"] == res[1][1]["iters"] and res[0][1]["restarts"] > 0
    # left-preconditioned GMRES (paper mode) with the exact residual: the same
    # iteration count as with the FP64 residual
    its = []
    for resid in ("fp64", "exact"):
        _, gpu = pair(w, variant="gmres_left", restart=20, tol=1e-10, resid=resid)
        x, st = gpu.solve(b)
        assert st["converged"]
        its.append(st["iters"])
    assert abs(its[0] - its[1]) <= 1
