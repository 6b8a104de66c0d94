"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 path): operator and transform outputs agree to 1e-12 of the
output's max norm (the FFT evaluation differs from the oracle's dense sums by
O(eps log L) of the operand norm); solves reach a true relative residual
<= 1e-10 and the solution differs from the oracle's by <= 1e-9 in relative
max norm.  FP32 preconditioner: the apply agrees to 1e-5 relative (FP32 FFTs),
while the solve still reaches the FP64 tolerance.  Split-BF16 tensor-core
preconditioner (about 16 significant bits per operand, FP32 accumulation over
up to n terms per pass, four passes): 2e-4 relative.  Double-FP32 operator
(~48-bit arithmetic): 2e-12 of the Toeplitz sums' scale; solves with it still
reach the FP64 tolerances because the true residual is FP64.
"""
import numpy as np
import pytest

import oracle
from paper_2102_11576_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_11576_gb300 import Solver, RsfdeError  # noqa: E402

SIZES = [(1, 1), (2, 3), (5, 7), (16, 16), (33, 20), (64, 64), (65, 127), (200, 96)]


def pair(w, **kw):
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
            w["dt"], w["eta"])
    return oracle.Problem(*args), Solver(*args, **kw)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n1,n2", SIZES)
def test_tables_match_oracle(n1, n2):
    w = workloads.random_problem(1, n1, n2)
    orc, gpu = pair(w)
    t = gpu.tables()
    tx, ty = orc.toeplitz()
    lx, ly = orc.tau_eigs()
    np.testing.assert_allclose(t["t_x"], tx, rtol=1e-14, atol=0)
    np.testing.assert_allclose(t["t_y"], ty, rtol=1e-14, atol=0)
    np.testing.assert_allclose(t["lam_x"], lx, rtol=1e-11, atol=1e-12 * np.abs(lx).max())
    np.testing.assert_allclose(t["lam_y"], ly, rtol=1e-11, atol=1e-12 * np.abs(ly).max())
    p = gpu.params()
    assert p["cx"] == pytest.approx(orc.cx, rel=1e-14) and p["pen"] == pytest.approx(orc.pen)


@pytest.mark.parametrize("n1,n2", SIZES)
@pytest.mark.parametrize("matvec,tol", [("fp64", 1e-13), ("df32", 2e-12), ("fp32", 2e-6)])
def test_apply_M(n1, n2, matvec, tol):
    w = workloads.random_problem(2, n1, n2)
    orc, gpu = pair(w, matvec=matvec)
    z = w["field"]
    ref = orc.apply_M(z)
    got = host(gpu.apply_M(dev(z)))
    # scale: the Toeplitz sums, not the (possibly cancelling) result
    scale = (np.abs(z).max() * (1 + np.abs(orc.toeplitz()[0]).sum() * 2 + np.abs(orc.toeplitz()[1]).sum() * 2
                                + orc.pen))
    assert np.abs(got - ref).max() <= tol * scale


@pytest.mark.parametrize("n1,n2", SIZES)
def test_dst2(n1, n2):
    w = workloads.random_problem(3, n1, n2)
    orc, gpu = pair(w)
    v = w["field"]
    ref = orc.dst2(v)
    got = host(gpu.dst2(dev(v)))
    assert rel(got, ref) <= 1e-12
    # involution S^2 = I on the GPU alone
    back = host(gpu.dst2(dev(got)))
    assert rel(back, v) <= 1e-12


@pytest.mark.parametrize("n1,n2", SIZES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5), ("bf16x3", 2e-4), ("bf16", 2e-2)])
def test_apply_precond(n1, n2, prec, tol):
    w = workloads.random_problem(4, n1, n2)
    orc, gpu = pair(w, precond=prec)
    v = w["field"]
    ref = orc.apply_precond(v)
    got = host(gpu.apply_precond(dev(v)))
    assert rel(got, ref) <= tol


# (operator arithmetic, Krylov basis and Gram-Schmidt, true residual's M x)
FORMS = [("fp64", "fp64", "fp64"), ("df32", "fp64", "fp64"), ("fp32", "fp64", "fp64"), ("df32", "df32", "fp64"),
         ("fp32", "fp32", "fp64"), ("fp32", "fp32", "df32"), ("df32", "df32", "df32")]


@pytest.mark.parametrize("n1,n2", [(1, 1), (5, 7), (33, 20), (64, 64), (65, 127)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16"])
@pytest.mark.parametrize("arnoldi", ["cgs", "cgs2"])
@pytest.mark.parametrize("matvec,basis,resid", FORMS)
def test_solve_matches_oracle(n1, n2, prec, arnoldi, matvec, basis, resid):
    w = workloads.random_problem(5, n1, n2)
    orc, gpu = pair(w, precond=prec, arnoldi=arnoldi, tol=1e-11, restart=10, matvec=matvec, resid=resid,
                    basis=basis)
    rng = np.random.default_rng(0)
    b = rng.standard_normal((n2, n1))
    x_ref, st_ref = orc.fgmres(b, restart=10, tol=1e-12)
    x, st = gpu.solve(dev(b))
    x = host(x)
    assert st["converged"] and st["rel_res"] <= 1e-11
    r = b - orc.apply_M(x)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b) * 1.01
    # Lemma 3.1 + Lemma 2.3: ||M^-1||_inf <= 1
    assert np.abs(x - x_ref).max() <= np.abs(r).max() + np.abs(b - orc.apply_M(x_ref)).max() + 1e-15
    assert rel(x, x_ref) <= 1e-9


@pytest.mark.parametrize("prec,matvec,basis,resid", [("fp64", "fp64", "fp64", "fp64"), ("fp32", "df32", "df32", "fp64"),
                                                     ("fp32", "fp32", "fp32", "fp64"), ("bf16", "fp32", "fp32", "df32"),
                                                     ("bf16x3", "fp32", "fp64", "fp64"),
                                                     ("bf16", "df32", "fp64", "fp64")])
def test_graph_loop_equals_direct_launches(prec, matvec, basis, resid):
    """The device-side graph loop and the host-driven loop run the same
    kernels in the same order with deterministic reductions: identical bits."""
    w = workloads.random_problem(8, 70, 46)
    rng = np.random.default_rng(3)
    b = dev(rng.standard_normal((46, 70)))
    res = []
    for use_graph in (True, False):
        _, gpu = pair(w, precond=prec, matvec=matvec, restart=6, tol=1e-12, use_graph=use_graph, resid=resid,
                      basis=basis)
        for _ in range(2):  # the second solve replays the captured graph
            x, st = gpu.solve(b)
        res.append((host(x), st))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1]["iters"] == res[1][1]["iters"] and res[0][1]["restarts"] == res[1][1]["restarts"] > 0


def test_unpreconditioned_and_dense_lu():
    w = workloads.random_problem(6, 9, 8)
    orc, gpu = pair(w, use_precond=False, tol=1e-12, restart=30)
    b = np.random.default_rng(1).standard_normal((8, 9))
    x, st = gpu.solve(dev(b))
    x_lu = oracle.lu_solve(orc.dense_M(), b.reshape(-1)).reshape(8, 9)
    assert st["converged"] and rel(host(x), x_lu) <= 1e-9


@pytest.mark.parametrize("prec,matvec,basis,resid", [("fp64", "fp64", "fp64", "fp64"), ("fp32", "df32", "df32", "fp64"),
                                                     ("bf16x3", "df32", "df32", "fp64"),
                                                     ("fp32", "fp32", "fp32", "fp64"),
                                                     ("bf16x3", "fp32", "fp32", "fp64"),
                                                     ("bf16", "fp32", "fp32", "df32"),
                                                     ("bf16x3", "fp32", "fp64", "fp64"),
                                                     ("fp32", "fp32", "fp64", "fp64")])
def test_march_disk64_matches_oracle(prec, matvec, basis, resid):
    w = workloads.make("disk64")
    orc, gpu = pair(w, tol=1e-12, restart=w["restart"], precond=prec, matvec=matvec, resid=resid, basis=basis)
    steps = 16
    u_ref, st_ref = orc.march(w["u0"], steps, restart=w["restart"], tol=1e-12)
    u, st = gpu.march(dev(w["u0"]), steps)
    u = host(u)
    assert all(s["converged"] for s in st)
    assert rel(u, u_ref) <= 1e-9
    it_gpu = np.mean([s["iters"] for s in st])
    it_ref = np.mean([s["iters"] for s in st_ref])
    if matvec == "fp32":
        # an FP32 Arnoldi operator bounds each restart cycle's residual reduction
        # near its rounding level: at this 1e-12 tolerance it takes extra cycles
        assert it_ref <= it_gpu + 1 and it_gpu <= 1.5 * it_ref + 1
    else:
        assert abs(it_gpu - it_ref) <= 0.1 * it_ref + 1  # same method, different Gram-Schmidt


def test_step_host_equals_step():
    w = workloads.make("disk64", n=48)
    _, gpu = pair(w)
    u0 = w["u0"]
    d, _ = gpu.step(dev(u0))
    h, _ = gpu.step_host(u0)
    np.testing.assert_array_equal(host(d), h)


def test_rhs_and_guess():
    w = workloads.make("ellipse512", n=40)
    orc, gpu = pair(w)
    rng = np.random.default_rng(2)
    u, uu = rng.standard_normal((40, 40)), rng.standard_normal((40, 40))
    b, x0 = gpu.rhs(dev(u), dev(uu), dev(w["src"]))
    np.testing.assert_allclose(host(b), orc.rhs(u, w["src"]), rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(host(x0), orc.initial_guess(u, uu), rtol=0, atol=0)


def test_edge_cases():
    w = workloads.random_problem(7, 12, 10)
    orc, gpu = pair(w)
    # b = 0 gives x = 0 in zero iterations
    x, st = gpu.solve(dev(np.zeros((10, 12))), dev(np.ones((10, 12))))
    assert st["converged"] and st["iters"] == 0 and np.all(host(x) == 0)
    # exact initial guess: no iteration
    xs = np.random.default_rng(3).standard_normal((10, 12))
    x, st = gpu.solve(dev(orc.apply_M(xs)), dev(xs))
    assert st["converged"] and st["iters"] == 0
    # NaN in the right side
    b = np.ones((10, 12))
    b[3, 4] = np.nan
    with pytest.raises(RsfdeError) as e:
        gpu.solve(dev(b))
    assert e.value.name == "ENONFINITE"
    # max_iter too small
    g2 = Solver(12, 10, w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
                w["eta"], max_iter=1, tol=1e-14)
    with pytest.raises(RsfdeError) as e:
        g2.solve(dev(np.random.default_rng(4).standard_normal((10, 12))))
    assert e.value.name == "ENOTCONV"
    # invalid arguments
    with pytest.raises(RsfdeError) as e:
        Solver(12, 10, w["box"], w["in_omega"], 2.5, 1.5, 1, 1, 0.1, 1e-3)
    assert e.value.name == "EINVAL"
    # all-inside and all-outside masks
    for val in (0, 1):
        w2 = dict(w, in_omega=np.full((10, 12), val, np.uint8))
        orc2, gpu2 = pair(w2, tol=1e-12)
        b = np.random.default_rng(5).standard_normal((10, 12))
        x, st = gpu2.solve(dev(b))
        x = host(x)
        assert st["converged"]
        assert np.linalg.norm(b - orc2.apply_M(x)) <= 1.01e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("n1,n2", [(2048, 40), (40, 2048), (2049, 24), (24, 2049)])
def test_full_length_transforms_elementwise(n1, n2):
    """The transforms at the full workload's lengths, element by element
    against the oracle: n = 2048 (GEMM K of 2048 through the TMA ring, the
    symmetric form, the FFT length 4096) and n = 2049 (odd: the natural GEMM
    layout, the FFT length 8192), along x and along y."""
    w = workloads.random_problem(9, n1, n2)
    orc = oracle.Problem(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
                         w["dt"], w["eta"])
    v = w["field"]
    ref = orc.apply_precond(v)
    for prec, tol in (("fp64", 1e-11), ("fp32", 2e-5), ("bf16x3", 2e-4), ("bf16", 2e-2)):
        gpu = Solver(w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
                     w["dt"], w["eta"], precond=prec, matvec="fp32" if prec != "fp64" else "fp64")
        assert rel(host(gpu.apply_precond(dev(v))), ref) <= tol, prec
        if prec == "fp64":
            assert rel(host(gpu.dst2(dev(v))), orc.dst2(v)) <= 1e-12
        else:
            z = rng_field(n2, n1)
            scale = np.abs(z).max() * (1 + 2 * np.abs(orc.toeplitz()[0]).sum() + 2 * np.abs(orc.toeplitz()[1]).sum()
                                       + orc.pen)
            assert np.abs(host(gpu.apply_M(dev(z))) - orc.apply_M(z)).max() <= 2e-6 * scale
        gpu.close()


def rng_field(n2, n1, seed=12):
    return np.random.default_rng(seed).standard_normal((n2, n1))


@pytest.mark.slow
def test_full_size_polygon2048_against_oracle():
    """The benchmark's 2048^2 workload at its launch configuration.
    (a) P-hat^-1 v in every precision against one full oracle P-hat^-1 v,
    element by element; (b) one step of the headline form (split-BF16
    preconditioner, FP32 operator arithmetic, FP64 basis, Gram-Schmidt,
    Givens and true residual, the residual's Toeplitz products exact) and of the FP64 form: the oracle's full-grid
    M x gives the true relative residual (<= 1e-10), and Lemma 3.1 with
    Lemma 2.3 (||M^-1||_inf <= 1) bounds the two solutions' difference by
    their residuals.  (c) P-hat^-1 v at 2048 x 1232 in the split-BF16 and FP32
    forms: between one and two waves of GEMM tiles (two tiles per CTA), with
    ragged last tiles in both GEMM dimensions.  The oracle runs in spawned
    processes while the GPU works."""
    import multiprocessing as mp
    import _oracle_jobs
    w = workloads.make("polygon2048")
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
            w["eta"])
    v = rng_field(w["n2"], w["n1"], seed=13)
    w2 = workloads.random_problem(9, 2048, 1232)
    args2 = (w2["n1"], w2["n2"], w2["box"], w2["in_omega"], w2["alpha1"], w2["alpha2"], w2["kx"], w2["ky"],
             w2["dt"], w2["eta"])
    v2 = w2["field"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(4) as pool:
        job_p = pool.apply_async(_oracle_jobs.apply_precond, (args, v))
        job_p2 = pool.apply_async(_oracle_jobs.apply_precond, (args2, v2))
        job_b = pool.apply_async(_oracle_jobs.rhs, (args, w["u0"]))
        got = {}
        for prec in ("fp64", "fp32", "bf16x3", "bf16"):
            gpu = Solver(*args, restart=w["restart"], precond=prec)
            got[prec] = host(gpu.apply_precond(dev(v)))
            gpu.close()
        got2 = {}
        for prec in ("fp32", "bf16x3"):
            gpu = Solver(*args2, precond=prec)
            got2[prec] = host(gpu.apply_precond(dev(v2)))
            gpu.close()
        steps = {}
        for name, kw in (("headline", dict(precond="bf16x3", matvec="fp32", basis="fp64", resid="exact")),
                         ("fp64", dict(precond="fp64", matvec="fp64", basis="fp64", resid="fp64"))):
            gpu = Solver(*args, restart=w["restart"], tol=w["tol"], **kw)
            u1, st = gpu.step(dev(w["u0"]))
            assert st["converged"] and st["rel_res"] <= 1e-10, (name, st)
            steps[name] = host(u1)
            gpu.close()
        jobs_m = {k: pool.apply_async(_oracle_jobs.apply_M, (args, x)) for k, x in steps.items()}
        ref = job_p.get()
        ref2 = job_p2.get()
        b = job_b.get()
        mx = {k: j.get() for k, j in jobs_m.items()}
    for prec, tol in (("fp64", 1e-11), ("fp32", 2e-5), ("bf16x3", 2e-4), ("bf16", 2e-2)):
        assert rel(got[prec], ref) <= tol, (prec, rel(got[prec], ref))
    for prec, tol in (("fp32", 2e-5), ("bf16x3", 2e-4)):
        assert rel(got2[prec], ref2) <= tol, (prec, rel(got2[prec], ref2))
    r = {k: b - mx[k] for k in steps}
    for k in steps:
        assert np.linalg.norm(r[k]) <= 1.01e-10 * np.linalg.norm(b), k
    diff = np.abs(steps["headline"] - steps["fp64"]).max()
    assert diff <= np.abs(r["headline"]).max() + np.abs(r["fp64"]).max() + 1e-15
    assert diff / np.abs(steps["fp64"]).max() <= 1e-9


def test_ellipse512_march_with_source():
    """The 512^2 ellipse workload (alpha = (1.2, 1.8), k = (2, 0.5), Gaussian
    source, FGMRES(30)): four steps in the mixed form; every step's true
    residual recomputed by the oracle, and the solution within the bound
    ||x - x*||_inf <= ||r||_inf that Lemma 3.1 with Lemma 2.3 gives."""
    w = workloads.make("ellipse512")
    orc, gpu = pair(w, restart=w["restart"], tol=w["tol"], precond="fp32", matvec="df32")
    _, g64 = pair(w, restart=w["restart"], tol=1e-13, precond="fp64", matvec="fp64")
    src = dev(w["src"])
    prev, prevprev = dev(w["u0"]), None
    for k in range(4):
        nxt, st = gpu.step(prev, prevprev, src)
        assert st["converged"] and st["rel_res"] <= 1e-10
        b = orc.rhs(host(prev), w["src"])
        x0 = orc.initial_guess(host(prev), None if prevprev is None else host(prevprev))
        r = b - orc.apply_M(host(nxt))
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * 1.01
        # a tighter FP64 solve from the same data: within the Lemma 3.1 bound
        ref, _ = g64.solve(dev(b), dev(x0))
        diff = np.abs(host(nxt) - host(ref)).max()
        assert diff <= np.abs(r).max() + np.abs(b - orc.apply_M(host(ref))).max() + 1e-15
        assert diff / np.abs(host(ref)).max() <= 1e-9
        prevprev, prev = prev, nxt


def test_resume_from_saved_state_reproduces_the_march():
    """Checkpoint and resume: the march's state is the pair (u^{k-1}, u^{k-2})
    (the extrapolated guess needs both, Section 5).  A fresh context started
    from a pair saved after step 3 reproduces steps 4-6 of the uninterrupted
    march bit for bit (the kernels and reductions are deterministic)."""
    w = workloads.random_problem(31, 60, 44)
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
            w["dt"], w["eta"])
    kw = dict(precond="bf16x3", matvec="fp32", basis="fp64", resid="exact", restart=10, tol=1e-11)
    a = Solver(*args, **kw)
    prev, pp = dev(np.abs(w["field"])), None
    saved = []
    for _ in range(6):
        nxt, st = a.step(prev, pp)
        assert st["converged"]
        pp, prev = prev, nxt.clone()
        saved.append((prev.clone(), pp.clone()))
    a.close()
    b = Solver(*args, **kw)
    prev, pp = saved[2]
    for k in range(3, 6):
        nxt, st = b.step(prev, pp)
        pp, prev = prev, nxt.clone()
        assert torch.equal(prev, saved[k][0]), k
    b.close()
