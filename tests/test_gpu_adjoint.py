"""The GPU discrete adjoint (rsfde_adjoint_step + checkpointed march) against
the CPU oracle's adjoint and against central finite differences of the GPU
forward march, to 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2102_11576_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_11576_gb300 import Solver  # noqa: E402
from paper_2102_11576_gb300.adjoint import march  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def setup(w, **kw):
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"],
            w["dt"], w["eta"])
    return oracle.Problem(*args), Solver(*args, **kw)


def grads(solver, u0, kx, ky, src, target, steps, every=None):
    u0t = dev(u0).requires_grad_(True)
    kxt = torch.tensor(kx, dtype=torch.float64, requires_grad=True)
    kyt = torch.tensor(ky, dtype=torch.float64, requires_grad=True)
    st = dev(src).requires_grad_(True)
    uT = march(solver, u0t, kxt, kyt, st, steps=steps, every=every)
    loss = ((uT - dev(target)) ** 2).sum()
    loss.backward()
    return (loss.item(), u0t.grad.cpu().numpy(), st.grad.cpu().numpy(), kxt.grad.item(), kyt.grad.item())


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec,matvec,basis", [("fp64", "fp64", "fp64"), ("fp32", "df32", "df32"), ("bf16", "fp32", "fp32"),
                                               ("bf16x3", "fp32", "fp64")])
def test_adjoint_matches_oracle(prec, matvec, basis):
    w = workloads.random_problem(31, 20, 16)
    rng = np.random.default_rng(1)
    u0 = rng.random((16, 20)) * w["in_omega"]
    src = rng.standard_normal((16, 20))
    target = rng.random((16, 20))
    orc, gpu = setup(w, restart=12, tol=1e-13, precond=prec, matvec=matvec, basis=basis)
    steps = 6
    loss_o, _, gu_o, gs_o, (gkx_o, gky_o) = orc.adjoint_march(u0, steps, target, src=src, restart=12)
    loss, gu, gs, gkx, gky = grads(gpu, u0, w["kx"], w["ky"], src, target, steps, every=2)
    assert loss == pytest.approx(loss_o, rel=1e-9)
    assert rel(gu, gu_o) <= 1e-6
    assert rel(gs, gs_o) <= 1e-6
    assert gkx == pytest.approx(gkx_o, rel=1e-6)
    assert gky == pytest.approx(gky_o, rel=1e-6)


def test_checkpoint_interval_does_not_change_gradients():
    w = workloads.random_problem(32, 24, 18)
    rng = np.random.default_rng(2)
    u0, src, target = rng.random((18, 24)), rng.standard_normal((18, 24)), rng.random((18, 24))
    _, gpu = setup(w, restart=10, tol=1e-12)
    ref = grads(gpu, u0, w["kx"], w["ky"], src, target, 7, every=1)
    for every in (2, 3, 7):
        out = grads(gpu, u0, w["kx"], w["ky"], src, target, 7, every=every)
        for a, b in zip(out, ref):
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_adjoint_central_differences_disk1024_shape():
    """The differentiation workload's grid, domain and parameters (1024^2, unit
    disk, alpha = 1.5) over a short march: d loss / d k_x, d k_y and one u0
    and one source entry against central differences of the GPU forward."""
    w = workloads.make("disk1024")
    steps = 4
    w["dt"] = 1.0 / 200
    _, gpu = setup(w, restart=w["restart"], tol=1e-13, precond="fp32", matvec="df32")
    rng = np.random.default_rng(3)
    src = 0.1 * rng.standard_normal((w["n2"], w["n1"])) * w["in_omega"]
    loss, gu, gs, gkx, gky = grads(gpu, w["u0"], w["kx"], w["ky"], src, w["target"], steps)

    def fwd(kx, ky, u0, s):
        with torch.no_grad():
            uT = march(gpu, dev(u0), kx, ky, dev(s), steps=steps)
            return float(((uT - dev(w["target"])) ** 2).sum())

    h = 1e-4
    fd_kx = (fwd(w["kx"] + h, w["ky"], w["u0"], src) - fwd(w["kx"] - h, w["ky"], w["u0"], src)) / (2 * h)
    fd_ky = (fwd(w["kx"], w["ky"] + h, w["u0"], src) - fwd(w["kx"], w["ky"] - h, w["u0"], src)) / (2 * h)
    assert gkx == pytest.approx(fd_kx, rel=1e-6)
    assert gky == pytest.approx(fd_ky, rel=1e-6)
    j, i = 500, 520  # inside the disk
    e = np.zeros_like(src)
    e[j, i] = 1e-3
    fd_u = (fwd(w["kx"], w["ky"], w["u0"] + e, src) - fwd(w["kx"], w["ky"], w["u0"] - e, src)) / 2e-3
    fd_s = (fwd(w["kx"], w["ky"], w["u0"], src + e) - fwd(w["kx"], w["ky"], w["u0"], src - e)) / 2e-3
    assert gu[j, i] == pytest.approx(fd_u, rel=1e-6)
    assert gs[j, i] == pytest.approx(fd_s, rel=1e-6)
