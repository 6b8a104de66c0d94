"""Failure detection on the GPU without a fault: the tensor-core
preconditioner's pipeline waits are bounded, and a bound small enough to run
out makes the launch give up and the call report RSFDE_ETIMEOUT, after every
copy and MMA the launch issued has completed; the context then still gives
correct results."""
import numpy as np
import pytest

import oracle
from paper_2102_11576_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_11576_gb300 import RsfdeError, Solver  # noqa: E402


@pytest.mark.parametrize("prec,tol", [("bf16x3", 2e-4), ("bf16", 2e-2)])
def test_pipeline_wait_gives_up_and_context_stays_usable(prec, tol):
    w = workloads.random_problem(21, 256, 192)
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
            w["eta"])
    ref = oracle.Problem(*args).apply_precond(w["field"])
    gpu = Solver(*args, precond=prec)
    v = torch.as_tensor(w["field"]).cuda()
    first = gpu.apply_precond(v).cpu().numpy()
    assert np.abs(first - ref).max() <= tol * np.abs(ref).max()
    gpu.set_wait_cycles(1)  # every pipeline wait that is not already satisfied gives up
    with pytest.raises(RsfdeError) as e:
        gpu.apply_precond(v)
        torch.cuda.synchronize()
    assert e.value.name == "ETIMEOUT"
    gpu.set_wait_cycles(0)  # the default bound again
    again = gpu.apply_precond(v).cpu().numpy()
    np.testing.assert_array_equal(again, first)
    # a whole solve after the give-up still meets the FP64 tolerance
    b = np.random.default_rng(2).standard_normal((192, 256))
    x, st = gpu.solve(torch.as_tensor(b).cuda())
    r = b - oracle.Problem(*args).apply_M(x.cpu().numpy())
    assert st["converged"] and np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    gpu.close()


def test_pipeline_wait_gives_up_with_two_tiles_per_cta():
    """The same at 2048 x 1232, where the split-BF16 GEMMs that follow the
    first two run one CTA per SM with two tiles each (the second tile's
    K slices streaming while the first one's epilogue runs): the give-up path
    commits the accumulators of every tile, so no epilogue wait is left
    without an arrival.  The reference result is the library's FP64 form
    (itself pinned to the oracle at the same transform lengths)."""
    w = workloads.random_problem(9, 2048, 1232)
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
            w["eta"])
    v = torch.as_tensor(w["field"]).cuda()
    f64 = Solver(*args, precond="fp64")
    ref = f64.apply_precond(v).cpu().numpy()
    f64.close()
    gpu = Solver(*args, precond="bf16x3")
    first = gpu.apply_precond(v).cpu().numpy()
    assert np.abs(first - ref).max() <= 2e-4 * np.abs(ref).max()
    gpu.set_wait_cycles(1)
    with pytest.raises(RsfdeError) as e:
        gpu.apply_precond(v)
        torch.cuda.synchronize()
    assert e.value.name == "ETIMEOUT"
    gpu.set_wait_cycles(0)
    np.testing.assert_array_equal(gpu.apply_precond(v).cpu().numpy(), first)
    gpu.close()
