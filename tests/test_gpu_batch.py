"""The batched form: instances of uneven size, alpha, k and domain advanced
together by one CUDA graph per step.  Each instance must equal the same
problem solved alone (same kernels, deterministic reductions: identical bits)
and its every step must meet the FP64 residual test, checked by the oracle."""
import numpy as np
import pytest

import oracle
from paper_2102_11576_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_11576_gb300 import Batch, Solver  # noqa: E402


# the FP32 FFT preconditioner with the FP32 operator and the FP64 residual
# (FP64 or FP32 basis), and the FP32 or split-BF16 preconditioner with the
# FP32 operator, FP64 basis and the FP64 or exact residual, run the
# multi-instance form (one launch per phase over all instances: the BF16 GEMMs
# of every instance in one grouped launch per pass, the exact residual's
# transforms and remaindering in four); the other forms the graph of
# per-instance branches
@pytest.mark.parametrize("precond,matvec,basis,resid,n_range", [
    ("fp32", "df32", "df32", "fp64", (9, 96)), ("bf16", "fp32", "fp32", "df32", (9, 96)),
    ("fp32", "fp32", "fp64", "fp64", (9, 96)), ("fp32", "fp32", "fp32", "fp64", (9, 96)),
    ("bf16x3", "fp32", "fp64", "exact", (9, 96)), ("bf16x3", "fp32", "fp64", "fp64", (9, 96)),
    ("bf16x3", "fp32", "fp64", "fp64", (100, 400)), ("fp32", "fp32", "fp64", "exact", (9, 96)),
    ("bf16x3", "fp32", "fp64", "exact", (100, 400)), ("bf16", "fp32", "fp64", "exact", (9, 96))])
def test_batch_equals_single_instances_and_meets_tolerance(precond, matvec, basis, resid, n_range):
    probs = workloads.make_batch(seed=5, count=7, n_range=n_range, steps=10)
    steps = 3
    rng = np.random.default_rng(0)
    srcs = [rng.standard_normal(p["u0"].shape) if i % 2 else None for i, p in enumerate(probs)]
    b = Batch(probs, precond=precond, matvec=matvec, resid=resid, basis=basis)
    for i, p in enumerate(probs):
        b.set(i, p["u0"], srcs[i])
    st = b.run(steps)
    assert all(s["converged"] and s["rel_res"] <= 1e-10 for s in st)
    launches = b.kernel_launches
    assert launches > 0
    if precond in ("fp32", "bf16x3") and matvec == "fp32" and resid in ("fp64", "exact"):
        # lock step: per step 6 launches (8 with the exact residual's four)
        # plus, per run of the loop body, 8 per Arnoldi column (10 with the
        # split and four grouped GEMMs) and 6 more (8), however many instances
        # there are (these problems need at most a few cycles a step)
        per_col = 10 if precond == "bf16x3" else 8
        extra = 2 if resid == "exact" else 0
        assert launches <= steps * (6 + extra + 12 * (per_col * 20 + 6 + extra))
    for i, p in enumerate(probs):
        args = (p["n1"], p["n2"], p["box"], p["in_omega"], p["alpha1"], p["alpha2"], p["kx"], p["ky"],
                p["dt"], p["eta"])
        single = Solver(*args, precond=precond, matvec=matvec, resid=resid, basis=basis)
        src = None if srcs[i] is None else torch.as_tensor(srcs[i]).cuda()
        prev, prevprev = torch.as_tensor(p["u0"]).cuda(), None
        orc = oracle.Problem(*args)
        for k in range(steps):
            nxt, s1 = single.step(prev, prevprev, src)
            bvec = orc.rhs(prev.cpu().numpy(), srcs[i])
            r = bvec - orc.apply_M(nxt.cpu().numpy())
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bvec)
            prevprev, prev = prev, nxt
        np.testing.assert_array_equal(b.get(i).cpu().numpy(), prev.cpu().numpy())
        single.close()
    # a second run continues the marches (later-step graph) and set() restarts one
    st2 = b.run(1)
    assert all(s["converged"] for s in st2)
    b.close()


def test_autotune_records_feasible_shapes_and_keeps_results():
    w = workloads.make("polygon2048", n=300)
    args = (w["n1"], w["n2"], w["box"], w["in_omega"], w["alpha1"], w["alpha2"], w["kx"], w["ky"], w["dt"],
            w["eta"])
    s = Solver(*args, precond="fp32", matvec="df32")
    u0 = torch.as_tensor(w["u0"]).cuda()
    before, st0 = s.step(u0)
    chosen = s.autotune(reps=2)
    assert set(chosen) >= {"toeplitz_rows", "toeplitz_cols", "dst_rows", "precond_cols", "precond_rows"}
    assert all(f >= 1 and (f & (f - 1)) == 0 for f in chosen.values())
    after, st1 = s.step(u0)
    assert st1["converged"]
    # each vector's transform does not depend on how many vectors a block holds
    rel = ((after - before).abs().max() / before.abs().max()).item()
    assert rel <= 1e-13
    probs = workloads.make_batch(seed=6, count=4, n_range=(40, 130), steps=10)
    b = Batch(probs)
    for i, p in enumerate(probs):
        b.set(i, p["u0"])
    b.autotune(reps=2)
    st = b.run(2)
    assert all(x["converged"] for x in st)
