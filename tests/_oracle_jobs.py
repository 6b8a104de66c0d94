"""Oracle computations run in spawned worker processes by the full-size GPU
parity test, so that the slow single-threaded oracle works while the GPU
does.  Imports only numpy and the oracle (no torch, no CUDA)."""
import oracle


def _problem(args):
    return oracle.Problem(*args)


def apply_precond(args, v):
    return _problem(args).apply_precond(v)


def apply_M(args, x):
    return _problem(args).apply_M(x)


def rhs(args, u):
    return _problem(args).rhs(u)
