"""Seeded synthetic inputs shaped like the paper's experiments.

Geometry (the domain mask), initial fields and sources only -- none of the
method's arithmetic.  Both the GPU tests / benchmark and the CPU oracle take
their inputs from here, as plain numpy arrays (mask uint8, fields float64,
shape (n2, n1), x fastest).  Randomness comes from numpy's PCG64
(``default_rng(seed)``).

Recipes (each a problem of Section 2 on the box [-1,1]^2, interior grid
points x_i = -1 + i h, h = 2/(n+1)):
  * disk64:     n=64, Omega the unit disk, alpha=(1.5,1.7), k=(1,1), eta=1e-8,
                u0=(1-x^2-y^2)_+^2, T=1 in 64 steps, FGMRES(20), tol 1e-10.
  * ellipse512: n=512, Omega x^2/0.9^2 + y^2/0.6^2 <= 1, alpha=(1.2,1.8),
                k=(2,0.5), source a Gaussian bump (sigma 0.15) at a seeded
                centre, u0=(1 - x^2/0.81 - y^2/0.36)_+^2, T=1 in 100 steps,
                FGMRES(30), tol 1e-10.
  * polygon2048: n=2048, Omega a convex 12-gon with seeded vertices on the
                unit circle, alpha=(1.3,1.6), k=(1,1), u0 the masked
                (1-x^2-y^2)_+^2, T=1 in 50 steps, FGMRES(20), tol 1e-10.
  * disk1024:   n=1024, unit disk, alpha=(1.5,1.5), T=1 in 200 steps, and a
                seeded smooth target (sum of 4 Gaussians) for the adjoint loss.
  * make_batch: 256 independent instances of uneven size and parameters.
"""
import numpy as np

BOX = (-1.0, 1.0, -1.0, 1.0)


def grid_xy(n1, n2, box=BOX):
    ax, bx, ay, by = box
    x = ax + (bx - ax) / (n1 + 1) * np.arange(1, n1 + 1)
    y = ay + (by - ay) / (n2 + 1) * np.arange(1, n2 + 1)
    return np.meshgrid(x, y)  # (n2, n1)


def ellipse_mask(X, Y, a, b, cx=0.0, cy=0.0, rot=0.0):
    c, s = np.cos(rot), np.sin(rot)
    xr = c * (X - cx) + s * (Y - cy)
    yr = -s * (X - cx) + c * (Y - cy)
    return ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0).astype(np.uint8)


def polygon_vertices(rng, k):
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=k))
    return np.stack([np.cos(ang), np.sin(ang)], axis=1)


def convex_polygon_mask(X, Y, verts):
    """Closed convex polygon with counter-clockwise vertices: inside iff on the
    left of (or on) every edge."""
    inside = np.ones(X.shape, dtype=bool)
    k = len(verts)
    for e in range(k):
        x0, y0 = verts[e]
        x1, y1 = verts[(e + 1) % k]
        cross = (x1 - x0) * (Y - y0) - (y1 - y0) * (X - x0)
        inside &= cross >= 0.0
    return inside.astype(np.uint8)


def bump(X, Y, a=1.0, b=1.0):
    return np.clip(1.0 - X ** 2 / a ** 2 - Y ** 2 / b ** 2, 0.0, None) ** 2


def gaussian(X, Y, x0, y0, sigma):
    return np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * sigma ** 2))


def make(name, seed=0, n=None):
    """Returns a dict describing one workload (all arrays numpy)."""
    rng = np.random.default_rng(seed)
    if name == "disk64":
        n = n or 64
        X, Y = grid_xy(n, n)
        mask = ellipse_mask(X, Y, 1.0, 1.0)
        w = dict(alpha1=1.5, alpha2=1.7, kx=1.0, ky=1.0, eta=1e-8, T=1.0, steps=64, restart=20,
                 u0=bump(X, Y) * mask, src=None)
    elif name == "ellipse512":
        n = n or 512
        X, Y = grid_xy(n, n)
        mask = ellipse_mask(X, Y, 0.9, 0.6)
        p0 = rng.uniform([-0.45, -0.3], [0.45, 0.3])
        w = dict(alpha1=1.2, alpha2=1.8, kx=2.0, ky=0.5, eta=1e-8, T=1.0, steps=100, restart=30,
                 u0=bump(X, Y, 0.9, 0.6) * mask, src=gaussian(X, Y, p0[0], p0[1], 0.15))
    elif name == "polygon2048":
        n = n or 2048
        X, Y = grid_xy(n, n)
        mask = convex_polygon_mask(X, Y, polygon_vertices(rng, 12))
        w = dict(alpha1=1.3, alpha2=1.6, kx=1.0, ky=1.0, eta=1e-8, T=1.0, steps=50, restart=20,
                 u0=bump(X, Y) * mask, src=None,
                 # mean FGMRES(20) iterations per step of the FP64 form over the
                 # default timed region of the benchmark (steps 4-13 of the march
                 # from the bump), used to scale the CPU oracle's sampled
                 # per-iteration time (FP64 arithmetic) to steps/s
                 iters_per_step_recorded=59.4)
    elif name == "disk1024":
        n = n or 1024
        X, Y = grid_xy(n, n)
        mask = ellipse_mask(X, Y, 1.0, 1.0)
        tgt = np.zeros_like(X)
        for _ in range(4):
            x0, y0 = rng.uniform(-0.5, 0.5, size=2)
            tgt += gaussian(X, Y, x0, y0, rng.uniform(0.1, 0.3))
        w = dict(alpha1=1.5, alpha2=1.5, kx=1.0, ky=1.0, eta=1e-8, T=1.0, steps=200, restart=20,
                 u0=bump(X, Y) * mask, src=None, target=tgt * mask)
    else:
        raise KeyError(name)
    w.update(name=name, n1=n, n2=n, box=BOX, in_omega=mask, tol=1e-10)
    w["dt"] = w["T"] / w["steps"]
    return w


def make_batch(seed=0, count=256, n_range=(64, 512), steps=20):
    """The batched workload: `count` independent instances, grid side
    uniform in n_range, alpha1, alpha2 ~ U(1.1, 1.9), k_x, k_y ~ U[0.5, 2],
    Omega a random ellipse (semi-axes U[0.4, 0.95], centre offset
    U[-0.05, 0.05]^2, random rotation) or a convex polygon with 5-12 vertices
    on the unit circle (equal odds), u0 the masked bump, T = 1 in `steps`
    steps, eta = 1e-8."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        X, Y = grid_xy(n, n)
        if rng.random() < 0.5:
            a, b = rng.uniform(0.4, 0.95, size=2)
            cx, cy = rng.uniform(-0.05, 0.05, size=2)
            mask = ellipse_mask(X, Y, a, b, cx, cy, rng.uniform(0.0, np.pi))
        else:
            mask = convex_polygon_mask(X, Y, polygon_vertices(rng, int(rng.integers(5, 13))))
        out.append(dict(n1=n, n2=n, box=BOX, in_omega=mask, alpha1=float(rng.uniform(1.1, 1.9)),
                        alpha2=float(rng.uniform(1.1, 1.9)), kx=float(rng.uniform(0.5, 2.0)),
                        ky=float(rng.uniform(0.5, 2.0)), eta=1e-8, T=1.0, steps=steps, dt=1.0 / steps,
                        u0=bump(X, Y) * mask, tol=1e-10, restart=20))
    return out


def random_problem(seed, n1, n2, p_in=0.6):
    """A small random problem for parity tests: random mask and parameters."""
    rng = np.random.default_rng(seed)
    X, Y = grid_xy(n1, n2)
    mask = (rng.random((n2, n1)) < p_in).astype(np.uint8)
    return dict(n1=n1, n2=n2, box=BOX, in_omega=mask, alpha1=float(rng.uniform(1.1, 1.9)),
                alpha2=float(rng.uniform(1.1, 1.9)), kx=float(rng.uniform(0.5, 2.0)),
                ky=float(rng.uniform(0.5, 2.0)), dt=float(rng.uniform(0.01, 0.1)),
                eta=float(10.0 ** rng.uniform(-8, -3)), field=rng.standard_normal((n2, n1)))
