"""Example 1 of Section 5 (test infrastructure only): the manufactured
solution on an ellipse, used to pin the oracle against Tables 1-3.

The printed example is garbled; this module takes the following reading
(each item below states the fix to the printed text):
  * the ellipse x^2/a^2 + y^2/b^2 <= 1 is centred in the box (-a,a) x (-b,b);
  * exact solution u_e = exp(-t) (x^2/a^2 + y^2/b^2 - 1)^2 on Omega, 0 outside;
  * the source follows from u_t = k_x R_x u + k_y R_y u + f with R the Riesz
    derivative.  Along x at fixed y the solution is a^-4 s^2 (s - 2c)^2 with
    s = x + c the distance to the left end of the chord, c = a sqrt(1-y^2/b^2)
    the half-chord; the left Riemann-Liouville derivative of s^p is
    Gamma(p+1)/Gamma(p+1-alpha) s^(p-alpha), which gives h(alpha, s, c) below
    (last power 2-alpha), and the right derivative is h at s' = c - x:
      f = -exp(-t) [k_x c_a1 a^-4 (h(a1, x+c_y, c_y) + h(a1, c_y-x, c_y))
                   + k_y c_a2 b^-4 (h(a2, y+c_x, c_x) + h(a2, c_x-y, c_x))] - u,
    where u in the last term is the numerical solution at t_{k-1} (f depends
    on u, Eq. 2.9), and f is zero outside Omega (Section 2).
"""
import math
import numpy as np

from . import Problem, c_alpha


def h_fun(alpha, s, d):
    return (24.0 * s ** (4.0 - alpha) / math.gamma(5.0 - alpha)
            - 24.0 * d * s ** (3.0 - alpha) / math.gamma(4.0 - alpha)
            + 8.0 * d * d * s ** (2.0 - alpha) / math.gamma(3.0 - alpha))


class Example1:
    def __init__(self, n, k, eta=1e-5, T=1.0, m=None, a=2.0, b=1.0, alpha1=1.4, alpha2=1.7):
        self.n, self.a, self.b = n, a, b
        self.alpha1, self.alpha2 = alpha1, alpha2
        self.k = k
        self.T = T
        self.m = n if m is None else m
        self.dt = T / self.m
        hx, hy = 2 * a / (n + 1), 2 * b / (n + 1)
        x = -a + hx * np.arange(1, n + 1)
        y = -b + hy * np.arange(1, n + 1)
        self.X, self.Y = np.meshgrid(x, y)  # shape (n2, n1), x fastest
        q = self.X ** 2 / a ** 2 + self.Y ** 2 / b ** 2
        self.inside = q <= 1.0
        self.w = np.where(self.inside, (q - 1.0) ** 2, 0.0)
        self.prob = Problem(n, n, (-a, a, -b, b), self.inside.astype(np.uint8), alpha1, alpha2,
                            k, k, self.dt, eta)
        # time-independent part of the source (the bracket of f)
        X, Y, ins = self.X, self.Y, self.inside
        cy = a * np.sqrt(np.clip(1.0 - Y ** 2 / b ** 2, 0.0, None))
        cx = b * np.sqrt(np.clip(1.0 - X ** 2 / a ** 2, 0.0, None))
        br = np.zeros_like(X)
        for jj, ii in zip(*np.nonzero(ins)):
            xx, yy, c1, c2 = X[jj, ii], Y[jj, ii], cy[jj, ii], cx[jj, ii]
            br[jj, ii] = (k * c_alpha(alpha1) * a ** -4 * (h_fun(alpha1, xx + c1, c1)
                                                          + h_fun(alpha1, c1 - xx, c1))
                          + k * c_alpha(alpha2) * b ** -4 * (h_fun(alpha2, yy + c2, c2)
                                                            + h_fun(alpha2, c2 - yy, c2)))
        self.bracket = br

    def exact(self, t):
        return math.exp(-t) * self.w

    def rhs(self, u_prev, t_prev):
        """Eq. 2.17 right side b = u^{k-1} + dt f^{k-1}, f zero outside Omega."""
        f = -math.exp(-t_prev) * self.bracket - u_prev
        return u_prev + self.dt * np.where(self.inside, f, 0.0)

    def run(self, mode="paper", precond=True, tol=None, restart=20):
        """March to T.  mode 'paper': left-preconditioned GMRES, stop test
        ||P^-1 r|| / ||P^-1 b|| < 1e-8; mode 'fgmres': right-preconditioned
        FGMRES with the true residual.  Returns (u^m, mean iterations)."""
        prev, prevprev = self.w.copy(), None
        total = 0
        for kk in range(1, self.m + 1):
            b = self.rhs(prev, (kk - 1) * self.dt)
            x0 = prev.copy() if prevprev is None else 2.0 * prev - prevprev
            if mode == "paper":
                x, st = self.prob.gmres_left(b, x0, restart, 1e-8 if tol is None else tol,
                                             precond=precond)
            else:
                x, st = self.prob.fgmres(b, x0, restart, 1e-10 if tol is None else tol,
                                         precond=precond)
            assert st["converged"], st
            total += st["iters"]
            prevprev, prev = prev, x
        return prev, total / self.m

    def error(self, u):
        """Section 5: ||u_e - u||_inf / ||u_e||_inf on Omega at t = T."""
        ue = self.exact(self.T)
        return np.abs(ue - u)[self.inside].max() / np.abs(ue)[self.inside].max()

    def outside_max(self, u):
        """Table 3: ||u_eta||_inf on the extension region."""
        return np.abs(u[~self.inside]).max()
