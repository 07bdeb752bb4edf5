"""A second, deliberately different FP64 formulation of the D2Q37 step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  It exists to
brute-force check the C oracle on tiny lattices, so it shares none of the C
oracle's code paths:

  * no halo frame: periodic x (and y with ``periodic_y``) by modular indexing
    with ``np.roll``; with walls the pull from beyond a wall yields 0;
  * the equilibrium is evaluated in the scalar form obtained by contracting
    the 4th-order Hermite expansion by hand, as a polynomial in
    a = xi.u, q = |u|^2, theta = T - 1 and x2 = |xi|^2 (D = 2):

      P = 1 + a + [a^2 - q + theta (x2 - 2)] / 2
            + a [a^2 - 3 q + 3 theta (x2 - 4)] / 6
            + [a^4 - 6 a^2 q + 3 q^2 + 6 theta (a^2 (x2 - 6) + q (4 - x2))
               + 3 theta^2 (x2^2 - 8 x2 + 8)] / 24,

    f^eq_l = w_l rho P(xi_l) (Eq. MASTERSHIFT3, 4th-order reading);
  * the wall bc walks explicit Python loops over (x, row, population).

Arrays are [37, Lx, Ly] in ``quadrature.velocity_set()`` order.
"""
import numpy as np

from . import quadrature

Q = 37


class Model:
    def __init__(self):
        vel = quadrature.velocity_set()
        s, w_shell = quadrature.weights_fp64()
        self.cx = np.array([c[0] for c in vel])
        self.cy = np.array([c[1] for c in vel])
        c2 = self.cx ** 2 + self.cy ** 2
        self.w = np.array([w_shell[quadrature.SHELL_C2.index(v)] for v in c2])
        self.s = s
        self.xix = s * self.cx
        self.xiy = s * self.cy
        self.x2 = self.xix ** 2 + self.xiy ** 2

    def feq(self, rho, ux, uy, T):
        """rho, ux, uy, T broadcastable arrays -> [37, ...] equilibrium."""
        rho, ux, uy, T = (np.asarray(v, dtype=np.float64) for v in (rho, ux, uy, T))
        sh = (Q,) + (1,) * np.broadcast(rho, ux, uy, T).ndim
        xix, xiy, x2, w = (v.reshape(sh) for v in (self.xix, self.xiy, self.x2, self.w))
        a = xix * ux + xiy * uy
        q = ux * ux + uy * uy
        th = T - 1.0
        P = (1.0 + a + (a * a - q + th * (x2 - 2.0)) / 2.0
             + a * (a * a - 3.0 * q + 3.0 * th * (x2 - 4.0)) / 6.0
             + (a ** 4 - 6.0 * a * a * q + 3.0 * q * q
                + 6.0 * th * (a * a * (x2 - 6.0) + q * (4.0 - x2))
                + 3.0 * th * th * (x2 * x2 - 8.0 * x2 + 8.0)) / 24.0)
        return w * rho * P

    def moments(self, f):
        sh = (Q,) + (1,) * (f.ndim - 1)
        xix, xiy = self.xix.reshape(sh), self.xiy.reshape(sh)
        rho = f.sum(0)
        ux = (xix * f).sum(0) / rho
        uy = (xiy * f).sum(0) / rho
        T = (((xix - ux) ** 2 + (xiy - uy) ** 2) * f).sum(0) / (2.0 * rho)
        return rho, ux, uy, T

    def collide(self, f, tau, g0):
        rho, ux, uy, T = self.moments(f)
        gy = -g0
        feq = self.feq(rho, ux, uy + tau * gy, T - tau * tau * gy * gy / 2.0)
        return f - (f - feq) / tau

    def propagate(self, f, periodic_y):
        Lx, Ly = f.shape[1:]
        out = np.zeros_like(f)
        for l in range(Q):
            g = np.roll(f[l], self.cx[l], axis=0)
            if periodic_y:
                out[l] = np.roll(g, self.cy[l], axis=1)
            else:
                cy = self.cy[l]
                for y in range(Ly):
                    if 0 <= y - cy < Ly:
                        out[l, :, y] = g[:, y - cy]
        return out

    def walls(self, src, dst, T_top, T_bot):
        Lx, Ly = src.shape[1:]
        out = dst.copy()
        for rows, Tw in ((range(0, 3), T_bot), (range(Ly - 3, Ly), T_top)):
            fw = self.feq(1.0, 0.0, 0.0, Tw)
            missing = [(y, l) for y in rows for l in range(Q) if not 0 <= y - self.cy[l] < Ly]
            leaving = [(y, l) for y in rows for l in range(Q) if not 0 <= y + self.cy[l] < Ly]
            den = sum(fw[l] for _, l in missing)
            for x in range(Lx):
                rho_w = sum(src[l, x, y] for y, l in leaving) / den
                for y, l in missing:
                    out[l, x, y] = rho_w * fw[l]
        return out

    def step(self, f, tau, g0, T_top, T_bot, periodic_y=False, phases=7):
        if phases & 1:
            g = self.propagate(f, periodic_y)
            if (phases & 2) and not periodic_y:
                g = self.walls(f, g, T_top, T_bot)
            f = g
        if phases & 4:
            f = self.collide(f, tau, g0)
        return f
