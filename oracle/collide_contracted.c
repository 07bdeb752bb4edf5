/*
 * One site collision with the equilibrium contracted by hand (TEST
 * INFRASTRUCTURE; compiled only into the counting build, flop_count.cpp,
 * after d2q37_oracle.c, whose velocity set and weights it uses).
 *
 * It computes what orc_collide_site computes (Eq. discrete with dt = 1, the
 * shifted fields of Eq. MASTERSHIFT3, the 4th-order Hermite equilibrium of the
 * Maxwellian), in the scalar form that the tensor contractions reduce to for
 * D = 2.  With a = xi.u, q = |u|^2, theta = T - 1 and x2 = |xi|^2:
 *
 *   P = 1 + a + [a^2 - q + theta (x2 - 2)] / 2
 *         + a [a^2 - 3 q + 3 theta (x2 - 4)] / 6
 *         + [a^4 - 6 a^2 q + 3 q^2 + 6 theta (a^2 (x2 - 6) + q (4 - x2))
 *            + 3 theta^2 (x2^2 - 8 x2 + 8)] / 24,
 *
 * f^eq_l = w_l rho P(xi_l).  Each population is evaluated on its own, with no
 * sharing between populations of a shell or of a (c, -c) pair: the plain
 * per-population arithmetic of the method, whose operation count is the FP64
 * work of one site update in the roofline's flop term.  The moments use
 * 2 rho T = sum |xi|^2 f - rho |u|^2 (sum |xi - u|^2 f expanded).
 */
void orc_collide_site_contracted(const double* f, double tau, double gx, double gy, double* out) {
  double rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
  for (int l = 0; l < Q; ++l) {
    const double x2 = xi_x[l] * xi_x[l] + xi_y[l] * xi_y[l];
    rho += f[l];
    jx += xi_x[l] * f[l];
    jy += xi_y[l] * f[l];
    e += x2 * f[l];
  }
  const double ux = jx / rho, uy = jy / rho;
  const double T = (e / rho - (ux * ux + uy * uy)) / DIM;
  const double ubx = ux + tau * gx, uby = uy + tau * gy;
  const double Tb = T - tau * tau * (gx * gx + gy * gy) / DIM;
  const double q = ubx * ubx + uby * uby;
  const double th = Tb - 1.0;
  for (int l = 0; l < Q; ++l) {
    const double x2 = xi_x[l] * xi_x[l] + xi_y[l] * xi_y[l];
    const double a = xi_x[l] * ubx + xi_y[l] * uby;
    const double a2 = a * a;
    const double P = 1.0 + a + (a2 - q + th * (x2 - 2.0)) / 2.0
                   + a * (a2 - 3.0 * q + 3.0 * th * (x2 - 4.0)) / 6.0
                   + (a2 * a2 - 6.0 * a2 * q + 3.0 * q * q
                      + 6.0 * th * (a2 * (x2 - 6.0) + q * (4.0 - x2))
                      + 3.0 * th * th * (x2 * x2 - 8.0 * x2 + 8.0)) / 24.0;
    const double feq = w_[l] * rho * P;
    out[l] = f[l] - (f[l] - feq) / tau;
  }
}
