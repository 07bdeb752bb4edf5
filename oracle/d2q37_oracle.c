/*
 * Plain FP64 CPU oracle of one thermal D2Q37 lattice Boltzmann time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: the velocity set
 * is enumerated here, and the shell weights come from oracle/quadrature.py.
 *
 * Built with -O2 -ffp-contract=off: every product and sum is rounded on its
 * own, in the order written.  OpenMP only splits the site loops across
 * threads; it changes no arithmetic.
 *
 * What each part follows (sections, equations and tables of the paper):
 *   - evolution Eq. discrete in the pull form Eq. master2: first gather the
 *     populations drifting into every site, then relax them (Sec. "Lattice
 *     Boltzmann methods"), kernel order pbc -> propagate -> bc -> collide
 *     (Sec. "Code Organization");
 *   - macroscopic fields rho = sum f, rho u = sum xi f,
 *     D rho T = sum |xi - u|^2 f (Sec. "Lattice Boltzmann methods");
 *   - shifted equilibrium Eq. MASTERSHIFT3: u_bar = u + tau g,
 *     T_bar = T - tau^2 g^2 / D; the Maxwellian is used through its Hermite
 *     expansion truncated at 4th order (reading: the paper's D2Q37 model is
 *     the 4th-order one of its refs. [JFM, POF]; the paper prints no formula);
 *   - periodic x through 3-column halos (Sec. "The propagate and bc Kernels",
 *     Sec. "Data Structure Analysis");
 *   - bc on rows 0..2 and Ly-3..Ly-1, constant wall temperature and zero
 *     velocity (Sec. "The propagate and bc Kernels").  The paper gives no
 *     formula; reading: diffuse wall whose injected mass equals the mass that
 *     left through the wall in the same column.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 37
#define DIM 2
#define NSHELL 8
#define H 3 /* halo width in x and y: populations hop at most 3 sites */

#define PHASE_PROPAGATE 1
#define PHASE_BC 2
#define PHASE_COLLIDE 4

/* ------------------------------------------------------------------ lattice */

static const int shell_c2[NSHELL] = {0, 1, 2, 4, 5, 8, 9, 10};
static int cx_[Q], cy_[Q], shell_[Q];
static double s_scale = 0.0;      /* xi_l = s * c_l */
static double w_[Q];              /* per-population weight */
static double xi_x[Q], xi_y[Q];
static int have_setup = 0;

static void enumerate_velocities(void) {
  int l = 0;
  for (int cx = -3; cx <= 3; ++cx)
    for (int cy = -3; cy <= 3; ++cy)
      if (cx * cx + cy * cy <= 10) {
        cx_[l] = cx;
        cy_[l] = cy;
        for (int k = 0; k < NSHELL; ++k)
          if (shell_c2[k] == cx * cx + cy * cy) shell_[l] = k;
        ++l;
      }
}

/* Install the quadrature computed by oracle/quadrature.py.  Returns the
 * number of velocities found (37) or -1 on a bad argument. */
int orc_setup(double s, const double* w_shell) {
  if (!(s > 0.0) || !w_shell) return -1;
  enumerate_velocities();
  s_scale = s;
  for (int l = 0; l < Q; ++l) {
    w_[l] = w_shell[shell_[l]];
    xi_x[l] = s * (double)cx_[l];
    xi_y[l] = s * (double)cy_[l];
  }
  have_setup = 1;
  return Q;
}

void orc_velocity_set(int* cx, int* cy) {
  enumerate_velocities();
  for (int l = 0; l < Q; ++l) {
    cx[l] = cx_[l];
    cy[l] = cy_[l];
  }
}

void orc_weights(double* w) {
  for (int l = 0; l < Q; ++l) w[l] = w_[l];
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the site loops from here on (n >= 1); the arithmetic does not
 * depend on it. */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------- equilibrium */

static double kron(int i, int j) { return i == j ? 1.0 : 0.0; }

/* Hermite tensors H^(n)(xi) of the standard Gaussian weight, n <= 4. */
static double herm2(const double* x, int i, int j) { return x[i] * x[j] - kron(i, j); }

static double herm3(const double* x, int i, int j, int k) {
  return x[i] * x[j] * x[k] - (x[i] * kron(j, k) + x[j] * kron(i, k) + x[k] * kron(i, j));
}

static double herm4(const double* x, int i, int j, int k, int m) {
  return x[i] * x[j] * x[k] * x[m]
       - (x[i] * x[j] * kron(k, m) + x[i] * x[k] * kron(j, m) + x[i] * x[m] * kron(j, k)
          + x[j] * x[k] * kron(i, m) + x[j] * x[m] * kron(i, k) + x[k] * x[m] * kron(i, j))
       + (kron(i, j) * kron(k, m) + kron(i, k) * kron(j, m) + kron(i, m) * kron(j, k));
}

/* Hermite coefficients of the Maxwellian of Eq. MASTERSHIFT3 divided by rho,
 * with reference temperature 1 and theta = T - 1. */
static double coef2(const double* u, double th, int i, int j) { return u[i] * u[j] + th * kron(i, j); }

static double coef3(const double* u, double th, int i, int j, int k) {
  return u[i] * u[j] * u[k] + th * (kron(i, j) * u[k] + kron(i, k) * u[j] + kron(j, k) * u[i]);
}

static double coef4(const double* u, double th, int i, int j, int k, int m) {
  return u[i] * u[j] * u[k] * u[m]
       + th * (kron(i, j) * u[k] * u[m] + kron(i, k) * u[j] * u[m] + kron(i, m) * u[j] * u[k]
               + kron(j, k) * u[i] * u[m] + kron(j, m) * u[i] * u[k] + kron(k, m) * u[i] * u[j])
       + th * th * (kron(i, j) * kron(k, m) + kron(i, k) * kron(j, m) + kron(i, m) * kron(j, k));
}

/* f_l^eq(rho, u, T) = w_l rho sum_{n<=4} (1/n!) A^(n) : H^(n)(xi_l), the full
 * tensor contractions written out over every index tuple. */
void orc_equilibrium(double rho, double ux, double uy, double T, double* feq) {
  const double u[DIM] = {ux, uy};
  const double th = T - 1.0;
  for (int l = 0; l < Q; ++l) {
    const double x[DIM] = {xi_x[l], xi_y[l]};
    double p1 = 0.0, p2 = 0.0, p3 = 0.0, p4 = 0.0;
    for (int i = 0; i < DIM; ++i) {
      p1 += u[i] * x[i];
      for (int j = 0; j < DIM; ++j) {
        p2 += coef2(u, th, i, j) * herm2(x, i, j);
        for (int k = 0; k < DIM; ++k) {
          p3 += coef3(u, th, i, j, k) * herm3(x, i, j, k);
          for (int m = 0; m < DIM; ++m) p4 += coef4(u, th, i, j, k, m) * herm4(x, i, j, k, m);
        }
      }
    }
    feq[l] = w_[l] * rho * (1.0 + p1 + p2 / 2.0 + p3 / 6.0 + p4 / 24.0);
  }
}

/* ----------------------------------------------------------------- moments */

/* rho = sum f, u = (sum xi f) / rho, T = sum |xi - u|^2 f / (D rho). */
void orc_site_moments(const double* f, double* rho_out, double* ux_out, double* uy_out, double* T_out) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int l = 0; l < Q; ++l) {
    rho += f[l];
    jx += xi_x[l] * f[l];
    jy += xi_y[l] * f[l];
  }
  const double ux = jx / rho, uy = jy / rho;
  double e = 0.0;
  for (int l = 0; l < Q; ++l) {
    const double dx = xi_x[l] - ux, dy = xi_y[l] - uy;
    e += (dx * dx + dy * dy) * f[l];
  }
  *rho_out = rho;
  *ux_out = ux;
  *uy_out = uy;
  *T_out = e / (DIM * rho);
}

/* One BGK relaxation of the populations of one site (Eq. discrete with
 * dt = 1), equilibrium at the shifted fields of Eq. MASTERSHIFT3. */
void orc_collide_site(const double* f, double tau, double gx, double gy, double* out) {
  double rho, ux, uy, T, feq[Q];
  orc_site_moments(f, &rho, &ux, &uy, &T);
  const double ubx = ux + tau * gx, uby = uy + tau * gy;
  const double Tb = T - tau * tau * (gx * gx + gy * gy) / DIM;
  orc_equilibrium(rho, ubx, uby, Tb, feq);
  for (int l = 0; l < Q; ++l) out[l] = f[l] - (f[l] - feq[l]) / tau;
}

/* ----------------------------------------------------------------- lattice */

typedef struct {
  int Lx, Ly, NX, NY, periodic_y;
  double tau, g0, T_top, T_bot;
  double* buf[2]; /* [Q][NX][NY], site (x, y) at (x + H) * NY + (y + H) */
  int cur;
} orc_lattice;

static size_t plane(const orc_lattice* a) { return (size_t)a->NX * a->NY; }
static size_t at(const orc_lattice* a, int x, int y) { return (size_t)(x + H) * a->NY + (y + H); }

orc_lattice* orc_create(int Lx, int Ly, double tau, double g0, double T_top, double T_bot, int periodic_y) {
  if (!have_setup || Lx < 3 || Ly < 6 || !(tau > 0.5)) return NULL;
  orc_lattice* a = (orc_lattice*)calloc(1, sizeof(orc_lattice));
  if (!a) return NULL;
  a->Lx = Lx; a->Ly = Ly; a->NX = Lx + 2 * H; a->NY = Ly + 2 * H;
  a->tau = tau; a->g0 = g0; a->T_top = T_top; a->T_bot = T_bot; a->periodic_y = periodic_y;
  for (int b = 0; b < 2; ++b) {
    a->buf[b] = (double*)calloc((size_t)Q * plane(a), sizeof(double)); /* halo rows stay 0 */
    if (!a->buf[b]) {
      free(a->buf[0]);
      free(a);
      return NULL;
    }
  }
  return a;
}

void orc_destroy(orc_lattice* a) {
  if (!a) return;
  free(a->buf[0]);
  free(a->buf[1]);
  free(a);
}

/* Physical populations in/out as [Q][Lx][Ly] in this oracle's velocity order. */
void orc_set_populations(orc_lattice* a, const double* f) {
  double* d = a->buf[a->cur];
  for (int l = 0; l < Q; ++l)
    for (int x = 0; x < a->Lx; ++x)
      for (int y = 0; y < a->Ly; ++y)
        d[l * plane(a) + at(a, x, y)] = f[((size_t)l * a->Lx + x) * a->Ly + y];
}

void orc_get_populations(const orc_lattice* a, double* f) {
  const double* d = a->buf[a->cur];
  for (int l = 0; l < Q; ++l)
    for (int x = 0; x < a->Lx; ++x)
      for (int y = 0; y < a->Ly; ++y)
        f[((size_t)l * a->Lx + x) * a->Ly + y] = d[l * plane(a) + at(a, x, y)];
}

/* pbc: copy the 3 rightmost physical columns into the left halo and the 3
 * leftmost into the right halo (whole columns, so halo rows come along);
 * with periodic_y the same is done for rows first. */
static void wrap_halos(orc_lattice* a, double* d) {
  const int Lx = a->Lx, Ly = a->Ly;
  for (int l = 0; l < Q; ++l) {
    double* p = d + l * plane(a);
    if (a->periodic_y)
      for (int x = 0; x < Lx; ++x)
        for (int k = 1; k <= H; ++k) {
          p[at(a, x, -k)] = p[at(a, x, Ly - k)];
          p[at(a, x, Ly - 1 + k)] = p[at(a, x, k - 1)];
        }
    for (int k = 1; k <= H; ++k)
      for (int y = -H; y < Ly + H; ++y) {
        p[at(a, -k, y)] = p[at(a, Lx - k, y)];
        p[at(a, Lx - 1 + k, y)] = p[at(a, k - 1, y)];
      }
  }
}

/* propagate, pull form (Eq. master2): dst_l(x, y) = src_l(x - cx_l, y - cy_l). */
static void propagate(orc_lattice* a, const double* src, double* dst) {
#pragma omp parallel for schedule(static)
  for (int x = 0; x < a->Lx; ++x)
    for (int l = 0; l < Q; ++l)
      for (int y = 0; y < a->Ly; ++y)
        dst[l * plane(a) + at(a, x, y)] = src[l * plane(a) + at(a, x - cx_[l], y - cy_[l])];
}

/* bc on one wall.  For column x, the outgoing populations are those at rows
 * 0..2 of src that the pull sends past the wall; the missing populations are
 * those at rows 0..2 of dst that the pull took from beyond the wall.  The
 * missing ones are replaced by rho_w * f^eq(1, 0, T_wall), with rho_w chosen
 * so the injected mass equals the outgoing mass of that column. */
static void wall(orc_lattice* a, const double* src, double* dst, int top) {
  const int Ly = a->Ly;
  const double Tw = top ? a->T_top : a->T_bot;
  double fw[Q];
  orc_equilibrium(1.0, 0.0, 0.0, Tw, fw);
  double denom = 0.0;
  for (int r = 0; r < 3; ++r) {
    const int y = top ? Ly - 1 - r : r;
    for (int l = 0; l < Q; ++l) {
      const int ys = y - cy_[l];
      if (ys < 0 || ys >= Ly) denom += fw[l];
    }
  }
#pragma omp parallel for schedule(static)
  for (int x = 0; x < a->Lx; ++x) {
    double out = 0.0;
    for (int r = 0; r < 3; ++r) {
      const int y = top ? Ly - 1 - r : r;
      for (int l = 0; l < Q; ++l) {
        const int yd = y + cy_[l];
        if (yd < 0 || yd >= Ly) out += src[l * plane(a) + at(a, x, y)];
      }
    }
    const double rho_w = out / denom;
    for (int r = 0; r < 3; ++r) {
      const int y = top ? Ly - 1 - r : r;
      for (int l = 0; l < Q; ++l) {
        const int ys = y - cy_[l];
        if (ys < 0 || ys >= Ly) dst[l * plane(a) + at(a, x, y)] = rho_w * fw[l];
      }
    }
  }
}

static void collide(orc_lattice* a, double* d) {
  const double gx = 0.0, gy = -a->g0;
#pragma omp parallel for schedule(static)
  for (int x = 0; x < a->Lx; ++x) {
    double f[Q], out[Q];
    for (int y = 0; y < a->Ly; ++y) {
      for (int l = 0; l < Q; ++l) f[l] = d[l * plane(a) + at(a, x, y)];
      orc_collide_site(f, a->tau, gx, gy, out);
      for (int l = 0; l < Q; ++l) d[l * plane(a) + at(a, x, y)] = out[l];
    }
  }
}

/* n time steps.  phases: 1 = pbc + propagate, 2 = bc (only together with 1),
 * 4 = collide; 7 is the full step.  Returns 0, or -1 on bad phases. */
int orc_run(orc_lattice* a, int nsteps, int phases) {
  if ((phases & PHASE_BC) && !(phases & PHASE_PROPAGATE)) return -1;
  for (int t = 0; t < nsteps; ++t) {
    if (phases & PHASE_PROPAGATE) {
      double* src = a->buf[a->cur];
      double* dst = a->buf[1 - a->cur];
      wrap_halos(a, src);
      propagate(a, src, dst);
      if ((phases & PHASE_BC) && !a->periodic_y) {
        wall(a, src, dst, 0);
        wall(a, src, dst, 1);
      }
      a->cur = 1 - a->cur;
    }
    if (phases & PHASE_COLLIDE) collide(a, a->buf[a->cur]);
  }
  return 0;
}

/* rho, u (ux plane then uy plane) and T of every physical site, [x * Ly + y]. */
void orc_fields(const orc_lattice* a, double* rho, double* u, double* T) {
  const size_t n = (size_t)a->Lx * a->Ly;
  const double* d = a->buf[a->cur];
#pragma omp parallel for schedule(static)
  for (int x = 0; x < a->Lx; ++x) {
    double f[Q];
    for (int y = 0; y < a->Ly; ++y) {
      for (int l = 0; l < Q; ++l) f[l] = d[l * plane(a) + at(a, x, y)];
      const size_t i = (size_t)x * a->Ly + y;
      orc_site_moments(f, &rho[i], &u[i], &u[n + i], &T[i]);
    }
  }
}

/* Populations at equilibrium with given fields, each [x * Ly + y]. */
void orc_set_equilibrium(orc_lattice* a, const double* rho, const double* ux, const double* uy, const double* T) {
  double* d = a->buf[a->cur];
#pragma omp parallel for schedule(static)
  for (int x = 0; x < a->Lx; ++x) {
    double feq[Q];
    for (int y = 0; y < a->Ly; ++y) {
      const size_t i = (size_t)x * a->Ly + y;
      orc_equilibrium(rho[i], ux[i], uy[i], T[i], feq);
      for (int l = 0; l < Q; ++l) d[l * plane(a) + at(a, x, y)] = feq[l];
    }
  }
}

/* ------------------------------------------------ Rayleigh-Taylor initial state */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one step of the generator
 * from state v, i.e. the finaliser applied to v + 0x9e3779b97f4a7c15. */
uint64_t orc_splitmix64(uint64_t v) {
  uint64_t z = v + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Initial temperature of the Rayleigh-Taylor set-up: cold (T_top) over hot
 * (T_bot), interface y_i(x) = Ly/2 + (Ly/64) sin(2 pi (x + 1/2) / Lx),
 * times (1 + 1e-3 (2U - 1)) with U = (splitmix64(seed + x Ly + y) >> 11) 2^-53. */
void orc_rt_temperature(int Lx, int Ly, uint64_t seed, double T_top, double T_bot, double* T) {
  for (int x = 0; x < Lx; ++x) {
    const double arg = (2.0 * M_PI * ((double)x + 0.5)) / (double)Lx;
    const double yi = 0.5 * (double)Ly + ((double)Ly / 64.0) * sin(arg);
    for (int y = 0; y < Ly; ++y) {
      const double T0 = ((double)y + 0.5 < yi) ? T_bot : T_top;
      const uint64_t r = orc_splitmix64(seed + (uint64_t)x * (uint64_t)Ly + (uint64_t)y);
      const double U = (double)(r >> 11) * 0x1.0p-53;
      T[(size_t)x * Ly + y] = T0 * (1.0 + 1e-3 * (2.0 * U - 1.0));
    }
  }
}

/* Populations at rest at equilibrium: rho = 1/T (uniform pressure), u = 0. */
void orc_init_rayleigh_taylor(orc_lattice* a, uint64_t seed) {
  const int Lx = a->Lx, Ly = a->Ly;
  double* T = (double*)malloc((size_t)Lx * Ly * sizeof(double));
  if (!T) return;
  orc_rt_temperature(Lx, Ly, seed, a->T_top, a->T_bot, T);
  double* d = a->buf[a->cur];
  memset(a->buf[0], 0, (size_t)Q * plane(a) * sizeof(double));
  memset(a->buf[1], 0, (size_t)Q * plane(a) * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int x = 0; x < Lx; ++x) {
    double feq[Q];
    for (int y = 0; y < Ly; ++y) {
      const double t = T[(size_t)x * Ly + y];
      orc_equilibrium(1.0 / t, 0.0, 0.0, t, feq);
      for (int l = 0; l < Q; ++l) d[l * plane(a) + at(a, x, y)] = feq[l];
    }
  }
  free(T);
}
