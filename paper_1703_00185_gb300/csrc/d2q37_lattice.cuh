// D2Q37 lattice description and the per-site FP64 arithmetic shared by the
// kernels of this library (host and device).
//
// Velocity set (reading of Sec. "Lattice Boltzmann methods"; the paper labels
// populations arbitrarily): every integer hop c with |c|^2 <= 10, 37 vectors
// in 8 shells.  This library orders them as the rest population followed by
// 18 pairs (c, -c), pairs grouped by shell, so that the even and odd parts of
// the equilibrium are shared inside a pair.
#pragma once

#include <cstdint>

namespace d2q37 {

constexpr int kQ = 37;
constexpr int kPairs = 18;
constexpr int kShells = 8;
constexpr int kHx = 3;   // halo columns: populations move at most 3 sites (Sec. "Data Structure Analysis")
constexpr int kHy = 16;  // halo rows: 16 doubles = 128 B keeps every column 128-byte aligned

// Population l = 0 is the rest population; pair p has l = 1 + 2p for +c and
// l = 2 + 2p for -c.
__host__ __device__ constexpr int pair_cx(int p) {
  switch (p) {
    case 0: return 1;  case 1: return 0;                      // shell |c|^2 = 1
    case 2: return 1;  case 3: return 1;                      // 2
    case 4: return 2;  case 5: return 0;                      // 4
    case 6: return 2;  case 7: return 2;  case 8: return 1;  case 9: return 1;   // 5
    case 10: return 2; case 11: return 2;                     // 8
    case 12: return 3; case 13: return 0;                     // 9
    case 14: return 3; case 15: return 3; case 16: return 1; case 17: return 1;  // 10
    default: return 0;
  }
}

__host__ __device__ constexpr int pair_cy(int p) {
  switch (p) {
    case 0: return 0;  case 1: return 1;
    case 2: return 1;  case 3: return -1;
    case 4: return 0;  case 5: return 2;
    case 6: return 1;  case 7: return -1; case 8: return 2;  case 9: return -2;
    case 10: return 2; case 11: return -2;
    case 12: return 0; case 13: return 3;
    case 14: return 1; case 15: return -1; case 16: return 3; case 17: return -3;
    default: return 0;
  }
}

__host__ __device__ constexpr int pair_shell(int p) {
  return p < 2 ? 1 : p < 4 ? 2 : p < 6 ? 3 : p < 10 ? 4 : p < 12 ? 5 : p < 14 ? 6 : 7;
}

__host__ __device__ constexpr int vel_cx(int l) { return l == 0 ? 0 : ((l - 1) % 2 == 0 ? 1 : -1) * pair_cx((l - 1) / 2); }
__host__ __device__ constexpr int vel_cy(int l) { return l == 0 ? 0 : ((l - 1) % 2 == 0 ? 1 : -1) * pair_cy((l - 1) / 2); }
__host__ __device__ constexpr int vel_shell(int l) { return l == 0 ? 0 : pair_shell((l - 1) / 2); }

// |c|^2 of each shell.
__host__ __device__ constexpr int shell_c2(int k) {
  return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 4 : k == 4 ? 5 : k == 5 ? 8 : k == 6 ? 9 : 10;
}

// Host tables (used by the quadrature solve and the ABI).
constexpr int kCx[kQ] = {vel_cx(0),  vel_cx(1),  vel_cx(2),  vel_cx(3),  vel_cx(4),  vel_cx(5),  vel_cx(6),
                         vel_cx(7),  vel_cx(8),  vel_cx(9),  vel_cx(10), vel_cx(11), vel_cx(12), vel_cx(13),
                         vel_cx(14), vel_cx(15), vel_cx(16), vel_cx(17), vel_cx(18), vel_cx(19), vel_cx(20),
                         vel_cx(21), vel_cx(22), vel_cx(23), vel_cx(24), vel_cx(25), vel_cx(26), vel_cx(27),
                         vel_cx(28), vel_cx(29), vel_cx(30), vel_cx(31), vel_cx(32), vel_cx(33), vel_cx(34),
                         vel_cx(35), vel_cx(36)};
constexpr int kCy[kQ] = {vel_cy(0),  vel_cy(1),  vel_cy(2),  vel_cy(3),  vel_cy(4),  vel_cy(5),  vel_cy(6),
                         vel_cy(7),  vel_cy(8),  vel_cy(9),  vel_cy(10), vel_cy(11), vel_cy(12), vel_cy(13),
                         vel_cy(14), vel_cy(15), vel_cy(16), vel_cy(17), vel_cy(18), vel_cy(19), vel_cy(20),
                         vel_cy(21), vel_cy(22), vel_cy(23), vel_cy(24), vel_cy(25), vel_cy(26), vel_cy(27),
                         vel_cy(28), vel_cy(29), vel_cy(30), vel_cy(31), vel_cy(32), vel_cy(33), vel_cy(34),
                         vel_cy(35), vel_cy(36)};
constexpr int kShellOf[kQ] = {
    vel_shell(0),  vel_shell(1),  vel_shell(2),  vel_shell(3),  vel_shell(4),  vel_shell(5),  vel_shell(6),
    vel_shell(7),  vel_shell(8),  vel_shell(9),  vel_shell(10), vel_shell(11), vel_shell(12), vel_shell(13),
    vel_shell(14), vel_shell(15), vel_shell(16), vel_shell(17), vel_shell(18), vel_shell(19), vel_shell(20),
    vel_shell(21), vel_shell(22), vel_shell(23), vel_shell(24), vel_shell(25), vel_shell(26), vel_shell(27),
    vel_shell(28), vel_shell(29), vel_shell(30), vel_shell(31), vel_shell(32), vel_shell(33), vel_shell(34),
    vel_shell(35), vel_shell(36)};

// Solve the quadrature (quadrature_dd.cpp).  False if no root was found.
bool solve_quadrature(double* s, double w_shell[kShells]);

// Constants of the equilibrium that depend only on the quadrature.  With
// a = xi.u, q = |u|^2, theta = T - 1 and x2 = |xi|^2 = s^2 |c|^2, the 4th-order
// Hermite equilibrium (D = 2) is f^eq = w rho P with
//   P = C0 + a C1 + a^2 C2 + a^3 / 6 + a^4 / 24,
//   C0 = 1 - q/2 + q^2/8 + theta [ (x2-2)/2 + q (4-x2)/4 + theta (x2^2-8 x2+8)/8 ],
//   C1 = 1 - q/2 + theta (x2-4)/2,
//   C2 = 1/2 - q/4 + theta (x2-6)/4,
// i.e. per shell: alpha = (x2-2)/2, beta = (4-x2)/4, gamma = (x2^2-8x2+8)/8,
// delta = (x2-4)/2, eps = (x2-6)/4.
struct ShellConsts {
  double s;
  double s2;
  double w[kShells];
  double alpha[kShells], beta[kShells], gamma[kShells], delta[kShells], eps[kShells];
};

// FP32 deviation storage: populations are stored as d_l = f_l - w_l in FP32,
// with 32 halo rows (128 bytes) above and below.
constexpr int kHy32 = 32;

// Quadrature constants for the FP32-storage kernels: the wide-precision ones
// as FP64 and as double-float (hi, lo) pairs, the rest in FP32.
struct ShellConsts32 {
  double s, s2, inv_s2;
  float s_hi, s_lo, s2_hi, s2_lo, inv_s2_hi, inv_s2_lo;
  double x2[kShells];  // s^2 |c|^2 per shell
  float x2_hi[kShells], x2_lo[kShells];
  double w64[kShells];
  float w[kShells];
  float delta[kShells], eps[kShells];  // (x2 - 4)/2, (x2 - 6)/4
};

// Per-lattice parameters of one step, passed by value to every kernel.
struct StepParams {
  int Lx, Ly;
  int NY;          // column stride (elements)
  int Hy;          // halo rows below the lattice (16 for FP64, 32 for FP32 storage)
  int periodic_y;
  long long plane; // population plane stride (elements) = (Lx + 2 kHx) * NY
  // byte offsets from a site to the source of its pull (l plane - c_l . (NY, 1))
  // and to its population planes (l plane), for the single-lattice kernels
  long long pull_off[kQ], plane_off[kQ];
  float omega_f, keep_f;  // 1/tau and 1 - 1/tau rounded to FP32 (FP32 storage)
  float uy_shift_df[2];    // uy_shift and theta_shift as double-float (hi, lo) pairs
  float theta_shift_df[2];
  double omega;    // 1 / tau
  double one_minus_omega;
  double uy_shift;    // tau g_y = -tau g0: u_bar = u + tau g (Eq. MASTERSHIFT3)
  double theta_shift; // T_bar - 1 - T = -tau^2 g0^2 / D - 1
  double fw[2][kQ];   // wall equilibria f^eq(1, 0, T_wall): [0] bottom, [1] top
  double inv_denom[2];// 1 / sum of fw over the missing (row, population) pairs
  // the same for the FP32-storage walls, rounded once from FP64:
  float fw32[2][kQ];    // fw
  float fwmw32[2][kQ];  // fw - w
  float wall_e32[2][2];   // (hi, lo): sum_M fwmw32 - sum_O w + sum_M w (M missing, O leaving pairs)
  float wall_inv32[2][2]; // (hi, lo): 1 / sum_M fw32
  // Fixed-point equilibrium constants of the FP64 step: per shell k,
  // omega w_k = c_k 2^fx_e[k] with c_k in [0.5, 1); as unsigned integers, each
  // at the scale that puts its product straight into the format it feeds:
  // c 2^60, 2^62, 2^64; c x2 2^59, 2^60; c x2^2 2^55; (c/6) 2^64, which is
  // also (c/24) 2^66 (x2 = s^2 |c_l|^2).
  unsigned long long fx_c60[kShells], fx_c62[kShells], fx_c64[kShells];
  unsigned long long fx_cx2_59[kShells], fx_cx2_60[kShells], fx_cx4_55[kShells];
  unsigned long long fx_c6[kShells];
  // subtracted from R0, R1, R2 (mod 2^64): y / 2 for each product whose site
  // value enters with its sign bit flipped (x + 2^63), less a rounding
  // correction
  unsigned long long fx_d0[kShells], fx_d1[kShells], fx_d2[kShells];
  int fx_e[kShells];
  unsigned long long fx_s62;  // s 2^62
  unsigned long long fx_s63, fx_s2_63;  // s 2^63, s^2 2^63
  long long fx_uy_shift;      // tau g_y 2^64
  long long fx_th_shift;      // (theta_shift) 2^60 = (-tau^2 g^2 / 2 - 1) 2^60
  int fx_on;                  // 0: the shifts do not fit the formats, every site takes FP64
};

// One lattice of a batched launch.  Tiles are one column x by `block_y`
// consecutive rows; this lattice owns tiles [tile0, tile0 + Lx * ytiles).
struct BatchEntry {
  StepParams p;
  void* buf[2];
  int cur;          // buffer holding the state when the launch parity is 0
  int ytiles;       // ceil(Ly / block_y)
  long long tile0;  // first tile of this lattice
};

// One lattice of a split batched launch (FP64, walls): its geometry, with
// the 37 pull and plane offsets as 32-bit byte offsets, in the launch's
// parameter space (BatchLaunch), where every block reads it through the
// constant cache.  Site tiles are one column x `block_y` rows (the rows
// outside the wall bands); wall tiles hold kBatchWallGroups (column, wall)
// groups of three wall rows each.
struct BatchGeo {
  int pull_off[kQ];   // byte offset from a site to the source of its pull
  int plane_off[kQ];  // byte offset from a site to its element of plane l
  int Lx, Ly, NY, Hy;
  int ytiles;         // site tiles per column
  int tile0, wtile0;  // first site tile and first wall tile of this lattice
  int cur;            // buffer holding the state when the launch parity is 0
  int entry;          // index of this lattice in the BatchEntry table (wall equilibria)
  long long plane;    // population plane stride (elements)
  void* buf[2];
  double inv_denom[2];
};

constexpr int kBatchGeoMax = 64;       // lattices per split launch (parameter space: 32 KB)
constexpr int kBatchWallGroups = 40;   // (column, wall) groups per wall tile: 10 per warp, 4 warps

struct BatchLaunch {
  StepParams common;  // the collision constants every lattice shares (same tau and g)
  int n;
  int site_tiles, wall_tiles;
  BatchGeo g[kBatchGeoMax];
};

// One lattice of a split batched launch in FP32 storage (BatchLaunch32): the
// fields of StepParams that the FP32 per-site code reads, under the same
// names, with the wall constants as pointers into the lattice's entry of the
// BatchEntry table (device memory; only wall rows read them).
struct BatchGeo32 {
  int Lx, Ly, NY, Hy, periodic_y;
  int tile0, cur;
  long long plane;
  void* buf[2];
  float omega_f, keep_f;
  float uy_shift_df[2], theta_shift_df[2];
  double theta_shift;
  const float (*fw32)[kQ];
  const float (*fwmw32)[kQ];
  const float (*wall_e32)[2];
  const float (*wall_inv32)[2];
};

constexpr int kBatchGeo32Max = 128;  // lattices per split FP32 launch

struct BatchLaunch32 {
  int n;
  BatchGeo32 g[kBatchGeo32Max];
};

// Index of the entry owning tile t (entries sorted by tile0, tile0[0] = 0).
__device__ __forceinline__ int batch_entry_of(const BatchEntry* __restrict__ tab, int n, long long t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].tile0 <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// f^eq of one site into feq[37] (host or device).
__host__ __device__ inline void equilibrium(const ShellConsts& c, double rho, double ux, double uy, double T,
                                            double* feq) {
  const double q = ux * ux + uy * uy;
  const double th = T - 1.0;
  const double A0 = 1.0 + q * (-0.5 + 0.125 * q);
  const double B1 = 1.0 - 0.5 * q;
  const double B2 = 0.5 - 0.25 * q;
  const double sux = c.s * ux, suy = c.s * uy;
  feq[0] = rho * c.w[0] * (A0 + th * (c.alpha[0] + q * c.beta[0] + th * c.gamma[0]));
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const int k = pair_shell(p);
    const double C0 = A0 + th * (c.alpha[k] + q * c.beta[k] + th * c.gamma[k]);
    const double C1 = B1 + th * c.delta[k];
    const double C2 = B2 + th * c.eps[k];
    const double a = pair_cx(p) * sux + pair_cy(p) * suy;
    const double b = a * a;
    const double even = C0 + b * (C2 + b * (1.0 / 24.0));
    const double odd = a * (C1 + b * (1.0 / 6.0));
    const double W = rho * c.w[k];
    feq[1 + 2 * p] = W * (even + odd);
    feq[2 + 2 * p] = W * (even - odd);
  }
}

}  // namespace d2q37
