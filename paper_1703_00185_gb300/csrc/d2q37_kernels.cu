// sm_103a kernels of one thermal D2Q37 time step, FP64 populations.
//
// Layout (Sec. "Data Structure Analysis"): structure of arrays, one plane per
// population, each plane column-major in y (y contiguous), in a halo frame of
// (Lx + 2*3) columns by NY rows, physical site (x, y) at
// (x + 3) * NY + (y + 16).  NY = Ly + 32 rounded up to a multiple of 16, so every
// column starts on a 128-byte boundary.  Two frames are double-buffered.
//
// Kernels and the step sequence (Sec. "Code Organization"):
//   wrap      pbc: fill the 3-column x halos (and y halos when y is periodic);
//             needed only after a state is uploaded or after a propagate
//             without collide, because collide and fused write the halo
//             images of the edge columns themselves (store_images)
//   propagate pull form of Eq. master2: dst_l(x,y) = src_l(x - c_lx, y - c_ly)
//   bc        diffuse walls on rows 0..2 and Ly-3..Ly-1
//   collide   BGK relaxation (Eq. discrete) to the shifted equilibrium of
//             Eq. MASTERSHIFT3, in place on dst
//   fused     propagate + bc + collide in one pass, src -> dst
//
// Threads: one per lattice site, blocks of 256 consecutive y of one column
// (the paper's 1-D blocks along y, Sec. "The propagate and bc Kernels").
// Every warp reads 32 consecutive doubles of each population plane, so each
// gather is a coalesced 256-byte row shifted by at most 3 elements.
#include <cuda_runtime.h>

#include "d2q37_launch.h"

namespace d2q37 {

__constant__ ShellConsts c_shell;

namespace {

constexpr int kBlockY = 256;
constexpr int kWallBlock = 128;

// Minimum resident blocks per SM requested for the FP64 site kernels (caps
// their registers at 65536 / (kBlockY * blocks)); tuned on GB300: 2 blocks of
// 256 (128 registers) ran the 2048 x 8192 fused step in 2.79 ms, against
// 2.84 ms with 8 of 64, 2.87 ms with 4 of 128 and 3.53 ms with 1 of 512.
#ifndef D2Q37_SITE_MIN_BLOCKS
#define D2Q37_SITE_MIN_BLOCKS 2
#endif
// The batched kernel (D2Q37_BATCH_MIN_BLOCKS x 128 threads per SM, whatever
// its block_y) reads its parameters from memory instead of the constant bank
// and spills a little at 128 registers (20 bytes per thread); with 3 blocks of
// 128 and no spills it was slower (2970 MLUPS against 3150 for 4, an earlier
// form of the kernel).  The batch's per-lattice shape (block_y = 0), which
// runs the single-lattice kernels, is faster still on the 64-lattice workload.
#ifndef D2Q37_BATCH_MIN_BLOCKS
#define D2Q37_BATCH_MIN_BLOCKS 4
#endif

// P: StepParams or BatchGeo (NY, Hy)
template <class P>
__device__ __forceinline__ long long site_index(const P& p, int x, int y) {
  return (long long)(x + kHx) * p.NY + (y + p.Hy);
}

// rho, u and T of one site (Sec. "Lattice Boltzmann methods"):
// rho = sum f, rho u = s sum c f, D rho T = sum |xi|^2 f - rho |u|^2 (D = 2),
// the last being sum |xi - u|^2 f expanded.  Pair sums and differences carry
// the even and odd moments.  FP64 arithmetic throughout (the fallback of
// site_moments below).
__device__ __forceinline__ void site_moments_fp64(const double (&f)[kQ], double& rho, double& ux, double& uy,
                                                  double& T) {
  double sh[kShells];
  sh[0] = f[0];
#pragma unroll
  for (int k = 1; k < kShells; ++k) sh[k] = 0.0;
  double jx = 0.0, jy = 0.0;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const double sum = f[1 + 2 * p] + f[2 + 2 * p];
    const double dif = f[1 + 2 * p] - f[2 + 2 * p];
    sh[pair_shell(p)] += sum;
    if (pair_cx(p) != 0) jx += (double)pair_cx(p) * dif;
    if (pair_cy(p) != 0) jy += (double)pair_cy(p) * dif;
  }
  rho = sh[0];
  double e = 0.0;
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    rho += sh[k];
    e += (double)shell_c2(k) * sh[k];
  }
  const double inv_rho = 1.0 / rho;
  ux = c_shell.s * jx * inv_rho;
  uy = c_shell.s * jy * inv_rho;
  T = 0.5 * (c_shell.s2 * e * inv_rho - (ux * ux + uy * uy));
}

// The same moments with the sums done in 64-bit integers, off the FP64 pipe
// (GB300 issues 2 FP64 operations per SM per clock but 64+ integer ones).
// Every population is rounded down to the grid of the site's largest
// exponent, 2^(emax - 1075), i.e. to 53 bits relative to the largest
// population, and summed exactly: rho and the moment sums carry one rounding
// per term at that grid (comparable to an FP64 sum) and none from the
// additions.  The roundings are floors, on average 0.5 below for a term whose
// shift drops many bits and less for the largest populations; the sums of r
// and e get a constant back (kFloorR, kFloorE: the mean deficits over
// near-equilibrium states, 16.3 and 104.8 grid units), and those of jx, jy
// need none (sum c = 0).  The remaining -0.3 units of r (-1.2e-17 of rho)
// offset most of the equilibrium's +1.7e-17 (see fx_d0).
// Headroom: |term| < 2^53, |c|^2 <= 10 and 37 terms keep every sum < 2^62.
// Sites with a population that is zero-exponent tiny (< 2^-960), infinite or
// NaN take the FP64 form.
constexpr long long kFloorR = 16, kFloorE = 105;

__device__ __forceinline__ long long fixed_term(double v, int emax) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int e = (hi >> 20) & 0x7FF;
  // the implicit one is set for zero and subnormal inputs too: with emax >= 64
  // their shift is the full 62 and they round to 0 (-1 for a negative zero)
  const long long mant = ((long long)((hi & 0xFFFFF) | 0x100000) << 32) | lo;
  const int sh = min(emax - e, 62);
  const long long s = hi >> 31;  // 0 or -1
  // a negative v as the one's complement of its magnitude, -mant - 1: its
  // arithmetic shift is floor(v 2^-sh) or, when the dropped bits are all zero,
  // one below it
  return (mant ^ s) >> sh;
}

// The exact sums r = sum f, jx, jy = sum c f, e = sum |c|^2 f on the grid
// 2^(emax - 1075); false for the sites that take the FP64 sums.
__device__ __forceinline__ bool site_sums(const double (&f)[kQ], long long& r, long long& jx, long long& jy,
                                          long long& e, int& emax) {
  int hmax = 0;  // the largest |high word|: its exponent field is the largest exponent
#pragma unroll
  for (int l = 0; l < kQ; ++l) hmax = max(hmax, __double2hiint(f[l]) & 0x7FFFFFFF);
  emax = hmax >> 20;
  if (emax < 64 || emax > 2046) return false;
  long long sh[kShells];
  sh[0] = fixed_term(f[0], emax);
#pragma unroll
  for (int k = 1; k < kShells; ++k) sh[k] = 0;
  jx = jy = 0;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const long long vp = fixed_term(f[1 + 2 * p], emax);
    const long long vm = fixed_term(f[2 + 2 * p], emax);
    sh[pair_shell(p)] += vp + vm;
    const long long d = vp - vm;
    jx += pair_cx(p) * d;
    jy += pair_cy(p) * d;
  }
  r = sh[0] + kFloorR;
  e = kFloorE;
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    r += sh[k];
    e += shell_c2(k) * sh[k];
  }
  return true;
}

__device__ __forceinline__ void moments_from_sums(long long r, long long jx, long long jy, long long e, int emax,
                                                  double& rho, double& ux, double& uy, double& T) {
  const double rd = (double)r;
  const double inv = 1.0 / rd;  // the grid scale cancels in u and T
  ux = c_shell.s * (double)jx * inv;
  uy = c_shell.s * (double)jy * inv;
  T = 0.5 * (c_shell.s2 * (double)e * inv - (ux * ux + uy * uy));
  rho = rd * __hiloint2double((emax - 52) << 20, 0);  // 2^(emax - 1075)
}

__device__ __forceinline__ void site_moments(const double (&f)[kQ], double& rho, double& ux, double& uy,
                                             double& T) {
  long long r, jx, jy, e;
  int emax;
  if (site_sums(f, r, jx, jy, e, emax))
    moments_from_sums(r, jx, jy, e, emax, rho, ux, uy, T);
  else
    site_moments_fp64(f, rho, ux, uy, T);
}

// c v for a hop component c in -3..3 given the multiples m = {v, 2v, 3v}.
__device__ __forceinline__ double hop_term(int c, const double (&m)[3]) {
  return c > 0 ? m[c - 1] : -m[-c - 1];
}

// cx ux + cy uy from precomputed multiples: one addition at most.
__device__ __forceinline__ double hop_dot(int cx, int cy, const double (&mx)[3], const double (&my)[3]) {
  if (cx == 0) return hop_term(cy, my);
  if (cy == 0) return hop_term(cx, mx);
  return hop_term(cx, mx) + hop_term(cy, my);
}

// ---- the equilibrium in 64-bit fixed point ---------------------------------
//
// GB300 issues 2 FP64 operations per SM per clock, while the high 64 bits of
// a 64 x 64-bit integer product take about four IMAD.WIDE on the integer
// pipes.  So the equilibrium of the FP64 step is evaluated in fixed point:
// each quantity is an int64 scaled by its own power of two ("Qn": v 2^-n),
// chosen from its range so that every product is the high word of a 128-bit
// product and keeps 2^-55 or better absolute precision on the order-1
// quantities; exact integer sums remove the cancellation that
// limits the FP64 form near T = 0.5 for the outer shells.  Per population
// the result is turned into an FP64 number (fx_to_double: the FP64 pipe's
// integer conversion, or integer operations for the shells of
// D2Q37_INT_CVT_MASK) and relaxed with one FP64 FMA.  The shell factor omega w_k is carried as
// c_k 2^E_k with c_k in [0.5, 1).  The ranges that keep every intermediate
// inside its format hold for rho in (0, 4), |T_bar - 1| < 1 and |u_bar| < 0.35
// per component; other sites take the FP64 evaluation.
//
// With K0 = rho (A0 - theta + theta q + theta^2), K1 = rho (theta/2 - theta q/4
// - theta^2), K2 = rho theta^2 / 8, L0 = rho (B1 - 2 theta), L1 = rho theta / 2,
// M0 = rho (B2 - 3 theta / 2), M1 = rho theta / 4 (site values), the shell
// coefficients of collide_site times c_k rho are
//   R0 = c (K0 + x2 K1 + x2^2 K2),  R1 = c (L0 + x2 L1),  R2 = c (M0 + x2 M1),
//   R3 = c rho / 6,  R4 = c rho / 24 (one product: (c/6) 2^64 is (c/24) 2^66),
// and per pair even = R0 + b (R2 + b R4), odd = a (R1 + b R3), b = a^2.
// A signed site value x meets the unsigned shell constants as x + 2^63 (its
// sign bit flipped), which needs no sign fix: x y 2^-64 = (x + 2^63) y 2^-64
// - y / 2, and the y / 2 terms of a shell are one constant subtracted from R0,
// R1 and R2 (fx_d0, fx_d1, fx_d2), together with corrections for the
// roundings of its sums and per-pair products (0.5 below on average for an
// exact high word, 0.75 for umulhi_t).  K0 > 0.74 rho inside the ranges and
// needs no shift.  With the set lowest bit of the conversion (+0.5 on
// average) and two corrections in fx_d0, the equilibrium's mass bias is
// +1.7e-17 per collision relative to omega rho (without the corrections:
// -7.6e-17), which the moment sums' -1.2e-17 nearly cancels.
// The odd part takes a rounded product: a bias there would act on the
// momentum the same way every step.
constexpr int kFxOut = 55;  // format of R0 and of the results G = even +- odd

using u64 = unsigned long long;

// floor(x y 2^-64) for signed x, unsigned y
__device__ __forceinline__ long long mulhi_su(long long x, u64 y) {
  return (long long)(__umul64hi((u64)x, y) - (y & (u64)(x >> 63)));  // x >> 63: 0 or all ones
}

// The high word of a y with the low-by-low partial product left out: three
// 32 x 32 -> 64-bit multiply-adds and one add, the floor of a y 2^-64 or one
// below it (0.75 below a y 2^-64 on average).  More instructions than the
// exact high word but a shorter dependency chain: the per-pair products,
// which form one chain per pair, take this form.
__device__ __forceinline__ u64 umulhi_t(u64 a, u64 y) {
  const unsigned al = (unsigned)a, ah = (unsigned)(a >> 32);
  const unsigned yl = (unsigned)y, yh = (unsigned)(y >> 32);
  const u64 lh = (u64)al * yh;
  const u64 hl = (u64)ah * yl + (lh & 0xFFFFFFFFull);  // < 2^64
  return (u64)ah * yh + (lh >> 32) + (hl >> 32);
}

// umulhi_t for signed x: x y = (x mod 2^64) y - 2^64 y [x < 0]
__device__ __forceinline__ long long mulhi_su_t(long long x, u64 y) {
  return (long long)(umulhi_t((u64)x, y) - (y & (u64)(x >> 63)));
}

// round(x y 2^-64) (half up) for signed x, unsigned y.  Used where a biased
// rounding would act the same way every step: the odd part of a pair, whose
// magnitude a floor after the sign split would always shrink (a momentum
// damping of 2^-56 per step relative to the odd part).
// The four 32 x 32-bit partial products are independent; the rounding half
// (2^63 of the 128-bit product) enters the middle column as 2^31.
__device__ __forceinline__ long long mulhi_su_rn(long long x, u64 y) {
  const unsigned xl = (unsigned)x, xh = (unsigned)((u64)x >> 32);
  const unsigned yl = (unsigned)y, yh = (unsigned)(y >> 32);
  const u64 ll = (u64)xl * yl, lh = (u64)xl * yh, hl = (u64)xh * yl, hh = (u64)xh * yh;
  const u64 mid = (ll >> 32) + (lh & 0xFFFFFFFFull) + (hl & 0xFFFFFFFFull) + 0x80000000ull;  // < 2^34
  const u64 hi = hh + (lh >> 32) + (hl >> 32) + (mid >> 32);  // floor(((x mod 2^64) y + 2^63) 2^-64)
  return (long long)(hi - (y & (u64)(x >> 63)));
}

// floor(x y 2^-sh) for signed x, y and 0 < sh < 64 (the result fits 64 bits)
__device__ __forceinline__ long long mul_shift(long long x, long long y, int sh) {
  const u64 h = (u64)__mul64hi(x, y);
  const u64 l = (u64)x * (u64)y;
  return (long long)((h << (64 - sh)) | (l >> sh));
}

// g 2^(E - 55) as an FP64 number, two ways: with the FP64 pipe's 64-bit
// integer conversion (round to nearest even) and the power of two added to
// the exponent field, or with integer operations only (round half away from
// zero).  The shells k whose bit is set in D2Q37_INT_CVT_MASK take the
// integer form.  On GB300, with the FP64 pipe about 75 % busy, the last
// shell's 8 populations that way (0x80) ran the 2048 x 8192 step in 2.742 ms,
// against 2.784 ms for none, 2.802 / 2.847 ms for the last two / three
// shells and 2.74-2.82 ms for shell 7 with one of shells 1, 3, 4, 5 (all of
// them, with 4 blocks of 128 per SM: 4.37 against 4.12).
#ifndef D2Q37_INT_CVT_MASK
#define D2Q37_INT_CVT_MASK 0x80
#endif

// g != 0
__device__ __forceinline__ double fx_to_double_fp64(long long g, int E) {
  const double d = (double)g;  // exact up to its one rounding
  const u64 bits = (u64)__double_as_longlong(d) + ((u64)(long long)(E - kFxOut) << 52);
  return __longlong_as_double((long long)bits);
}

// |g| < 2^32 (including 0): the general normalisation
__device__ __noinline__ double fx_to_double_small(u64 m, int E, u64 sign) {
  if (!m) return 0.0;
  const int lz = __clzll((long long)m);
  const u64 n = m << (lz - 1);  // leading one at bit 62
  const u64 mant = (n + 0x200) >> 10;
  const u64 bits = ((u64)(long long)(1023 + 62 - kFxOut + E - lz) << 52) + mant;
  return __longlong_as_double((long long)(bits | sign));
}

__device__ __forceinline__ double fx_to_double_int(long long g, int E) {
  const u64 sm = (u64)(g >> 63);
  const u64 sign = sm & 0x8000000000000000ull;
  const u64 m = ((u64)g ^ sm) - sm;  // |g| < 2^63
  const unsigned mh = (unsigned)(m >> 32);
  if (mh == 0u) return fx_to_double_small(m, E, sign);
  // value = m 2^(E - 55); with the leading one moved to bit 62,
  // n = m 2^(lz - 1) and value = (n / 2^62) 2^(E + 8 - lz); lz >= 1 as m < 2^63
  const int lz = __clz(mh);
  const u64 n = m << (lz - 1);
  const u64 mant = (n + 0x200) >> 10;  // 53 bits, 54 when the rounding carries
  // the leading one of mant adds 1 to the exponent field (and a carry one more)
  const u64 bits = ((u64)(long long)(1023 + 62 - kFxOut + E - lz) << 52) + mant;
  return __longlong_as_double((long long)(bits | sign));
}

// The population of shell k.  The lowest bit of g is set first: g is never
// zero (which the exponent add of the FP64 form needs), and it is 0.5 larger
// on average, which the per-shell corrections of the equilibrium take into
// account.
__device__ __forceinline__ double fx_to_double(long long g, int E, int k) {
  return ((D2Q37_INT_CVT_MASK >> k) & 1) ? fx_to_double_int(g | 1, E) : fx_to_double_fp64(g | 1, E);
}

// c v for a hop component c in -3..3 given the multiples m = {v, 2v, 3v}.
__device__ __forceinline__ long long fx_hop_term(int c, const long long (&m)[3]) {
  return c > 0 ? m[c - 1] : -m[-c - 1];
}

__device__ __forceinline__ long long fx_hop_dot(int cx, int cy, const long long (&mx)[3],
                                                const long long (&my)[3]) {
  if (cx == 0) return fx_hop_term(cy, my);
  if (cy == 0) return fx_hop_term(cx, mx);
  return fx_hop_term(cx, mx) + fx_hop_term(cy, my);
}

// Fixed-point site values: rho (Q61), u_x and u_bar_y = u_y + tau g_y (Q64),
// theta = T_bar - 1 (Q62).
struct FxSite {
  u64 R;
  long long UX, UY, TH;
};

// The fixed-point site values straight from the exact moment sums (no FP64
// arithmetic): with r normalised to rn = r 2^n in [2^63, 2^64), X = 2^126 / rn
// from a float seed and two Newton steps (about 2^-60 relative), then
// j / r = (j 2^n) X 2^-126, u = s j / r, 2 T = s^2 e / r - |u|^2 (unshifted u,
// reading R6), rho = r 2^(emax - 1075).  False when the site is outside the
// fixed-point ranges (rho in (0, 4), |u_x|, |u_bar_y| < 0.35, |theta| < 1) or
// its sums do not fit the scaled forms; those sites take the FP64 collision.
__device__ __forceinline__ bool fx_site_from_sums(long long r, long long jx, long long jy, long long e, int emax,
                                                  const StepParams& p, FxSite& o) {
  if (!p.fx_on || r <= 0 || e < 0) return false;
  const u64 ur = (u64)r;
  const u64 ajx = jx < 0 ? 0ull - (u64)jx : (u64)jx, ajy = jy < 0 ? 0ull - (u64)jy : (u64)jy;
  // |j| < r / 2 and e < 3 r keep the scaled sums inside 64 bits (r < 37 2^53)
  if ((ajx << 1) >= ur || (ajy << 1) >= ur || (u64)e >= ur + ur + ur) return false;
  const int n = __clzll(r);  // >= 5
  const u64 rn = ur << n;
  const unsigned top = (unsigned)(rn >> 40);  // [2^23, 2^24), exactly a float below
  const unsigned rb = __float_as_uint(__frcp_rn(__int_as_float(0x4B000000 | (int)(top & 0x7FFFFF))));
  u64 X = (u64)((rb & 0x7FFFFF) | 0x800000) << (((rb >> 23) & 0xFF) - 64);  // 1/top 2^86, Q62 of 2^64/rn
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const u64 pq = __umul64hi(rn, X);          // Q62 of rn X, about 1
    X = __umul64hi(X, (1ull << 63) - pq) << 2;  // X (2 - rn X), Q62; never above 2^64 / rn
  }
  const long long qx = mulhi_su((long long)((u64)jx << n), X);  // Q62 of jx / r
  const long long qy = mulhi_su((long long)((u64)jy << n), X);
  const long long ux61 = mulhi_su(qx, p.fx_s63);  // Q61 of u_x = s jx / r
  const long long uy61 = mulhi_su(qy, p.fx_s63);
  constexpr long long kU = 0x0B33333333333333LL;  // 0.35 2^61
  if (ux61 >= kU || ux61 <= -kU) return false;
  const long long UX = (long long)((u64)ux61 << 3);                      // Q64
  const long long UY0 = (long long)((u64)uy61 << 3);                     // Q64, unshifted
  const long long UY = UY0 + p.fx_uy_shift;                              // Q64 of u_bar_y
  if (UY >= 0x5999999999999999LL || UY <= -0x5999999999999999LL) return false;  // 0.35 2^64
  const u64 aux = UX < 0 ? 0ull - (u64)UX : (u64)UX, auy = UY0 < 0 ? 0ull - (u64)UY0 : (u64)UY0;
  const u64 er = __umul64hi((u64)e << (n - 2), X);                      // Q60 of e / r (< 3)
  const u64 s2er = __umul64hi(er, p.fx_s2_63);                           // Q59 of s^2 e / r
  const u64 q0 = __umul64hi(aux, aux) + __umul64hi(auy, auy);            // Q64 of |u|^2
  const long long th60 = (long long)s2er - (long long)(q0 >> 5) + p.fx_th_shift;  // Q60 of T + shift
  if (th60 >= (1LL << 60) || th60 <= -(1LL << 60)) return false;
  const int sR = emax - 1014;  // rho 2^61 = r 2^sR
  u64 R;
  if (sR >= 0) {
    if (sR >= n) return false;
    R = ur << sR;
  } else {
    const int rs = min(-sR, 63);
    R = (ur + (1ull << (rs - 1))) >> rs;
  }
  if (R == 0 || R >= (1ull << 63)) return false;
  o.R = R;
  o.UX = UX;
  o.UY = UY;
  o.TH = (long long)((u64)th60 << 2);
  return true;
}

// Where a collision puts the relaxed populations: straight into the site's
// planes of the destination, so that each pair's registers are free once it
// is relaxed.
struct ToPlanes {
  char* d;              // the site's element of plane 0
  const StepParams& p;  // plane_off
  __device__ __forceinline__ void put(int l, double v) const { *(double*)(d + p.plane_off[l]) = v; }
};
struct ToPlanesStride {  // the same with the planes addressed as multiples of the stride
  double* d;
  long long plane;
  __device__ __forceinline__ void put(int l, double v) const { d[l * plane] = v; }
};

// The collision of collide_site_fp64 below with the equilibrium in fixed
// point (formats in the comments), for a site inside the fixed-point ranges.
template <class O>
__device__ __forceinline__ void collide_site_fx(const double (&f)[kQ], const StepParams& p, const FxSite& fs,
                                                const O& out) {
  const long long UX = fs.UX, UY = fs.UY;  // Q64
  const long long TH = fs.TH;              // Q62
  const u64 R = fs.R;                      // Q61
  const u64 AUX = UX < 0 ? 0ull - (u64)UX : (u64)UX, AUY = UY < 0 ? 0ull - (u64)UY : (u64)UY;
  const u64 q = __umul64hi(AUX, AUX) + __umul64hi(AUY, AUY);  // Q64
  const u64 q2 = __umul64hi(q, q);                            // Q64
  const u64 B1 = (1ull << 62) - (q >> 3);                     // Q62: 1 - q/2
  const u64 B2 = (1ull << 61) - (q >> 4);                     //      1/2 - q/4
  const u64 A0 = B1 + (q2 >> 5);                              //      1 - q/2 + q^2/8
  const long long SX = mulhi_su(UX, p.fx_s62), SY = mulhi_su(UY, p.fx_s62);  // Q62
  const long long rA0 = (long long)__umul64hi(R, A0);        // Q59
  const long long rB1 = (long long)__umul64hi(R, B1);        // Q59
  const long long rB2 = (long long)__umul64hi(R, B2);        // Q59
  const long long rth = mul_shift((long long)R, TH, 62);     // Q61: rho theta
  const long long rth2 = mul_shift(rth, TH, 62);             // Q61: rho theta^2
  const long long rthq = mulhi_su(rth, q);                   // Q61: rho theta q
  const long long K0 = rA0 - (rth >> 2) + (rthq >> 2) + (rth2 >> 2);  // Q59
  const long long K1 = (rth >> 2) - (rthq >> 3) - (rth2 >> 1);        // Q60
  const u64 K2 = (u64)rth2;                                           // Q64 (rho theta^2 / 8)
  const long long L0 = rB1 - (rth >> 1);                              // Q59
  const long long M0 = rB2 - (rth >> 2) - (rth >> 3);                 // Q59
  const long long mx[3] = {SX, SX + SX, SX + SX + SX};                // Q62
  const long long my[3] = {SY, SY + SY, SY + SY + SY};
  const u64 kSign = 1ull << 63;
  const u64 uK0 = (u64)K0, uK1 = (u64)K1 ^ kSign, uL0 = (u64)L0 ^ kSign;  // x + 2^63
  const u64 uM0 = (u64)M0 ^ kSign, uTH = (u64)rth ^ kSign;                // L1 = M1 = rth
  const double keep = p.one_minus_omega;
  out.put(0, fma(keep, f[0], fx_to_double((long long)(__umul64hi(uK0, p.fx_c60[0]) - p.fx_d0[0]), p.fx_e[0], 0)));  // x2 = 0
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    const long long R0 = (long long)(__umul64hi(uK0, p.fx_c60[k]) + __umul64hi(uK1, p.fx_cx2_59[k]) +
                                     __umul64hi(K2, p.fx_cx4_55[k]) - p.fx_d0[k]);  // Q55
    const long long R1 = (long long)(__umul64hi(uL0, p.fx_c62[k]) + __umul64hi(uTH, p.fx_cx2_59[k]) -
                                     p.fx_d1[k]);  // Q57
    const long long R2 = (long long)(__umul64hi(uM0, p.fx_c64[k]) + __umul64hi(uTH, p.fx_cx2_60[k]) -
                                     p.fx_d2[k]);  // Q59
    const u64 R3 = __umul64hi(R, p.fx_c6[k]);  // Q61 of c rho / 6, and Q63 of R4 = c rho / 24
    const int E = p.fx_e[k];
#pragma unroll
    for (int pr = 0; pr < kPairs; ++pr) {
      if (pair_shell(pr) != k) continue;
      const long long a = fx_hop_dot(pair_cx(pr), pair_cy(pr), mx, my);  // Q62
      const long long sa = a >> 63;                                      // 0 or -1
      const u64 A = (u64)((a ^ sa) - sa);
      const u64 b = umulhi_t(A, A);                                      // Q60
      const long long t = R2 + (long long)umulhi_t(b, R3);              // Q59: R2 + b R4
      const long long even = R0 + mulhi_su_t(t, b);                      // Q55
      const long long s = R1 + (long long)umulhi_t(b, R3);              // Q57
      const long long oa = mulhi_su_rn(s, A);                            // Q55: |a| (R1 + b R3)
      const long long odd = (oa ^ sa) - sa;                              // the sign of a
      out.put(1 + 2 * pr, fma(keep, f[1 + 2 * pr], fx_to_double(even + odd, E, k)));
      out.put(2 + 2 * pr, fma(keep, f[2 + 2 * pr], fx_to_double(even - odd, E, k)));
    }
  }
}

// BGK collision of one site, f <- f - (f - f^eq(rho, u_bar, T_bar)) / tau with
// u_bar = u + tau g, T_bar = T - tau^2 g^2 / D (Eq. MASTERSHIFT3, Eq. discrete).
// The equilibrium is evaluated per pair as even +- odd parts with per-shell
// coefficients (see ShellConsts), pre-scaled by omega rho w_shell.
template <class O>
__device__ __forceinline__ void collide_site_fp64(const double (&f)[kQ], const StepParams& p, double rho, double ux,
                                                  double uy, double T, const O& out) {
  const double ubx = ux;
  const double uby = uy + p.uy_shift;
  const double q = ubx * ubx + uby * uby;
  const double th = T + p.theta_shift;
  const double A0 = 1.0 + q * (-0.5 + 0.125 * q);
  const double B1 = 1.0 - 0.5 * q;
  const double B2 = 0.5 - 0.25 * q;
  const double sux = c_shell.s * ubx, suy = c_shell.s * uby;
  // a = xi.u_bar = cx sux + cy suy with |cx|, |cy| <= 3: multiples formed once
  const double mx[3] = {sux, sux + sux, sux + sux + sux};
  const double my[3] = {suy, suy + suy, suy + suy + suy};
  const double wr = p.omega * rho;
  const double keep = p.one_minus_omega;
  {
    const double C0 = A0 + th * (c_shell.alpha[0] + q * c_shell.beta[0] + th * c_shell.gamma[0]);
    out.put(0, fma(keep, f[0], wr * c_shell.w[0] * C0));
  }
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    const double W = wr * c_shell.w[k];
    const double P0 = W * (A0 + th * (c_shell.alpha[k] + q * c_shell.beta[k] + th * c_shell.gamma[k]));
    const double P1 = W * (B1 + th * c_shell.delta[k]);
    const double P2 = W * (B2 + th * c_shell.eps[k]);
    const double P3 = W * (1.0 / 6.0);
    const double P4 = W * (1.0 / 24.0);
#pragma unroll
    for (int pr = 0; pr < kPairs; ++pr) {
      if (pair_shell(pr) != k) continue;
      const double a = hop_dot(pair_cx(pr), pair_cy(pr), mx, my);
      const double b = a * a;
      const double even = P0 + b * (P2 + b * P4);
      const double odd = a * (P1 + b * P3);
      out.put(1 + 2 * pr, fma(keep, f[1 + 2 * pr], even + odd));
      out.put(2 + 2 * pr, fma(keep, f[2 + 2 * pr], even - odd));
    }
  }
}

// One site's collision: moments as exact integer sums, then the fixed-point
// form inside its ranges, else the FP64 form; the relaxed populations to out.
template <class O>
__device__ __forceinline__ void collide_site_to(double (&f)[kQ], const StepParams& p, const O& out) {
  long long r, jx, jy, e;
  int emax;
  FxSite fs;
  const bool sums = site_sums(f, r, jx, jy, e, emax);
  if (sums && fx_site_from_sums(r, jx, jy, e, emax, p, fs)) {
    collide_site_fx(f, p, fs, out);
    return;
  }
  double rho, ux, uy, T;
  if (sums)
    moments_from_sums(r, jx, jy, e, emax, rho, ux, uy, T);
  else
    site_moments_fp64(f, rho, ux, uy, T);
  collide_site_fp64(f, p, rho, ux, uy, T, out);
}

// Wall bc for a site of a wall band, applied to its gathered populations:
// rows r = 0..2 from the wall; a population is missing when the pull took it
// from beyond the wall, outgoing when it leaves the column past the wall.
// Missing ones become rho_w f^eq_l(1, 0, T_wall), rho_w = outgoing mass of the
// column / sum of f^eq over the missing pairs, so the wall injects exactly the
// mass that left through it (reading of Sec. "The propagate and bc Kernels").
//
// The outgoing mass is summed row by row, each row's populations in index
// order, and the three row sums as (row 0 + row 1) + row 2: the same grouping
// whether one thread sums the column (wall_density) or the three threads of a
// column's wall rows each sum their own row and combine the sums by warp
// shuffles (wall_band_kernel), so both give the same bits.
template <class P>  // StepParams or BatchGeo (Ly, NY, Hy, plane)
__device__ __forceinline__ double wall_row_outgoing(const double* __restrict__ src, const P& p, int x, int wall,
                                                    int r) {
  const int y = wall ? p.Ly - 1 - r : r;
  const long long i = site_index(p, x, y);
  double s = 0.0;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int cy = vel_cy(l);
    if (wall ? (cy > r) : (cy < -r)) s += src[l * p.plane + i];
  }
  return s;
}

__device__ __forceinline__ double wall_density(const double* __restrict__ src, const StepParams& p, int x,
                                               int wall) {
  const double s0 = wall_row_outgoing(src, p, x, wall, 0);
  const double s1 = wall_row_outgoing(src, p, x, wall, 1);
  const double s2 = wall_row_outgoing(src, p, x, wall, 2);
  return ((s0 + s1) + s2) * p.inv_denom[wall];
}

// The missing populations of a wall-band site at row r from the wall; fw:
// the wall's equilibrium f^eq_l(1, 0, T_wall).
__device__ __forceinline__ void apply_wall(double (&f)[kQ], const double* fw, int wall, int r, double rho_w) {
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int cy = vel_cy(l);
    if (wall ? (cy < -r) : (cy > r)) f[l] = rho_w * fw[l];
  }
}

// Write the populations of physical site (x, y) and, for sites within 3 of a
// periodic edge, their halo images, so the next pull finds the halos filled
// (the pbc step folded into the writer; the halo columns see the same values
// the wrap kernel would copy).  x is uniform across a block, so the extra
// stores are divergence-free except on periodic y edges.
__global__ void __launch_bounds__(256) wrap_kernel(double* __restrict__ buf, StepParams p) {
  const int rows_a = p.periodic_y ? p.Ly + 2 * kHx : p.Ly;
  const int y0 = p.periodic_y ? -kHx : 0;
  const long long n_a = (long long)kQ * 6 * rows_a;
  const long long n_b = p.periodic_y ? (long long)kQ * p.Lx * 6 : 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_a + n_b;
       t += (long long)gridDim.x * blockDim.x) {
    int l, xd, yd, xs, ys;
    if (t < n_a) {  // x halo columns, whole height (corners included when y is periodic)
      const int yy = (int)(t % rows_a);
      const int h = (int)((t / rows_a) % 6);
      l = (int)(t / (6LL * rows_a));
      xd = h < 3 ? h - 3 : p.Lx + h - 3;
      xs = h < 3 ? p.Lx + h - 3 : h - 3;
      yd = y0 + yy;
      ys = yd < 0 ? yd + p.Ly : (yd >= p.Ly ? yd - p.Ly : yd);
    } else {  // y halo rows of the physical columns (periodic y only)
      const long long u = t - n_a;
      const int r = (int)(u % 6);
      xd = (int)((u / 6) % p.Lx);
      l = (int)(u / (6LL * p.Lx));
      xs = xd;
      yd = r < 3 ? r - 3 : p.Ly + r - 3;
      ys = r < 3 ? p.Ly + r - 3 : r - 3;
    }
    buf[l * p.plane + site_index(p, xd, yd)] = buf[l * p.plane + site_index(p, xs, ys)];
  }
}

__global__ void __launch_bounds__(kBlockY) propagate_kernel(const double* __restrict__ src,
                                                            double* __restrict__ dst, StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const long long i = site_index(p, x, y);
#pragma unroll
  for (int l = 0; l < kQ; ++l) dst[l * p.plane + i] = src[l * p.plane + i - vel_cx(l) * p.NY - vel_cy(l)];
}

__global__ void __launch_bounds__(128) bc_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                 StepParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * p.Lx) return;
  const int wall = t >= p.Lx;
  const int x = t - wall * p.Lx;
  const double rho_w = wall_density(src, p, x, wall);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int y = wall ? p.Ly - 1 - r : r;
    const long long i = site_index(p, x, y);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cy = vel_cy(l);
      if (wall ? (cy < -r) : (cy > r)) dst[l * p.plane + i] = rho_w * p.fw[wall][l];
    }
  }
}

// The halo images of a site whose populations are already in its own
// element of dst (written by this thread): read back and copied out.  OFF:
// the planes addressed with the byte offsets of p (read from the constant
// bank by the single-lattice kernels) instead of multiples of p.plane.
template <bool OFF>
__device__ __forceinline__ void store_images(double* __restrict__ dst, const StepParams& p, int x, int y) {
  if (x >= kHx && x < p.Lx - kHx && (!p.periodic_y || (y >= kHx && y < p.Ly - kHx))) return;
  const double* s = dst + site_index(p, x, y);
  double f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l)
    f[l] = OFF ? *(const double*)((const char*)s + p.plane_off[l]) : s[l * p.plane];
  int xs[3] = {x, 0, 0}, ys[3] = {y, 0, 0};
  int nx = 1, ny = 1;
  if (x < kHx) xs[nx++] = x + p.Lx;
  if (x >= p.Lx - kHx) xs[nx++] = x - p.Lx;
  if (p.periodic_y) {
    if (y < kHx) ys[ny++] = y + p.Ly;
    if (y >= p.Ly - kHx) ys[ny++] = y - p.Ly;
  }
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b) {
      if (a == 0 && b == 0) continue;  // the site's own element
      double* d = dst + site_index(p, xs[a], ys[b]);
#pragma unroll
      for (int l = 0; l < kQ; ++l) {
        if (OFF)
          *(double*)((char*)d + p.plane_off[l]) = f[l];
        else
          d[l * p.plane] = f[l];
      }
    }
}

__global__ void __launch_bounds__(kBlockY, D2Q37_SITE_MIN_BLOCKS) collide_kernel(double* __restrict__ buf, StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  double* const b = buf + site_index(p, x, y);
  double f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = *(const double*)((const char*)b + p.plane_off[l]);
  // in place: every population is read above before its pair is written back
  collide_site_to(f, p, ToPlanes{(char*)b, p});
  store_images<true>(buf, p, x, y);
}

// One site of the fused step: gather (pull), wall bc on the wall bands,
// collide, store with halo images.
// p: the lattice (geometry, walls); px: the constants of its collision (tau,
// g: the fixed-point tables, omega, the field shifts), the same object for a
// single lattice.  OFF: addresses from the byte offsets of p (see store_images).
// WALLS = false: the caller never passes a wall-band site.
template <bool OFF, bool WALLS = true>
__device__ __forceinline__ void fused_site(const double* __restrict__ src, double* __restrict__ dst,
                                           const StepParams& p, const StepParams& px, int x, int y) {
  const long long i = site_index(p, x, y);
  double f[kQ];
  if constexpr (OFF) {
    const char* s = (const char*)(src + i);
#pragma unroll
    for (int l = 0; l < kQ; ++l) f[l] = *(const double*)(s + p.pull_off[l]);
  } else {
#pragma unroll
    for (int l = 0; l < kQ; ++l) f[l] = src[l * p.plane + i - vel_cx(l) * p.NY - vel_cy(l)];
  }
  if (WALLS && !p.periodic_y && (y < 3 || y >= p.Ly - 3)) {
    const int wall = y >= p.Ly - 3;
    apply_wall(f, p.fw[wall], wall, wall ? p.Ly - 1 - y : y, wall_density(src, p, x, wall));
  }
  // each pair straight to the site's planes, then the halo images, if any
  if constexpr (OFF)
    collide_site_to(f, px, ToPlanes{(char*)(dst + i), p});
  else
    collide_site_to(f, px, ToPlanesStride{dst + i, p.plane});
  store_images<OFF>(dst, p, x, y);
}

__global__ void __launch_bounds__(kBlockY, D2Q37_SITE_MIN_BLOCKS) fused_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                        StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  // the wall-band kernel, launched next with programmatic stream
  // serialization, reads and writes nothing this kernel writes: it may start
  // once every block of this one has started, and fill the tail
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (y >= p.Ly) return;
  if (!p.periodic_y && (y < 3 || y >= p.Ly - 3)) return;  // wall_band_kernel's
  fused_site<true, false>(src, dst, p, p, x, y);
}

// The fused step of the six wall-band rows of every column (y = 0..2 and
// Ly - 3..Ly - 1, walls only), packed into full warps so that the wall bc's
// work runs at warp width instead of in three lanes of a fused_kernel warp (a
// warp holding wall rows cost about three ordinary warps there).  Each warp
// takes ten (column, wall) groups of three lanes, one lane per wall row (lanes
// 30 and 31 idle); every lane sums the populations of its own row that leave
// through the wall, and the group's three row sums meet by warp shuffles, so
// the column's outgoing mass is read once instead of once per wall site.
// When it is launched as a programmatic dependent of fused_kernel it may run
// while that kernel's last blocks still run; every thread then waits for the
// sites kernel to complete (griddepcontrol.wait: the prerequisite grid has
// finished and its writes are visible) before it exits.  So this grid never
// completes before the sites kernel, and whatever the stream runs after it
// (the next step's sites kernel reads both kernels' rows) is ordered after
// both, in a stream and in a captured graph alike.  Launched normally, the
// wait returns at once.
constexpr int kWallGroupsPerWarp = 10;

__global__ void __launch_bounds__(kWallBlock) wall_band_kernel(const double* __restrict__ src,
                                                              double* __restrict__ dst, StepParams p) {
  const int lane = threadIdx.x & 31;
  const int g = (blockIdx.x * (kWallBlock / 32) + (threadIdx.x >> 5)) * kWallGroupsPerWarp + lane / 3;
  const int r = lane - 3 * (lane / 3);  // row from the wall
  const bool active = lane < 3 * kWallGroupsPerWarp && g < 2 * p.Lx;
  const int x = g >> 1, wall = g & 1;
  const double s = active ? wall_row_outgoing(src, p, x, wall, r) : 0.0;
  const int base = lane - r;  // the group's row-0 lane (idle lanes read lanes 30, 31, 32 mod 32)
  const double s0 = __shfl_sync(0xffffffffu, s, base);
  const double s1 = __shfl_sync(0xffffffffu, s, base + 1);
  const double s2 = __shfl_sync(0xffffffffu, s, base + 2);
  if (active) {
    const int y = wall ? p.Ly - 1 - r : r;
    const long long i = site_index(p, x, y);
    double f[kQ];
    const char* sp = (const char*)(src + i);
#pragma unroll
    for (int l = 0; l < kQ; ++l) f[l] = *(const double*)(sp + p.pull_off[l]);
    apply_wall(f, p.fw[wall], wall, r, ((s0 + s1) + s2) * p.inv_denom[wall]);
    collide_site_to(f, p, ToPlanes{(char*)(dst + i), p});
    store_images<true>(dst, p, x, y);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Many lattices in one launch: block-sized tiles (one column x, BY
// consecutive y) of every lattice in the table, walked by a grid-stride loop
// (persistent when the grid is sized to the resident blocks).  Lattice i
// reads buffer cur_i ^ parity and writes the other one.
// UNIFORM: every lattice of the launch shares tau and g, so the collision
// constants come from the kernel argument `common` (constant bank, like the
// single-lattice kernel) instead of each lattice's entry.
template <int BY, bool UNIFORM>
__global__ void __launch_bounds__(BY, (D2Q37_BATCH_MIN_BLOCKS * 128) / BY > 0 ? (D2Q37_BATCH_MIN_BLOCKS * 128) / BY : 1)
    batch_fused_kernel(const BatchEntry* __restrict__ tab, const int* __restrict__ tile_entry, int n, long long tiles,
                       int parity, StepParams common) {
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    // owning lattice: per-tile table when given, else binary search; its
    // parameters are read in place (read-only, cached)
    const BatchEntry& e = tab[tile_entry ? tile_entry[t] : batch_entry_of(tab, n, t)];
    const int local = (int)(t - e.tile0);  // tiles of one lattice < 2^31: 32-bit division
    const int x = local / e.ytiles;
    const int y = (local - x * e.ytiles) * BY + threadIdx.x;
    const int c = e.cur ^ parity;
    if (y < e.p.Ly)
      fused_site<false>((const double*)e.buf[c], (double*)e.buf[c ^ 1], e.p, UNIFORM ? common : e.p, x, y);
  }
}

// ---- many lattices in one launch, split into site tiles and wall tiles ----
//
// One block per tile, no grid-stride loop: the blocks of site tiles (one
// column x BY rows, the wall rows left out) run fused_kernel's per-site work,
// and the blocks of wall tiles run wall_band_kernel's (three lanes per
// column and wall, the outgoing mass combined by warp shuffles), so that no
// warp of the launch holds a few wall rows among ordinary ones.  Every
// lattice's offsets come from the launch's parameter space (BatchLaunch,
// through the constant cache) and its collision constants from `common`; the
// per-site arithmetic is the single-lattice kernels', so results are the same
// bit for bit.  Requires walls, the same tau and g for every lattice and
// offsets that fit 32 bits (checked on the host).
static_assert(sizeof(BatchLaunch) <= 32764, "BatchLaunch must fit the kernel parameter space");


struct GeoPlanes {
  char* d;  // the site's element of plane 0
  const BatchGeo& g;
  __device__ __forceinline__ void put(int l, double v) const { *(double*)(d + g.plane_off[l]) = v; }
};

// The same with the plane offsets from a shared-memory copy.
struct SharedPlanes {
  char* d;
  const int* off;  // shared memory: plane offsets of the block's lattice
  __device__ __forceinline__ void put(int l, double v) const { *(double*)(d + off[l]) = v; }
};

// The lattice owning block b of the site tiles (wall = false) or wall tiles.
__device__ __forceinline__ int split_owner(const BatchLaunch& L, int b, bool wall) {
  int lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((wall ? L.g[mid].wtile0 : L.g[mid].tile0) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The x halo image(s) of a site of a walled lattice (copied from dst[i]).
__device__ __forceinline__ void split_images(double* __restrict__ dst, const BatchGeo& g, int x, long long i) {
  if (x >= kHx && x < g.Lx - kHx) return;
  const char* s = (const char*)(dst + i);
  double f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = *(const double*)(s + g.plane_off[l]);
  const long long shift = (long long)g.Lx * g.NY;
  if (x < kHx) {
    char* d = (char*)(dst + i + shift);
#pragma unroll
    for (int l = 0; l < kQ; ++l) *(double*)(d + g.plane_off[l]) = f[l];
  }
  if (x >= g.Lx - kHx) {
    char* d = (char*)(dst + i - shift);
#pragma unroll
    for (int l = 0; l < kQ; ++l) *(double*)(d + g.plane_off[l]) = f[l];
  }
}

template <int BY>
__global__ void __launch_bounds__(BY, (D2Q37_BATCH_MIN_BLOCKS * 128) / BY > 0 ? (D2Q37_BATCH_MIN_BLOCKS * 128) / BY : 1)
    batch_split_kernel(const __grid_constant__ BatchLaunch L, const BatchEntry* __restrict__ tab,
                       const int* __restrict__ tile_entry, int parity) {
  const int b = blockIdx.x;
  if (b < L.site_tiles) {
    const BatchGeo& g = L.g[tile_entry[b]];
    // the lattice's 74 offsets in shared memory: the blocks of an SM serve
    // different lattices, whose parameter slices crowd the constant cache
    // (read from there: 5796 MLUPS on the 64-lattice workload, against 5881)
    __shared__ int off[2 * kQ];
    for (int k = threadIdx.x; k < 2 * kQ; k += BY) off[k] = k < kQ ? g.pull_off[k] : g.plane_off[k - kQ];  // BY may be < 74
    __syncthreads();
    // x fastest, as in fused_kernel: the columns a tile pulls from run at the same time
    const int local = b - g.tile0;
    const int yt = local / g.Lx;
    const int x = local - yt * g.Lx;
    const int y = yt * BY + threadIdx.x;
    if (y < 3 || y >= g.Ly - 3) return;  // the wall tiles'
    const int c = g.cur ^ parity;
    const long long i = site_index(g, x, y);
    const char* s = (const char*)((const double*)g.buf[c] + i);
    double f[kQ];
    double* dst = (double*)g.buf[c ^ 1];
#pragma unroll
    for (int l = 0; l < kQ; ++l) f[l] = *(const double*)(s + off[l]);
    collide_site_to(f, L.common, SharedPlanes{(char*)(dst + i), off + kQ});
    split_images(dst, g, x, i);
    return;
  }
  // wall tile: kWallGroupsPerWarp (column, wall) groups per warp, one lane per wall row
  const int w = b - L.site_tiles;
  const BatchGeo& g = L.g[split_owner(L, w, true)];
  const int lane = threadIdx.x & 31;
  const int grp = ((w - g.wtile0) * (BY / 32) + (threadIdx.x >> 5)) * kWallGroupsPerWarp + lane / 3;
  const int r = lane - 3 * (lane / 3);
  const bool active = lane < 3 * kWallGroupsPerWarp && grp < 2 * g.Lx;
  const int x = grp >> 1, wall = grp & 1;
  const int c = g.cur ^ parity;
  const double* src = (const double*)g.buf[c];
  const double sum = active ? wall_row_outgoing(src, g, x, wall, r) : 0.0;
  const int base = lane - r;
  const double s0 = __shfl_sync(0xffffffffu, sum, base);
  const double s1 = __shfl_sync(0xffffffffu, sum, base + 1);
  const double s2 = __shfl_sync(0xffffffffu, sum, base + 2);
  if (!active) return;
  const int y = wall ? g.Ly - 1 - r : r;
  const long long i = site_index(g, x, y);
  const char* s = (const char*)(src + i);
  double f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = *(const double*)(s + g.pull_off[l]);
  apply_wall(f, tab[g.entry].p.fw[wall], wall, r, ((s0 + s1) + s2) * g.inv_denom[wall]);
  double* dst = (double*)g.buf[c ^ 1];
  collide_site_to(f, L.common, GeoPlanes{(char*)(dst + i), g});
  split_images(dst, g, x, i);
}

__global__ void __launch_bounds__(kBlockY) fields_kernel(const double* __restrict__ buf, double* __restrict__ rho,
                                                         double* __restrict__ u, double* __restrict__ T,
                                                         StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const long long i = site_index(p, x, y);
  double f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = buf[l * p.plane + i];
  double r, ux, uy, t;
  site_moments(f, r, ux, uy, t);
  const long long o = (long long)x * p.Ly + y;
  const long long n = (long long)p.Lx * p.Ly;
  rho[o] = r;
  u[o] = ux;
  u[n + o] = uy;
  T[o] = t;
}

__global__ void __launch_bounds__(kBlockY) init_equilibrium_kernel(double* __restrict__ buf,
                                                                   const double* __restrict__ T, StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const double t = T[(long long)x * p.Ly + y];
  double feq[kQ];
  equilibrium(c_shell, 1.0 / t, 0.0, 0.0, t, feq);
  const long long i = site_index(p, x, y);
#pragma unroll
  for (int l = 0; l < kQ; ++l) buf[l * p.plane + i] = feq[l];
}

// The same initial state stored as FP32 deviations d_l = f_l - w_l.
__global__ void __launch_bounds__(kBlockY) init_equilibrium32_kernel(float* __restrict__ buf,
                                                                     const double* __restrict__ T, StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const double t = T[(long long)x * p.Ly + y];
  double feq[kQ];
  equilibrium(c_shell, 1.0 / t, 0.0, 0.0, t, feq);
  const long long i = site_index(p, x, y);
#pragma unroll
  for (int l = 0; l < kQ; ++l) buf[l * p.plane + i] = (float)(feq[l] - c_shell.w[vel_shell(l)]);
}

dim3 site_grid(const StepParams& p) { return dim3(p.Lx, (p.Ly + kBlockY - 1) / kBlockY); }

// (column, wall) groups of the wall-band kernel: 2 Lx, ten per warp
int wall_grid(const StepParams& p) {
  constexpr int per_block = kWallGroupsPerWarp * (kWallBlock / 32);
  return (2 * p.Lx + per_block - 1) / per_block;
}

int done(int n) { return cudaGetLastError() == cudaSuccess ? n : -1; }

}  // namespace

cudaError_t upload_shell_consts(const ShellConsts& c) { return cudaMemcpyToSymbol(c_shell, &c, sizeof(c)); }

int launch_wrap(double* buf, const StepParams& p, cudaStream_t stream) {
  const long long n = (long long)kQ * 6 * (p.periodic_y ? p.Ly + 2 * kHx : p.Ly) +
                      (p.periodic_y ? (long long)kQ * p.Lx * 6 : 0);
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  wrap_kernel<<<(unsigned)blocks, 256, 0, stream>>>(buf, p);
  return done(1);
}

int launch_propagate(const double* src, double* dst, const StepParams& p, cudaStream_t stream) {
  propagate_kernel<<<site_grid(p), kBlockY, 0, stream>>>(src, dst, p);
  return done(1);
}

int launch_bc(const double* src, double* dst, const StepParams& p, cudaStream_t stream) {
  bc_kernel<<<(2 * p.Lx + 127) / 128, 128, 0, stream>>>(src, dst, p);
  return done(1);
}

int launch_collide(double* buf, const StepParams& p, cudaStream_t stream) {
  collide_kernel<<<site_grid(p), kBlockY, 0, stream>>>(buf, p);
  return done(1);
}

int launch_fused(const double* src, double* dst, const StepParams& p, cudaStream_t stream, bool overlap) {
  fused_kernel<<<site_grid(p), kBlockY, 0, stream>>>(src, dst, p);
  if (p.periodic_y) return done(1);
  if (!overlap) {
    wall_band_kernel<<<wall_grid(p), kWallBlock, 0, stream>>>(src, dst, p);
    return done(2);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(wall_grid(p));
  cfg.blockDim = dim3(kWallBlock);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, wall_band_kernel, src, dst, p) != cudaSuccess) return -1;
  return done(2);
}

template <int BY>
int batch_launch(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity, int grid,
                 const StepParams* common, cudaStream_t stream) {
  if (common)
    batch_fused_kernel<BY, true><<<grid, BY, 0, stream>>>(tab, tile_entry, n, tiles, parity, *common);
  else
    batch_fused_kernel<BY, false><<<grid, BY, 0, stream>>>(tab, tile_entry, n, tiles, parity, StepParams{});
  return done(1);
}

template <int BY>
int batch_occupancy() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_fused_kernel<BY, true>, BY, 0);
  return b;
}

int launch_batch_fused(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity,
                       int block_y, int grid, const StepParams* common, cudaStream_t stream) {
  switch (block_y) {
    case 64: return batch_launch<64>(tab, tile_entry, n, tiles, parity, grid, common, stream);
    case 128: return batch_launch<128>(tab, tile_entry, n, tiles, parity, grid, common, stream);
    case 256: return batch_launch<256>(tab, tile_entry, n, tiles, parity, grid, common, stream);
    default: return -1;
  }
}

int launch_batch_split(const BatchLaunch& L, const BatchEntry* tab, const int* tile_entry, int parity, int block_y,
                       cudaStream_t stream) {
  const int grid = L.site_tiles + L.wall_tiles;
  switch (block_y) {
    case 64: batch_split_kernel<64><<<grid, 64, 0, stream>>>(L, tab, tile_entry, parity); break;
    case 128: batch_split_kernel<128><<<grid, 128, 0, stream>>>(L, tab, tile_entry, parity); break;
    case 256: batch_split_kernel<256><<<grid, 256, 0, stream>>>(L, tab, tile_entry, parity); break;
    default: return -1;
  }
  return done(1);
}

int batch_wall_groups_per_tile(int block_y) { return (block_y / 32) * kWallGroupsPerWarp; }

int batch_blocks_per_sm(int block_y) {
  switch (block_y) {
    case 64: return batch_occupancy<64>();
    case 128: return batch_occupancy<128>();
    case 256: return batch_occupancy<256>();
    default: return 0;
  }
}

int launch_fields(const double* buf, double* rho, double* u, double* T, const StepParams& p, cudaStream_t stream) {
  fields_kernel<<<site_grid(p), kBlockY, 0, stream>>>(buf, rho, u, T, p);
  return done(1);
}

int launch_init_equilibrium(double* buf, const double* T, const StepParams& p, cudaStream_t stream) {
  init_equilibrium_kernel<<<site_grid(p), kBlockY, 0, stream>>>(buf, T, p);
  return done(1);
}

int launch_init_equilibrium32(float* buf, const double* T, const StepParams& p, cudaStream_t stream) {
  init_equilibrium32_kernel<<<site_grid(p), kBlockY, 0, stream>>>(buf, T, p);
  return done(1);
}

}  // namespace d2q37
