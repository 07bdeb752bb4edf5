// sm_103a kernels of the D2Q37 step with FP32 deviation storage.
//
// Populations are stored as d_l = f_l - w_l in FP32 (half the HBM bytes of
// FP64: 296 B per site update).  Precision split, per site:
//   * moment sums (density, momentum, energy): exact 64-bit integer sums of
//     the stored FP32 values (no rounding in the additions);
//   * rho, u, T and the temperature-dependent part of the equilibrium,
//     G0_k = rho C0_k - 1 per shell (where theta-terms cancel near T = 0.5),
//     in a "wide" type: FP64, or double-float on the FP32 pipes;
//   * the velocity-dependent part of each population pair and the relaxation
//     in FP32, with d' = (1 - omega) d + omega w (rho P - 1).
// Layout and step sequence are those of the FP64 kernels (d2q37_kernels.cu)
// with 32 halo rows so FP32 columns stay 128-byte aligned.
#include <cuda_runtime.h>

#include "d2q37_launch.h"
#include "dfloat.cuh"

namespace d2q37 {

__constant__ ShellConsts32 c_shell32;

namespace {

constexpr int kBlockY = 128;

// Resident blocks of 128 threads per SM requested for the FP32 site kernels:
// 6 caps registers at 80 (20 bytes of spills per thread) and gives 24 warps
// per SM to hide the memory latency; on GB300 the 2048 x 8192 fused step ran
// at 19.9 G sites/s against 19.5 with 5 (96 registers) and 19.8 with 7.
#ifndef D2Q37_FP32_MIN_BLOCKS
#define D2Q37_FP32_MIN_BLOCKS 6
#endif

template <class P>  // StepParams or BatchGeo32 (NY, Hy)
__device__ __forceinline__ long long site_index(const P& p, int x, int y) {
  return (long long)(x + kHx) * p.NY + (y + p.Hy);
}

// ---- the wide type: FP64 or double-float, behind one set of names ----------

struct WideF64 {
  using T = double;
  static __device__ __forceinline__ T from_fixed(long long v, int e) { return (double)v * exp2_d(e); }
  static __device__ __forceinline__ double exp2_d(int e) { return __hiloint2double((e + 1023) << 20, 0); }
  static __device__ __forceinline__ T c(double hi, float, float) { return hi; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T add(T a, float b) { return a + (double)b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T mul(T a, float b) { return a * (double)b; }
  static __device__ __forceinline__ T rcp(T a) { return 1.0 / a; }
  static __device__ __forceinline__ float fixed_to_float(long long v, int e) { return (float)from_fixed(v, e); }
  static __device__ __forceinline__ float tof(T a) { return (float)a; }
  // K0 + x2 (K1 + x2 K2) rounded to float
  static __device__ __forceinline__ float quad(T K0, T K1, T K2, double x2, float, float) {
    return (float)fma(x2, fma(x2, K2, K1), K0);
  }
};

struct WideDF {
  using T = dfloat;
  static __device__ __forceinline__ T from_fixed(long long v, int e) { return df_from_int64(v, e); }
  static __device__ __forceinline__ T c(double, float hi, float lo) { return {hi, lo}; }
  // about 44 bits: far more than the ~30 the FP32-storage step needs here
  static __device__ __forceinline__ T add(T a, T b) { return df_add_fast(a, b); }
  static __device__ __forceinline__ T add(T a, float b) { return df_add(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return df_add_fast(a, df_neg(b)); }
  static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
  static __device__ __forceinline__ T mul(T a, float b) { return df_mul(a, b); }
  static __device__ __forceinline__ T rcp(T a) { return df_rcp_fast(a); }
  static __device__ __forceinline__ float fixed_to_float(long long v, int e) { return float_from_int64(v, e); }
  static __device__ __forceinline__ float tof(T a) { return df_to_float(a); }
  static __device__ __forceinline__ float quad(T K0, T K1, T K2, double, float x2h, float x2l) {
    return df_to_float(df_quad(K0, K1, K2, {x2h, x2l}));
  }
};

// ---- moment sums of the stored deviations in integer arithmetic ------------

// Fast path (|d| < 1.5 at every population): each deviation is split with two
// float additions of "magic" constants into d ~ (hi 2^22 + lo) 2^-43 with
// integers |hi| < 2^22, |lo| <= 2^21 (error <= 2^-44, none at all for
// |d| >= 2^-20): t1 = d + 6 has an ulp of 2^-21, so its bit pattern minus that
// of 6 is hi = round(d 2^21) and d - (t1 - 6) is exact; the remainder gets the
// same treatment around 1.5 2^-20 (ulp 2^-43).  The moment sums (37 terms,
// weights |c|^2 <= 10) are then exact sums of 32-bit integers, all on the
// integer and FP32 pipes (a float-to-int64 conversion would use the FP64 pipe).
// Other sites (|d| >= 2, non-finite) take the exact 64-bit conversion.
constexpr int kFixExp = -43;

struct Sums {
  long long s, jx, jy, e;  // sum d, sum cx d, sum cy d, sum |c|^2 d on the grid 2^ex
  int ex;
  bool ok;
};

struct Split {
  int hi, lo;
};

__device__ __forceinline__ Split split_deviation(float v) {
  const float m1 = 6.0f, m2 = 0x1.8p-20f;
  const float t1 = __fadd_rn(v, m1);
  const float r = __fsub_rn(v, __fsub_rn(t1, m1));
  const float t2 = __fadd_rn(r, m2);
  return {__float_as_int(t1) - __float_as_int(m1), __float_as_int(t2) - __float_as_int(m2)};
}

// The same split for the two populations of a pair at once, with the
// packed FP32 instructions of sm_100+ (two lanes per instruction issue;
// the arithmetic, and so the result, is that of split_deviation).
__device__ __forceinline__ void split_pair(float vp, float vm, Split& sp, Split& sm) {
  const float m1 = 6.0f, m2 = 0x1.8p-20f;
  const float2 v = make_float2(vp, vm);
  const float2 t1 = __fadd2_rn(v, make_float2(m1, m1));
  const float2 u = __fadd2_rn(t1, make_float2(-m1, -m1));
  const float2 r = __ffma2_rn(u, make_float2(-1.0f, -1.0f), v);  // v - u, exact
  const float2 t2 = __fadd2_rn(r, make_float2(m2, m2));
  sp = {__float_as_int(t1.x) - __float_as_int(m1), __float_as_int(t2.x) - __float_as_int(m2)};
  sm = {__float_as_int(t1.y) - __float_as_int(m1), __float_as_int(t2.y) - __float_as_int(m2)};
}

__device__ __forceinline__ long long join(int hi, int lo) { return (long long)hi * (1LL << 22) + lo; }

__device__ __forceinline__ Sums deviation_sums_wide(const float (&d)[kQ]) {
  // |d| < 16: d 2^43 is an integer below 2^47 for |d| >= 2^-20; sums < 2^63
  Sums r;
  r.ex = kFixExp;
  long long sh[kShells];
  sh[0] = __float2ll_rn(d[0] * 0x1p43f);
#pragma unroll
  for (int k = 1; k < kShells; ++k) sh[k] = 0;
  long long jx = 0, jy = 0;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const long long vp = __float2ll_rn(d[1 + 2 * p] * 0x1p43f);
    const long long vm = __float2ll_rn(d[2 + 2 * p] * 0x1p43f);
    sh[pair_shell(p)] += vp + vm;
    jx += pair_cx(p) * (vp - vm);
    jy += pair_cy(p) * (vp - vm);
  }
  long long s = sh[0], e = 0;
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    s += sh[k];
    e += shell_c2(k) * sh[k];
  }
  r.s = s;
  r.jx = jx;
  r.jy = jy;
  r.e = e;
  return r;
}

__device__ __forceinline__ Sums deviation_sums(const float (&d)[kQ]) {
  float amax = 0.0f;
#pragma unroll
  for (int l = 0; l < kQ; ++l) amax = fmaxf(amax, fabsf(d[l]));
  if (!(amax < 1.5f)) {  // keeps d + 6 inside [4, 8) after rounding
    Sums r = deviation_sums_wide(d);
    r.ok = amax < 16.0f;  // false for NaN
    return r;
  }
  int sh_hi[kShells], sh_lo[kShells];
  {
    const Split v = split_deviation(d[0]);
    sh_hi[0] = v.hi;
    sh_lo[0] = v.lo;
  }
#pragma unroll
  for (int k = 1; k < kShells; ++k) sh_hi[k] = sh_lo[k] = 0;
  int jx_hi = 0, jx_lo = 0, jy_hi = 0, jy_lo = 0;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    Split vp, vm;
    split_pair(d[1 + 2 * p], d[2 + 2 * p], vp, vm);
    const int k = pair_shell(p);
    sh_hi[k] += vp.hi + vm.hi;
    sh_lo[k] += vp.lo + vm.lo;
    const int dh = vp.hi - vm.hi, dl = vp.lo - vm.lo;
    jx_hi += pair_cx(p) * dh;
    jx_lo += pair_cx(p) * dl;
    jy_hi += pair_cy(p) * dh;
    jy_lo += pair_cy(p) * dl;
  }
  int s_hi = sh_hi[0], s_lo = sh_lo[0], e_hi = 0, e_lo = 0;
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    s_hi += sh_hi[k];
    s_lo += sh_lo[k];
    e_hi += shell_c2(k) * sh_hi[k];
    e_lo += shell_c2(k) * sh_lo[k];
  }
  Sums r;
  r.ok = true;
  r.ex = kFixExp;
  r.s = join(s_hi, s_lo);
  r.jx = join(jx_hi, jx_lo);
  r.jy = join(jy_hi, jy_lo);
  r.e = join(e_hi, e_lo);
  return r;
}

// ---- one site ---------------------------------------------------------------

// Float value of an integer sum on the grid 2^ex.
template <class W>
__device__ __forceinline__ float fixed_to_float(long long v, int ex) {
  return W::fixed_to_float(v, ex);
}

// BGK collision of one site in deviation form:
//   d_l' = (1 - omega) d_l + omega w_l (rho P_l - 1),
//   rho P - 1 = G0_k + rho b (C2_k + b/24) +- rho a (C1_k + b/6), b = a^2,
// with the shifted fields of Eq. MASTERSHIFT3; G0_k = rho C0_k - 1 is
// written as K0 + x2_k (K1 + x2_k K2) (C0 is quadratic in x2 = |xi|^2).
//
// Which quantities need more than FP32: with d stored to 2^-24 of itself,
// the result needs errors of that order.  rho and E = sum |xi|^2 f are O(1)
// sums whose small differences matter (T, the energy change), and G0_k
// cancels terms of size ~10 near T = 0.5: those take the wide type (K0..K2
// in their theta-parts, G0_k, rho, E, T).  The velocity (|u| << 1) enters
// only through a = xi.u_bar and q = |u_bar|^2, whose FP32 errors are scaled
// down by |u|, and the q-parts of K0, K1 are ~q theta: FP32.
// P: StepParams, or BatchGeo32 (the same collision fields)
template <class W, class P>
__device__ __forceinline__ void collide_site32(float (&d)[kQ], const P& p) {
  using T = typename W::T;
  const ShellConsts32& c = c_shell32;
  const Sums sm = deviation_sums(d);
  T S, Ec;  // sum d (= rho - 1) and sum |c|^2 d
  float jx, jy;
  if (sm.ok) {
    S = W::from_fixed(sm.s, sm.ex);
    Ec = W::from_fixed(sm.e, sm.ex);
    jx = fixed_to_float<W>(sm.jx, sm.ex);
    jy = fixed_to_float<W>(sm.jy, sm.ex);
  } else {  // a deviation of 16 or more (or non-finite): FP32 sums
    float s = 0.f, e = 0.f;
    jx = jy = 0.f;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      s += d[l];
      jx += vel_cx(l) * d[l];
      jy += vel_cy(l) * d[l];
      e += (vel_cx(l) * vel_cx(l) + vel_cy(l) * vel_cy(l)) * d[l];
    }
    S = W::c(s, s, 0.0f);
    Ec = W::c(e, e, 0.0f);
  }
  // rho = 1 + sum d, rho u = s sum c d, E = 2 + s^2 sum |c|^2 d, 2 rho T = E - rho |u|^2
  // (sum_l w_l = 1, sum_l w_l c_l = 0, sum_l w_l |xi_l|^2 = D = 2 by the quadrature)
  const T rho = W::add(S, 1.0f);
  const T inv = W::rcp(rho);
  const float rho_f = W::tof(rho);
  const float inv_f = W::tof(inv);
  const float ux = c.s_hi * jx * inv_f;
  const float uy = c.s_hi * jy * inv_f;
  const T E = W::add(W::mul(W::c(c.s2, c.s2_hi, c.s2_lo), Ec), 2.0f);
  const T half_T = W::add(W::mul(E, inv), -(ux * ux + uy * uy));  // 2 T
  // theta = T_bar - 1 = T - tau^2 g^2 / D - 1
  const T th = W::add(W::mul(half_T, 0.5f), W::c(p.theta_shift, p.theta_shift_df[0], p.theta_shift_df[1]));
  const float th_f = W::tof(th);
  const float uby = uy + p.uy_shift_df[0];
  const float q = fmaf(ux, ux, uby * uby);
  const T rth = W::mul(rho, th);
  const T rth2 = W::mul(rth, th);
  // rho C0 - 1 = [S - rho theta + rho theta^2 + rho (q (q/8 - 1/2) + theta q)]
  //            + x2 [rho theta / 2 - rho theta^2 - rho theta q / 4] + x2^2 [rho theta^2 / 8]
  const float rq = rho_f * q;
  const T K0 = W::add(W::add(W::sub(S, rth), rth2), rq * (fmaf(0.125f, q, -0.5f) + th_f));
  const T K1 = W::add(W::sub(W::mul(rth, 0.5f), rth2), -0.25f * rq * th_f);
  const T K2 = W::mul(rth2, 0.125f);
  // energy change of the collision in c-units: sum |c|^2 (d' - d) =
  // omega (E_eq - E) / s^2, E_eq = rho (|u_bar|^2 + D T_bar) = 2 (rho + rho theta) + rho q
  const float target_e =
      p.omega_f * c.inv_s2_hi * W::tof(W::add(W::sub(W::mul(W::add(rho, rth), 2.0f), E), rq));
  float G0[kShells];
#pragma unroll
  for (int k = 0; k < kShells; ++k) G0[k] = W::quad(K0, K1, K2, c.x2[k], c.x2_hi[k], c.x2_lo[k]);
  const float sux = c.s_hi * ux, suy = c.s_hi * uby;
  const float B1 = fmaf(-0.5f, q, 1.0f);
  const float B2 = fmaf(-0.25f, q, 0.5f);
  const float keep = p.keep_f;
  // Collision conserves mass exactly (sum_l w_l P_l = 1).  With FP32 weights
  // and rounding that sum is off by ~1e-8 per site and step, always with the
  // same sign, which would make the mass drift (likewise the energy).  So the
  // rest population takes the mass-conserving value
  // d_0' = d_0 - sum_{l>0} (d_l' - d_l), equal to (1 - omega) d_0 +
  // omega w_0 G0_0 in exact arithmetic.
  float moved = 0.0f, moved_e = 0.0f;
#pragma unroll
  for (int k = 1; k < kShells; ++k) {
    float2 moved_k2 = make_float2(0.0f, 0.0f);  // per lane: the +c and the -c populations
    const float ow = p.omega_f * c.w[k];
    const float rC1 = rho_f * fmaf(th_f, c.delta[k], B1);
    const float rC2 = rho_f * fmaf(th_f, c.eps[k], B2);
    const float r6 = rho_f * (1.0f / 6.0f), r24 = rho_f * (1.0f / 24.0f);
#pragma unroll
    for (int pr = 0; pr < kPairs; ++pr) {
      if (pair_shell(pr) != k) continue;
      const int cx = pair_cx(pr), cy = pair_cy(pr);
      const float a = cx == 0 ? cy * suy : (cy == 0 ? cx * sux : fmaf((float)cx, sux, cy * suy));
      const float b = a * a;
      // (even, odd) = (b (b/24 + C2), a (b/6 + C1)) rho, in one packed FMA and multiply
      const float2 eo = __fmul2_rn(make_float2(b, a), __ffma2_rn(make_float2(b, b), make_float2(r24, r6),
                                                               make_float2(rC2, rC1)));
      const float ge = G0[k] + eo.x;
      // (G0 + even + odd, G0 + even - odd), exact sign flips
      const float2 gpm = __ffma2_rn(make_float2(eo.y, eo.y), make_float2(1.0f, -1.0f), make_float2(ge, ge));
      const float2 dd = make_float2(d[1 + 2 * pr], d[2 + 2 * pr]);
      const float2 nn = __ffma2_rn(make_float2(keep, keep), dd, __fmul2_rn(make_float2(ow, ow), gpm));
      moved_k2 = __fadd2_rn(moved_k2, __ffma2_rn(dd, make_float2(-1.0f, -1.0f), nn));  // += nn - dd
      d[1 + 2 * pr] = nn.x;
      d[2 + 2 * pr] = nn.y;
    }
    const float moved_k = moved_k2.x + moved_k2.y;
    moved += moved_k;
    moved_e = fmaf((float)shell_c2(k), moved_k, moved_e);
  }
  // Same for energy: the rounding residue of sum |c|^2 (d' - d) goes evenly
  // to the four |c| = 1 populations (momentum unchanged), then the rest
  // population restores mass.
  const float fix = 0.25f * (target_e - moved_e);
#pragma unroll
  for (int l = 1; l <= 4; ++l) d[l] += fix;
  d[0] -= moved + 4.0f * fix;
}

// Site fields (FP64) from the stored deviations, for lbm_fields.
__device__ __forceinline__ void fields_of_site32(const float (&d)[kQ], double& rho, double& ux, double& uy,
                                                 double& T) {
  const ShellConsts32& c = c_shell32;
  const Sums sm = deviation_sums(d);
  double S, jx, jy, Ec;
  if (sm.ok) {
    const double sc = __hiloint2double((sm.ex + 1023) << 20, 0);
    S = (double)sm.s * sc;
    jx = (double)sm.jx * sc;
    jy = (double)sm.jy * sc;
    Ec = (double)sm.e * sc;
  } else {
    S = jx = jy = Ec = 0.0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      S += d[l];
      jx += vel_cx(l) * (double)d[l];
      jy += vel_cy(l) * (double)d[l];
      Ec += (vel_cx(l) * vel_cx(l) + vel_cy(l) * vel_cy(l)) * (double)d[l];
    }
  }
  rho = 1.0 + S;
  const double inv = 1.0 / rho;
  ux = c.s * jx * inv;
  uy = c.s * jy * inv;
  T = 0.5 * ((2.0 + c.s2 * Ec) * inv - (ux * ux + uy * uy));
}

// Halo images as in the FP64 store_site.
template <class P>
__device__ __forceinline__ void store_site32(float* __restrict__ dst, const P& p, int x, int y,
                                             const float (&d)[kQ]) {
  if (x >= kHx && x < p.Lx - kHx && (!p.periodic_y || (y >= kHx && y < p.Ly - kHx))) {
    float* q = dst + (int)site_index(p, x, y);  // no halo image: the common case
#pragma unroll
    // streaming stores (evict-first): the next step reads these rows from
    // DRAM anyway; 0.8378 -> 0.8293 ms per 2048 x 8192 step (streaming loads
    // instead: 0.8931, the pull's rows are shared by neighbouring warps)
    for (int l = 0; l < kQ; ++l) __stcs(q + l * p.plane, d[l]);
    return;
  }
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
      float* q = dst + (int)site_index(p, xs[a], ys[b]);  // a plane holds < 2^31 elements
#pragma unroll
      for (int l = 0; l < kQ; ++l) q[l * p.plane] = d[l];
    }
}

// Wall bc in deviation form (rows 0..2 from each wall), in FP32 like the
// stored values (an FP64 version made the wall warps of small lattices the
// slowest ones).  The missing deviations are d_l = (rho_w - 1) fw_l + (fw_l - w_l)
// with FP32 constants fw_l and fw_l - w_l.  rho_w - 1 is solved from the mass
// balance those rounded constants actually give: with D = sum_M fw_l and
// B = sum_M (fw_l - w_l) summed exactly, the missing mass sum_M d_l equals the
// leaving mass sum_O d_l + sum_O w_l - sum_M w_l when
//   rho_w - 1 = (sum_O d - E) / D,   E = B - sum_O w + sum_M w,
// with E and 1/D carried as (hi, lo) float pairs, so that no rounding of a
// constant biases the wall's mass the same way every step.
template <class P>
__device__ __forceinline__ float wall_rho_minus_1(const float* __restrict__ src, const P& p, int x,
                                                  int wall) {
  float out_d = 0.0f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int y = wall ? p.Ly - 1 - r : r;
    const int i = (int)site_index(p, x, y);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cy = vel_cy(l);
      if (wall ? (cy > r) : (cy < -r)) out_d += (src + l * p.plane)[i];
    }
  }
  const float t = (out_d - p.wall_e32[wall][0]) - p.wall_e32[wall][1];
  return fmaf(t, p.wall_inv32[wall][0], t * p.wall_inv32[wall][1]);
}

template <class P>
__device__ __forceinline__ float missing32(const P& p, float rho_w_minus_1, int wall, int l) {
  return fmaf(rho_w_minus_1, p.fw32[wall][l], p.fwmw32[wall][l]);
}

__global__ void __launch_bounds__(256) wrap32_kernel(float* __restrict__ buf, StepParams p) {
  const int rows_a = p.periodic_y ? p.Ly + 2 * kHx : p.Ly;
  const int y0 = p.periodic_y ? -kHx : 0;
  const long long n_a = (long long)kQ * 6 * rows_a;
  const long long n_b = p.periodic_y ? (long long)kQ * p.Lx * 6 : 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_a + n_b;
       t += (long long)gridDim.x * blockDim.x) {
    int l, xd, yd, xs, ys;
    if (t < n_a) {
      const int yy = (int)(t % rows_a);
      const int h = (int)((t / rows_a) % 6);
      l = (int)(t / (6LL * rows_a));
      xd = h < 3 ? h - 3 : p.Lx + h - 3;
      xs = h < 3 ? p.Lx + h - 3 : h - 3;
      yd = y0 + yy;
      ys = yd < 0 ? yd + p.Ly : (yd >= p.Ly ? yd - p.Ly : yd);
    } else {
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

// One site of the fused step (pull, wall bc on the wall bands, collide,
// store with halo images).
template <class W, class P>
__device__ __forceinline__ void fused_site32(const float* __restrict__ src, float* __restrict__ dst, const P& p,
                                             int x, int y) {
  // the site's pointer once per thread; each population at an offset that is
  // the same for the whole block (l plane - cx NY - cy)
  const float* q = src + (int)site_index(p, x, y);
  float d[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) d[l] = q[l * p.plane - vel_cx(l) * p.NY - vel_cy(l)];
  if (!p.periodic_y && (y < 3 || y >= p.Ly - 3)) {
    const int wall = y >= p.Ly - 3;
    const int r = wall ? p.Ly - 1 - y : y;
    const float rho_w_m1 = wall_rho_minus_1(src, p, x, wall);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cy = vel_cy(l);
      if (wall ? (cy < -r) : (cy > r)) d[l] = missing32(p, rho_w_m1, wall, l);
    }
  }
  collide_site32<W>(d, p);
  store_site32(dst, p, x, y, d);
}

template <class W>
__global__ void __launch_bounds__(kBlockY, D2Q37_FP32_MIN_BLOCKS) fused32_kernel(const float* __restrict__ src,
                                                                                 float* __restrict__ dst,
                                                                                 StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  fused_site32<W>(src, dst, p, x, y);
}

// Many lattices in one launch (see batch_fused_kernel of the FP64 kernels).
template <class W, int BY>
__global__ void __launch_bounds__(BY, (D2Q37_FP32_MIN_BLOCKS * 128) / BY) batch_fused32_kernel(
    const BatchEntry* __restrict__ tab, const int* __restrict__ tile_entry, int n, long long tiles, int parity) {
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const BatchEntry& e = tab[tile_entry ? tile_entry[t] : batch_entry_of(tab, n, t)];
    const int local = (int)(t - e.tile0);  // tiles of one lattice < 2^31: 32-bit division
    const int x = local / e.ytiles;
    const int y = (local - x * e.ytiles) * BY + threadIdx.x;
    const int c = e.cur ^ parity;
    if (y < e.p.Ly) fused_site32<W>((const float*)e.buf[c], (float*)e.buf[c ^ 1], e.p, x, y);
  }
}

// Many lattices in one launch, one block per tile (a column x BY rows, x
// fastest, as fused32_kernel orders its blocks), no grid-stride loop: each
// lattice's geometry and collision constants come from the launch's parameter
// space (BatchLaunch32), its wall constants from its entry of the table.  The
// per-site arithmetic is fused32_kernel's.
static_assert(sizeof(BatchLaunch32) <= 32764, "BatchLaunch32 must fit the kernel parameter space");

template <class W, int BY>
__global__ void __launch_bounds__(BY, (D2Q37_FP32_MIN_BLOCKS * 128) / BY)
    batch_split32_kernel(const __grid_constant__ BatchLaunch32 L, const int* __restrict__ tile_entry, int parity) {
  const int b = blockIdx.x;
  // the lattice's parameters in shared memory: the blocks of an SM serve
  // different lattices, whose parameter slices would crowd the constant cache
  __shared__ BatchGeo32 g;
  static_assert(sizeof(BatchGeo32) % sizeof(int) == 0, "BatchGeo32 is copied as ints");
  {
    const int* from = (const int*)&L.g[tile_entry[b]];
    for (int k = threadIdx.x; k < (int)(sizeof(BatchGeo32) / sizeof(int)); k += BY) ((int*)&g)[k] = from[k];
  }
  __syncthreads();
  const int local = b - g.tile0;
  const int yt = local / g.Lx;
  const int x = local - yt * g.Lx;
  const int y = yt * BY + threadIdx.x;
  if (y >= g.Ly) return;
  const int c = g.cur ^ parity;
  fused_site32<W>((const float*)g.buf[c], (float*)g.buf[c ^ 1], g, x, y);
}

__global__ void __launch_bounds__(kBlockY) propagate32_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                              StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const long long i = site_index(p, x, y);
#pragma unroll
  for (int l = 0; l < kQ; ++l) dst[l * p.plane + i] = src[l * p.plane + i - vel_cx(l) * p.NY - vel_cy(l)];
}

__global__ void __launch_bounds__(128) bc32_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                   StepParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * p.Lx) return;
  const int wall = t >= p.Lx;
  const int x = t - wall * p.Lx;
  const float rho_w_m1 = wall_rho_minus_1(src, p, x, wall);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int y = wall ? p.Ly - 1 - r : r;
    const long long i = site_index(p, x, y);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cy = vel_cy(l);
      if (wall ? (cy < -r) : (cy > r)) dst[l * p.plane + i] = missing32(p, rho_w_m1, wall, l);
    }
  }
}

template <class W>
__global__ void __launch_bounds__(kBlockY, D2Q37_FP32_MIN_BLOCKS) collide32_kernel(float* __restrict__ buf,
                                                                                   StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const long long i = site_index(p, x, y);
  float d[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) d[l] = buf[l * p.plane + i];
  collide_site32<W>(d, p);
  store_site32(buf, p, x, y, d);
}

// Fields in FP64 from the stored deviations.
__global__ void __launch_bounds__(kBlockY) fields32_kernel(const float* __restrict__ buf, double* __restrict__ rho,
                                                           double* __restrict__ u, double* __restrict__ T,
                                                           StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  const long long i = site_index(p, x, y);
  float d[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) d[l] = buf[l * p.plane + i];
  double r, ux, uy, t;
  fields_of_site32(d, r, ux, uy, t);
  const long long o = (long long)x * p.Ly + y;
  const long long n = (long long)p.Lx * p.Ly;
  rho[o] = r;
  u[o] = ux;
  u[n + o] = uy;
  T[o] = t;
}

__global__ void __launch_bounds__(kBlockY) plane_to_frame32_kernel(float* __restrict__ frame,
                                                                   const double* __restrict__ plane, int l,
                                                                   StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  frame[l * p.plane + site_index(p, x, y)] =
      (float)(plane[(long long)x * p.Ly + y] - c_shell32.w64[vel_shell(l)]);
}

__global__ void __launch_bounds__(kBlockY) frame32_to_plane_kernel(double* __restrict__ plane,
                                                                   const float* __restrict__ frame, int l,
                                                                   StepParams p) {
  const int x = blockIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.x;
  if (y >= p.Ly) return;
  plane[(long long)x * p.Ly + y] = c_shell32.w64[vel_shell(l)] + (double)frame[l * p.plane + site_index(p, x, y)];
}

dim3 site_grid(const StepParams& p) { return dim3(p.Lx, (p.Ly + kBlockY - 1) / kBlockY); }

int done(int n) { return cudaGetLastError() == cudaSuccess ? n : -1; }

}  // namespace

int launch_plane_to_frame32(float* frame, const double* plane, int l, const StepParams& p, cudaStream_t stream) {
  plane_to_frame32_kernel<<<site_grid(p), kBlockY, 0, stream>>>(frame, plane, l, p);
  return done(1);
}

int launch_frame32_to_plane(double* plane, const float* frame, int l, const StepParams& p, cudaStream_t stream) {
  frame32_to_plane_kernel<<<site_grid(p), kBlockY, 0, stream>>>(plane, frame, l, p);
  return done(1);
}

cudaError_t upload_shell_consts32(const ShellConsts32& c) { return cudaMemcpyToSymbol(c_shell32, &c, sizeof(c)); }

int launch_wrap32(float* buf, const StepParams& p, cudaStream_t stream) {
  const long long n = (long long)kQ * 6 * (p.periodic_y ? p.Ly + 2 * kHx : p.Ly) +
                      (p.periodic_y ? (long long)kQ * p.Lx * 6 : 0);
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  wrap32_kernel<<<(unsigned)blocks, 256, 0, stream>>>(buf, p);
  return done(1);
}

int launch_propagate32(const float* src, float* dst, const StepParams& p, cudaStream_t stream) {
  propagate32_kernel<<<site_grid(p), kBlockY, 0, stream>>>(src, dst, p);
  return done(1);
}

int launch_bc32(const float* src, float* dst, const StepParams& p, cudaStream_t stream) {
  bc32_kernel<<<(2 * p.Lx + 127) / 128, 128, 0, stream>>>(src, dst, p);
  return done(1);
}

int launch_collide32(float* buf, const StepParams& p, bool wide_fp64, cudaStream_t stream) {
  if (wide_fp64)
    collide32_kernel<WideF64><<<site_grid(p), kBlockY, 0, stream>>>(buf, p);
  else
    collide32_kernel<WideDF><<<site_grid(p), kBlockY, 0, stream>>>(buf, p);
  return done(1);
}

int launch_fused32(const float* src, float* dst, const StepParams& p, bool wide_fp64, cudaStream_t stream) {
  if (wide_fp64)
    fused32_kernel<WideF64><<<site_grid(p), kBlockY, 0, stream>>>(src, dst, p);
  else
    fused32_kernel<WideDF><<<site_grid(p), kBlockY, 0, stream>>>(src, dst, p);
  return done(1);
}

template <class W, int BY>
int batch32_launch(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity, int grid,
                   cudaStream_t stream) {
  batch_fused32_kernel<W, BY><<<grid, BY, 0, stream>>>(tab, tile_entry, n, tiles, parity);
  return done(1);
}

template <class W, int BY>
int batch32_occupancy() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_fused32_kernel<W, BY>, BY, 0);
  return b;
}

int launch_batch_fused32(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity,
                         int block_y, int grid, bool wide_fp64, cudaStream_t stream) {
  switch (block_y) {
    case 64: return wide_fp64 ? batch32_launch<WideF64, 64>(tab, tile_entry, n, tiles, parity, grid, stream)
                              : batch32_launch<WideDF, 64>(tab, tile_entry, n, tiles, parity, grid, stream);
    case 128: return wide_fp64 ? batch32_launch<WideF64, 128>(tab, tile_entry, n, tiles, parity, grid, stream)
                               : batch32_launch<WideDF, 128>(tab, tile_entry, n, tiles, parity, grid, stream);
    case 256: return wide_fp64 ? batch32_launch<WideF64, 256>(tab, tile_entry, n, tiles, parity, grid, stream)
                               : batch32_launch<WideDF, 256>(tab, tile_entry, n, tiles, parity, grid, stream);
    default: return -1;
  }
}

template <class W, int BY>
int split32_launch(const BatchLaunch32& L, const int* tile_entry, int tiles, int parity, cudaStream_t stream) {
  batch_split32_kernel<W, BY><<<tiles, BY, 0, stream>>>(L, tile_entry, parity);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_batch_split32(const BatchLaunch32& L, const int* tile_entry, int tiles, int parity, int block_y,
                         bool wide_fp64, cudaStream_t stream) {
  switch (block_y) {
    case 64: return wide_fp64 ? split32_launch<WideF64, 64>(L, tile_entry, tiles, parity, stream)
                              : split32_launch<WideDF, 64>(L, tile_entry, tiles, parity, stream);
    case 128: return wide_fp64 ? split32_launch<WideF64, 128>(L, tile_entry, tiles, parity, stream)
                               : split32_launch<WideDF, 128>(L, tile_entry, tiles, parity, stream);
    case 256: return wide_fp64 ? split32_launch<WideF64, 256>(L, tile_entry, tiles, parity, stream)
                               : split32_launch<WideDF, 256>(L, tile_entry, tiles, parity, stream);
    default: return -1;
  }
}

int batch32_blocks_per_sm(int block_y, bool wide_fp64) {
  switch (block_y) {
    case 64: return wide_fp64 ? batch32_occupancy<WideF64, 64>() : batch32_occupancy<WideDF, 64>();
    case 128: return wide_fp64 ? batch32_occupancy<WideF64, 128>() : batch32_occupancy<WideDF, 128>();
    case 256: return wide_fp64 ? batch32_occupancy<WideF64, 256>() : batch32_occupancy<WideDF, 256>();
    default: return 0;
  }
}

int launch_fields32(const float* buf, double* rho, double* u, double* T, const StepParams& p, cudaStream_t stream) {
  fields32_kernel<<<site_grid(p), kBlockY, 0, stream>>>(buf, rho, u, T, p);
  return done(1);
}

}  // namespace d2q37
