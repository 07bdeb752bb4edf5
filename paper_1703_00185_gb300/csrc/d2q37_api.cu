// C ABI of the D2Q37 library (declared in include/d2q37.h): handle life
// cycle, device memory layout, step scheduling and host<->device transfers.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/d2q37.h"
#include "d2q37_handle.h"

using namespace d2q37;

namespace {

std::once_flag g_quad_once;
bool g_quad_ok = false;
ShellConsts g_consts;
ShellConsts32 g_consts32;
std::mutex g_dev_mutex;
bool g_dev_ready[256];

// hi + lo split of a double into two floats (hi = nearest float).
void split_df(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

// round((hi + lo) 2^Q) as an unsigned 64-bit integer (0 <= value < 2^64).
unsigned long long fixed_u64(double hi, double lo, int Q) {
  const double H = std::ldexp(hi, Q), L = std::ldexp(lo, Q);
  const double Hr = std::nearbyint(H);
  return (unsigned long long)Hr + (unsigned long long)std::llround((H - Hr) + L);
}

// Constants of the fixed-point equilibrium (see StepParams), from the
// double-double product omega w_k = (c_k hi + c_k lo) 2^E_k.
void fill_fixed_consts(StepParams& sp) {
  const ShellConsts& c = g_consts;
  for (int k = 0; k < kShells; ++k) {
    const double wh = sp.omega * c.w[k];
    const double wl = std::fma(sp.omega, c.w[k], -wh);
    int E;
    std::frexp(wh, &E);  // wh = m 2^E, m in [0.5, 1)
    sp.fx_e[k] = E;
    const double ch = std::ldexp(wh, -E), cl = std::ldexp(wl, -E);
    const double x2 = c.s2 * shell_c2(k);
    const double x2h = x2, x2l = std::fma(c.s2, (double)shell_c2(k), -x2);  // exact: c.s2 times a small integer
    // c x2 and c x2^2 in double-double
    const double p1h = ch * x2h, p1l = std::fma(ch, x2h, -p1h) + (cl * x2h + ch * x2l);
    const double p2h = p1h * x2h, p2l = std::fma(p1h, x2h, -p2h) + (p1l * x2h + p1h * x2l);
    sp.fx_c60[k] = fixed_u64(ch, cl, 60);
    sp.fx_c62[k] = fixed_u64(ch, cl, 62);
    sp.fx_c64[k] = fixed_u64(ch, cl, 64);
    sp.fx_cx2_59[k] = fixed_u64(p1h, p1l, 59);
    sp.fx_cx2_60[k] = fixed_u64(p1h, p1l, 60);
    sp.fx_cx4_55[k] = fixed_u64(p2h, p2l, 55);
    const double q6 = ch / 6.0, q6l = (std::fma(-q6, 6.0, ch) + cl) / 6.0;
    sp.fx_c6[k] = fixed_u64(q6, q6l, 64);  // also (c/24) 2^66: one product serves R3 and R4
    // R0 = K0 c60 + (K1 + 2^63) cx2_59 + K2 cx4_55, R1 = (L0 + 2^63) c62 +
    // (L1 + 2^63) cx2_59, R2 = (M0 + 2^63) c64 + (M1 + 2^63) cx2_60, with
    // corrections for their floors and those of the pair's product each
    // feeds (b t, b R3, b R4; with the conversion's lowest bit for R0): +2 for
    // R0, +1 for R1 and R2; the shell-0 population, K0 c60 alone, needs none
    sp.fx_d0[k] = k == 0 ? 0ull : (sp.fx_cx2_59[k] >> 1) - 2ull;
    sp.fx_d1[k] = (sp.fx_c62[k] >> 1) + (sp.fx_cx2_59[k] >> 1) - 1ull;
    sp.fx_d2[k] = (sp.fx_c64[k] >> 1) + (sp.fx_cx2_60[k] >> 1) - 1ull;
  }
  sp.fx_s62 = fixed_u64(c.s, 0.0, 62);
  sp.fx_s63 = fixed_u64(c.s, 0.0, 63);
  const double s2h = c.s * c.s, s2l = std::fma(c.s, c.s, -s2h);
  sp.fx_s2_63 = fixed_u64(s2h, s2l, 63);
  // the shifted-field constants: tau g_y in Q64 and theta_shift in Q60 (signed)
  sp.fx_on = std::fabs(sp.uy_shift) < 0.35 && sp.theta_shift > -4.0 && sp.theta_shift < 4.0;
  sp.fx_uy_shift = sp.fx_on ? std::llround(std::ldexp(sp.uy_shift, 64)) : 0;
  sp.fx_th_shift = sp.fx_on ? std::llround(std::ldexp(sp.theta_shift, 60)) : 0;
}

void solve_once() {
  double s, w[kShells];
  if (!solve_quadrature(&s, w)) return;
  ShellConsts& c = g_consts;
  c.s = s;
  c.s2 = s * s;
  ShellConsts32& c32 = g_consts32;
  c32.s = c.s;
  c32.s2 = c.s2;
  split_df(c.s, &c32.s_hi, &c32.s_lo);
  split_df(c.s2, &c32.s2_hi, &c32.s2_lo);
  c32.inv_s2 = 1.0 / c.s2;
  split_df(c32.inv_s2, &c32.inv_s2_hi, &c32.inv_s2_lo);
  for (int k = 0; k < kShells; ++k) {
    const double x2 = c.s2 * shell_c2(k);
    c.w[k] = w[k];
    c.alpha[k] = (x2 - 2.0) / 2.0;
    c.beta[k] = (4.0 - x2) / 4.0;
    c.gamma[k] = (x2 * x2 - 8.0 * x2 + 8.0) / 8.0;
    c.delta[k] = (x2 - 4.0) / 2.0;
    c.eps[k] = (x2 - 6.0) / 4.0;
    c32.x2[k] = x2;
    split_df(x2, &c32.x2_hi[k], &c32.x2_lo[k]);
    c32.w64[k] = w[k];
    c32.w[k] = (float)w[k];
    c32.delta[k] = (float)c.delta[k];
    c32.eps[k] = (float)c.eps[k];
  }
  g_quad_ok = true;
}

bool quadrature_ready() {
  std::call_once(g_quad_once, solve_once);
  return g_quad_ok;
}

int ensure_device_consts() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return LBM_ECUDA;
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  if (!g_dev_ready[dev]) {
    if (upload_shell_consts(g_consts) != cudaSuccess) return LBM_ECUDA;
    if (upload_shell_consts32(g_consts32) != cudaSuccess) return LBM_ECUDA;
    g_dev_ready[dev] = true;
  }
  return LBM_OK;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

bool is_fp32(int prec) { return prec != LBM_PRECISION_FP64; }

int halo_rows(int prec) { return is_fp32(prec) ? kHy32 : kHy; }

// Column stride: 128-byte multiples (16 doubles or 32 floats).
int frame_ny(int Ly, int prec) {
  const int q = is_fp32(prec) ? 32 : 16;
  return ((Ly + 2 * halo_rows(prec)) + q - 1) / q * q;
}

size_t elem_bytes(int prec) { return is_fp32(prec) ? sizeof(float) : sizeof(double); }

bool valid_params(int Lx, int Ly, const lbm_params* p) {
  if (!p || Lx < 3 || Ly < 6) return false;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau) || !std::isfinite(p->g0)) return false;
  if (!(p->T_top > 0.0) || !(p->T_bot > 0.0)) return false;
  if (p->precision != LBM_PRECISION_FP64 && p->precision != LBM_PRECISION_FP32_FP64 &&
      p->precision != LBM_PRECISION_FP32_DF)
    return false;
  if (p->kernel != LBM_KERNEL_SEPARATE && p->kernel != LBM_KERNEL_FUSED && p->kernel != LBM_KERNEL_FUSED_SERIAL)
    return false;
  if ((long long)Lx * Ly > (1LL << 34)) return false;
  // one population plane must stay below 2^31 elements (32-bit in-plane offsets)
  if ((long long)(Lx + 2 * kHx) * frame_ny(Ly, p->precision) >= (1LL << 31)) return false;
  return true;
}

size_t buffer_bytes(int Lx, int Ly, int prec) {
  return align256((size_t)kQ * (size_t)(Lx + 2 * kHx) * (size_t)frame_ny(Ly, prec) * elem_bytes(prec));
}

size_t scratch_bytes(int Lx, int Ly) { return align256((size_t)4 * Lx * Ly * sizeof(double)); }

void fill_step_params(lbm_t* h) {
  StepParams& sp = h->sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.Lx = h->Lx;
  sp.Ly = h->Ly;
  sp.NY = h->NY;
  sp.Hy = halo_rows(h->prec);
  sp.periodic_y = h->prm.periodic_y ? 1 : 0;
  sp.plane = (long long)h->NX * h->NY;
  for (int l = 0; l < kQ; ++l) {
    sp.pull_off[l] = (l * sp.plane - kCx[l] * (long long)sp.NY - kCy[l]) * (long long)sizeof(double);
    sp.plane_off[l] = l * sp.plane * (long long)sizeof(double);
  }
  const double tau = h->prm.tau;
  sp.omega = 1.0 / tau;
  sp.one_minus_omega = 1.0 - sp.omega;
  sp.omega_f = (float)sp.omega;
  sp.keep_f = 1.0f - sp.omega_f;  // exact for omega in (0, 2): keep_f + omega_f == 1
  const double gy = -h->prm.g0;
  sp.uy_shift = tau * gy;
  sp.theta_shift = -(tau * tau * gy * gy) / 2.0 - 1.0;
  split_df(sp.uy_shift, &sp.uy_shift_df[0], &sp.uy_shift_df[1]);
  split_df(sp.theta_shift, &sp.theta_shift_df[0], &sp.theta_shift_df[1]);
  fill_fixed_consts(sp);
  const double Tw[2] = {h->prm.T_bot, h->prm.T_top};
  for (int wall = 0; wall < 2; ++wall) {
    equilibrium(g_consts, 1.0, 0.0, 0.0, Tw[wall], sp.fw[wall]);
    for (int l = 0; l < kQ; ++l) {
      sp.fw32[wall][l] = (float)sp.fw[wall][l];
      sp.fwmw32[wall][l] = (float)(sp.fw[wall][l] - g_consts.w[kShellOf[l]]);
    }
    // D, B, sum_M w and sum_O w over the (row, population) pairs of rows 0..2
    double den = 0.0, d32 = 0.0, b32 = 0.0, w_miss = 0.0, w_out = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int l = 0; l < kQ; ++l) {
        const bool missing = wall ? (kCy[l] < -r) : (kCy[l] > r);
        const bool leaving = wall ? (kCy[l] > r) : (kCy[l] < -r);
        if (missing) {
          den += sp.fw[wall][l];
          d32 += sp.fw32[wall][l];
          b32 += sp.fwmw32[wall][l];
          w_miss += g_consts.w[kShellOf[l]];
        }
        if (leaving) w_out += g_consts.w[kShellOf[l]];
      }
    sp.inv_denom[wall] = 1.0 / den;
    split_df(b32 - w_out + w_miss, &sp.wall_e32[wall][0], &sp.wall_e32[wall][1]);
    split_df(1.0 / d32, &sp.wall_inv32[wall][0], &sp.wall_inv32[wall][1]);
  }
}

int check(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

cudaEvent_t pooled_event(lbm_t* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Enqueue one launcher; with timing on, bracket it with an event pair.
template <typename F>
int run_kernel(lbm_t* h, int kind, F&& launcher) {
  cudaEvent_t start = nullptr, stop = nullptr;
  if (h->timing) {
    start = pooled_event(h);
    stop = pooled_event(h);
    if (!start || !stop || cudaEventRecord(start, h->stream) != cudaSuccess) return LBM_ECUDA;
  }
  const int n = launcher();
  if (n < 0) return LBM_ECUDA;
  h->launches += n;
  if (h->timing) {
    if (cudaEventRecord(stop, h->stream) != cudaSuccess) return LBM_ECUDA;
    h->pending.push_back({kind, start, stop});
    h->kind_launches[kind] += n;
  }
  return LBM_OK;
}

// Fold recorded event pairs into the per-kind totals (stream already synced).
int drain_timing(lbm_t* h) {
  int rc = LBM_OK;
  for (auto& p : h->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.start, p.stop) != cudaSuccess) rc = LBM_ECUDA;
    h->kind_ms[p.kind] += ms;
    h->event_pool.push_back(p.start);
    h->event_pool.push_back(p.stop);
  }
  h->pending.clear();
  return rc;
}

// ---- kernel dispatch by storage precision -----------------------------------

int k_wrap(lbm_t* h, void* b) {
  return is_fp32(h->prec) ? launch_wrap32((float*)b, h->sp, h->stream) : launch_wrap((double*)b, h->sp, h->stream);
}

int k_propagate(lbm_t* h, const void* s, void* d) {
  return is_fp32(h->prec) ? launch_propagate32((const float*)s, (float*)d, h->sp, h->stream)
                          : launch_propagate((const double*)s, (double*)d, h->sp, h->stream);
}

int k_bc(lbm_t* h, const void* s, void* d) {
  return is_fp32(h->prec) ? launch_bc32((const float*)s, (float*)d, h->sp, h->stream)
                          : launch_bc((const double*)s, (double*)d, h->sp, h->stream);
}

int k_collide(lbm_t* h, void* b) {
  return is_fp32(h->prec) ? launch_collide32((float*)b, h->sp, h->prec == LBM_PRECISION_FP32_FP64, h->stream)
                          : launch_collide((double*)b, h->sp, h->stream);
}

int k_fused(lbm_t* h, const void* s, void* d) {
  return is_fp32(h->prec)
             ? launch_fused32((const float*)s, (float*)d, h->sp, h->prec == LBM_PRECISION_FP32_FP64, h->stream)
             : launch_fused((const double*)s, (double*)d, h->sp, h->stream, h->prm.kernel != LBM_KERNEL_FUSED_SERIAL);
}

int k_fields(lbm_t* h, const void* b, double* rho, double* u, double* T) {
  return is_fp32(h->prec) ? launch_fields32((const float*)b, rho, u, T, h->sp, h->stream)
                          : launch_fields((const double*)b, rho, u, T, h->sp, h->stream);
}

int k_init(lbm_t* h, void* b, const double* T) {
  return is_fp32(h->prec) ? launch_init_equilibrium32((float*)b, T, h->sp, h->stream)
                          : launch_init_equilibrium((double*)b, T, h->sp, h->stream);
}

int setup_handle(lbm_t* h, int Lx, int Ly, const lbm_params* p, void* mem, cudaStream_t stream) {
  h->Lx = Lx;
  h->Ly = Ly;
  h->prec = p->precision;
  h->elem = elem_bytes(h->prec);
  h->NX = Lx + 2 * kHx;
  h->NY = frame_ny(Ly, h->prec);
  h->prm = *p;
  const size_t bb = buffer_bytes(Lx, Ly, h->prec);
  char* base = (char*)mem;
  h->buf[0] = base;
  h->buf[1] = base + bb;
  h->scratch = (double*)(base + 2 * bb);
  h->cur = 0;
  h->stream = stream;
  fill_step_params(h);
  // halo rows must read as zero (FP64) or as f = w (FP32 deviations): the pull
  // takes the populations a wall replaces from there
  int rc = check(cudaMemsetAsync(base, 0, 2 * bb, stream));
  if (rc == LBM_OK) rc = check(cudaStreamSynchronize(stream));
  return rc;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the finaliser applied to
// state v + 0x9e3779b97f4a7c15.
uint64_t splitmix64(uint64_t v) {
  uint64_t z = v + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

int step_once(lbm_t* h, int phases, bool fused) {
  int rc = LBM_OK;
  if (phases & LBM_PHASE_PROPAGATE) {
    void* src = h->buf[h->cur];
    void* dst = h->buf[1 - h->cur];
    if (!h->halo_valid) {
      rc = run_kernel(h, LBM_KIND_WRAP, [&] { return k_wrap(h, src); });
      if (rc) return rc;
      h->halo_valid = true;
    }
    if (fused) {
      rc = run_kernel(h, LBM_KIND_FUSED, [&] { return k_fused(h, src, dst); });
      if (rc) return rc;
      h->cur = 1 - h->cur;  // fused writes the halo images of dst
      return LBM_OK;
    }
    rc = run_kernel(h, LBM_KIND_PROPAGATE, [&] { return k_propagate(h, src, dst); });
    if (rc) return rc;
    if ((phases & LBM_PHASE_BC) && !h->prm.periodic_y) {
      rc = run_kernel(h, LBM_KIND_BC, [&] { return k_bc(h, src, dst); });
      if (rc) return rc;
    }
    h->cur = 1 - h->cur;
    h->halo_valid = false;  // propagate writes physical sites only
  }
  if (phases & LBM_PHASE_COLLIDE) {
    rc = run_kernel(h, LBM_KIND_COLLIDE, [&] { return k_collide(h, h->buf[h->cur]); });
    if (!rc) h->halo_valid = true;  // collide writes the halo images
  }
  return rc;
}

// An even number of fused steps (2 or kLongGraphSteps) captured once per
// starting buffer and replayed: one graph launch instead of one kernel launch
// per kernel.  Returns false (and the caller launches directly) when the
// stream cannot be captured, e.g. the legacy default stream.
bool fused_graph(lbm_t* h, int steps, cudaGraphExec_t* out) {
  if (h->graph_unavailable) return false;
  const bool lng = steps == kLongGraphSteps;
  cudaGraphExec_t& g = lng ? h->graph_long[h->cur] : h->graph2[h->cur];
  if (!g) {
    const int c = h->cur;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graph_unavailable = true;
      return false;
    }
    int launched = 0;
    bool ok = true;
    for (int k = 0; k < steps; ++k) {
      const int from = (k & 1) ? 1 - c : c;
      const int nk = k_fused(h, h->buf[from], h->buf[1 - from]);
      ok = ok && nk >= 0;
      launched += nk;
    }
    const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess || !ok || cudaGraphInstantiate(&g, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g = nullptr;
      h->graph_unavailable = true;
      return false;
    }
    cudaGraphDestroy(graph);
    (lng ? h->graph_long_launches : h->graph2_launches) = launched;
  }
  *out = g;
  return true;
}

size_t plane_offset_bytes(const lbm_t* h, int l) {
  return ((size_t)l * h->sp.plane + (size_t)kHx * h->NY + h->sp.Hy) * h->elem;
}

}  // namespace

namespace d2q37 {

int handle_prepare_halos(lbm_t* h, cudaStream_t stream) {
  if (h->halo_valid) return LBM_OK;
  void* b = h->buf[h->cur];
  const int n = is_fp32(h->prec) ? launch_wrap32((float*)b, h->sp, stream) : launch_wrap((double*)b, h->sp, stream);
  if (n < 0) return LBM_ECUDA;
  h->launches += n;
  h->halo_valid = true;
  return LBM_OK;
}

int handle_device_consts() {
  if (!quadrature_ready()) return LBM_ESTATE;
  return ensure_device_consts();
}

}  // namespace d2q37

extern "C" {

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  p->tau = 0.8;
  p->g0 = 1e-4;
  p->T_top = 0.5;
  p->T_bot = 1.5;
  p->precision = LBM_PRECISION_FP64;
  p->kernel = LBM_KERNEL_FUSED;
  p->periodic_y = 0;
}

int lbm_velocity_set(int* cx, int* cy) {
  if (!cx || !cy) return LBM_EINVAL;
  for (int l = 0; l < kQ; ++l) {
    cx[l] = kCx[l];
    cy[l] = kCy[l];
  }
  return LBM_OK;
}

int lbm_quadrature(double* s, double* w) {
  if (!s || !w) return LBM_EINVAL;
  if (!quadrature_ready()) return LBM_ESTATE;
  *s = g_consts.s;
  for (int l = 0; l < kQ; ++l) w[l] = g_consts.w[kShellOf[l]];
  return LBM_OK;
}

size_t lbm_required_bytes(int Lx, int Ly, const lbm_params* p) {
  if (!valid_params(Lx, Ly, p)) return 0;
  return 2 * buffer_bytes(Lx, Ly, p->precision) + scratch_bytes(Lx, Ly);
}

int lbm_create(int Lx, int Ly, const lbm_params* p, lbm_t** out) {
  if (!out || !valid_params(Lx, Ly, p)) return LBM_EINVAL;
  if (!quadrature_ready()) return LBM_ESTATE;
  int rc = ensure_device_consts();
  if (rc) return rc;
  void* mem = nullptr;
  if (cudaMalloc(&mem, lbm_required_bytes(Lx, Ly, p)) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaStream_t stream;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(mem);
    return LBM_ECUDA;
  }
  lbm_t* h = new lbm_t();
  h->owned = mem;
  h->owns_stream = true;
  rc = setup_handle(h, Lx, Ly, p, mem, stream);
  if (rc) {
    lbm_destroy(h);
    return rc;
  }
  *out = h;
  return LBM_OK;
}

int lbm_create_ext(int Lx, int Ly, const lbm_params* p, void* dev_buf, size_t bytes, void* cuda_stream,
                   lbm_t** out) {
  if (!out || !dev_buf || !valid_params(Lx, Ly, p)) return LBM_EINVAL;
  if (((uintptr_t)dev_buf & 255) != 0) return LBM_EINVAL;
  if (bytes < lbm_required_bytes(Lx, Ly, p)) return LBM_ENOMEM;
  if (!quadrature_ready()) return LBM_ESTATE;
  int rc = ensure_device_consts();
  if (rc) return rc;
  lbm_t* h = new lbm_t();
  h->owned = nullptr;
  h->owns_stream = false;
  rc = setup_handle(h, Lx, Ly, p, dev_buf, (cudaStream_t)cuda_stream);
  if (rc) {
    lbm_destroy(h);
    return rc;
  }
  *out = h;
  return LBM_OK;
}

int lbm_init_rayleigh_taylor(lbm_t* h, uint64_t seed) {
  const TraceRange trace("lbm_init_rayleigh_taylor");
  if (!h) return LBM_EINVAL;
  const int Lx = h->Lx, Ly = h->Ly;
  std::vector<double> T((size_t)Lx * Ly);
  const double Tt = h->prm.T_top, Tb = h->prm.T_bot;
  for (int x = 0; x < Lx; ++x) {
    const double arg = (2.0 * M_PI * ((double)x + 0.5)) / (double)Lx;
    const double yi = 0.5 * (double)Ly + ((double)Ly / 64.0) * std::sin(arg);
    for (int y = 0; y < Ly; ++y) {
      const double T0 = ((double)y + 0.5 < yi) ? Tb : Tt;
      const uint64_t r = splitmix64(seed + (uint64_t)x * (uint64_t)Ly + (uint64_t)y);
      const double U = (double)(r >> 11) * 0x1.0p-53;
      T[(size_t)x * Ly + y] = T0 * (1.0 + 1e-3 * (2.0 * U - 1.0));
    }
  }
  int rc = check(cudaMemcpyAsync(h->scratch, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream));
  if (!rc) rc = check(cudaMemsetAsync(h->buf[h->cur], 0, buffer_bytes(Lx, Ly, h->prec), h->stream));
  if (!rc) rc = run_kernel(h, LBM_KIND_INIT, [&] { return k_init(h, h->buf[h->cur], h->scratch); });
  if (!rc) rc = check(cudaStreamSynchronize(h->stream));
  if (!rc) {
    h->have_state = true;
    h->halo_valid = false;
  }
  return rc;
}

int lbm_set_populations(lbm_t* h, const double* f) {
  if (!h || !f) return LBM_EINVAL;
  char* d = (char*)h->buf[h->cur];
  const size_t n = (size_t)h->Lx * h->Ly;
  for (int l = 0; l < kQ; ++l) {
    if (!is_fp32(h->prec)) {
      if (cudaMemcpy2DAsync(d + plane_offset_bytes(h, l), h->NY * sizeof(double), f + (size_t)l * n,
                            h->Ly * sizeof(double), h->Ly * sizeof(double), h->Lx, cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
        return LBM_ECUDA;
      continue;
    }
    // FP32 storage: stage the FP64 plane in scratch, convert to deviations on the device
    if (cudaMemcpyAsync(h->scratch, f + (size_t)l * n, n * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess)
      return LBM_ECUDA;
    const int rc = run_kernel(h, LBM_KIND_CONVERT, [&] {
      return launch_plane_to_frame32((float*)h->buf[h->cur], h->scratch, l, h->sp, h->stream);
    });
    if (rc) return rc;
  }
  if (is_fp32(h->prec) && cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
  h->have_state = true;
  h->halo_valid = false;
  return LBM_OK;
}

int lbm_get_populations(lbm_t* h, double* f) {
  if (!h || !f) return LBM_EINVAL;
  if (!h->have_state) return LBM_ESTATE;
  const char* d = (const char*)h->buf[h->cur];
  const size_t n = (size_t)h->Lx * h->Ly;
  for (int l = 0; l < kQ; ++l) {
    if (!is_fp32(h->prec)) {
      if (cudaMemcpy2DAsync(f + (size_t)l * n, h->Ly * sizeof(double), d + plane_offset_bytes(h, l),
                            h->NY * sizeof(double), h->Ly * sizeof(double), h->Lx, cudaMemcpyDeviceToHost,
                            h->stream) != cudaSuccess)
        return LBM_ECUDA;
      continue;
    }
    const int rc = run_kernel(h, LBM_KIND_CONVERT, [&] {
      return launch_frame32_to_plane(h->scratch, (const float*)h->buf[h->cur], l, h->sp, h->stream);
    });
    if (rc) return rc;
    if (cudaMemcpyAsync(f + (size_t)l * n, h->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) !=
        cudaSuccess)
      return LBM_ECUDA;
  }
  return check(cudaStreamSynchronize(h->stream));
}

int lbm_step(lbm_t* h, int n) {
  const TraceRange trace("lbm_step");
  if (!h || n < 0) return LBM_EINVAL;
  if (!h->have_state) return LBM_ESTATE;
  const bool fused = h->prm.kernel != LBM_KERNEL_SEPARATE;
  int t = 0;
  if (fused && !h->timing && n >= 4) {
    if (!h->halo_valid) {
      const int rc = step_once(h, LBM_PHASE_ALL, true);
      if (rc) return rc;
      ++t;
    }
    cudaGraphExec_t g;
    while (n - t >= kLongGraphSteps && fused_graph(h, kLongGraphSteps, &g)) {
      if (cudaGraphLaunch(g, h->stream) != cudaSuccess) return LBM_ECUDA;
      h->launches += h->graph_long_launches;
      t += kLongGraphSteps;  // an even number of swaps: the current buffer is unchanged
    }
    while (n - t >= 2 && fused_graph(h, 2, &g)) {
      if (cudaGraphLaunch(g, h->stream) != cudaSuccess) return LBM_ECUDA;
      h->launches += h->graph2_launches;
      t += 2;
    }
  }
  for (; t < n; ++t) {
    const int rc = step_once(h, LBM_PHASE_ALL, fused);
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_run_phases(lbm_t* h, int n, int phases) {
  if (!h || n < 0 || phases <= 0 || phases > LBM_PHASE_ALL) return LBM_EINVAL;
  if ((phases & LBM_PHASE_BC) && !(phases & LBM_PHASE_PROPAGATE)) return LBM_EINVAL;
  if (!h->have_state) return LBM_ESTATE;
  for (int t = 0; t < n; ++t) {
    const int rc = step_once(h, phases, false);
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_fields_device(lbm_t* h, double* rho, double* u, double* T) {
  if (!h || !rho || !u || !T) return LBM_EINVAL;
  if (!h->have_state) return LBM_ESTATE;
  return run_kernel(h, LBM_KIND_FIELDS, [&] { return k_fields(h, h->buf[h->cur], rho, u, T); });
}

int lbm_fields(lbm_t* h, double* rho, double* u, double* T) {
  if (!h || !rho || !u || !T) return LBM_EINVAL;
  const size_t n = (size_t)h->Lx * h->Ly;
  double* s = h->scratch;
  int rc = lbm_fields_device(h, s, s + n, s + 3 * n);
  if (rc) return rc;
  rc = check(cudaMemcpyAsync(rho, s, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (!rc) rc = check(cudaMemcpyAsync(u, s + n, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (!rc) rc = check(cudaMemcpyAsync(T, s + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (!rc) rc = check(cudaStreamSynchronize(h->stream));
  return rc;
}

int lbm_synchronize(lbm_t* h) {
  if (!h) return LBM_EINVAL;
  return check(cudaStreamSynchronize(h->stream));
}

int64_t lbm_launch_count(const lbm_t* h) { return h ? h->launches : 0; }

int lbm_set_timing(lbm_t* h, int enable) {
  if (!h) return LBM_EINVAL;
  int rc = check(cudaStreamSynchronize(h->stream));
  if (drain_timing(h) != LBM_OK) rc = LBM_ECUDA;
  for (int k = 0; k < LBM_KIND_COUNT; ++k) {
    h->kind_ms[k] = 0.0;
    h->kind_launches[k] = 0;
  }
  h->timing = enable != 0;
  return rc;
}

int lbm_kernel_times(lbm_t* h, double* ms, int64_t* launches) {
  if (!h) return LBM_EINVAL;
  int rc = check(cudaStreamSynchronize(h->stream));
  if (drain_timing(h) != LBM_OK) rc = LBM_ECUDA;
  for (int k = 0; k < LBM_KIND_COUNT; ++k) {
    if (ms) ms[k] = h->kind_ms[k];
    if (launches) launches[k] = h->kind_launches[k];
  }
  return rc;
}

void lbm_destroy(lbm_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drain_timing(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  for (cudaGraphExec_t g : h->graph2)
    if (g) cudaGraphExecDestroy(g);
  for (cudaGraphExec_t g : h->graph_long)
    if (g) cudaGraphExecDestroy(g);
  if (h->owns_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->owned) cudaFree(h->owned);
  delete h;
}

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "success";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of device memory or caller buffer too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ETIMEOUT: return "bounded device wait timed out";
    case LBM_ESTATE: return "call out of order (no state yet, or quadrature unavailable)";
    case LBM_ETOOBIG: return "more lattices than the static table of lbm_batch_step_static holds";
    default: return "unknown error code";
  }
}

}  // extern "C"
