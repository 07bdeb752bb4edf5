// Internal: the lattice handle behind the C ABI's opaque lbm_t, shared by
// d2q37_api.cu (single lattices) and d2q37_batch.cu (many lattices per launch).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/d2q37.h"
#include "d2q37_launch.h"

using namespace d2q37;

struct lbm_t {
  int Lx, Ly, NX, NY;
  int prec;     // LBM_PRECISION_*
  size_t elem;  // bytes per stored population value
  lbm_params prm;
  StepParams sp;
  void* buf[2];
  int cur;
  double* scratch;  // 4 Lx Ly doubles: fields, the initial temperature, or one FP64 plane
  void* owned;      // cudaMalloc'ed block, NULL for lbm_create_ext
  cudaStream_t stream;
  bool owns_stream;
  bool have_state;
  bool halo_valid;  // halo columns (and rows, if y is periodic) mirror the current state
  int64_t launches;
  cudaGraphExec_t graph2[2];  // two fused steps starting from buffer 0 / 1
  int64_t graph2_launches;  // kernels in one replay of graph2 (2 steps)
  cudaGraphExec_t graph_long[2];  // kLongGraphSteps fused steps from buffer 0 / 1
  int64_t graph_long_launches;
  bool graph_unavailable;
  // per-kernel timing: event pairs recorded around launches, folded into the
  // totals when the stream is synchronised
  bool timing;
  struct Pending {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  double kind_ms[LBM_KIND_COUNT];
  int64_t kind_launches[LBM_KIND_COUNT];
};

namespace d2q37 {

// An NVTX range over a scope (host side), so that profilers' timelines show
// the library's entry points; free when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Fused steps per replay of a handle's long graph (lbm_step with n >= this).
constexpr int kLongGraphSteps = 16;

// Launch the pbc kernel on `stream` if the handle's halos are stale.
int handle_prepare_halos(lbm_t* h, cudaStream_t stream);

// Quadrature constants on the current device (0 or an LBM_E* code).
int handle_device_consts();

}  // namespace d2q37
