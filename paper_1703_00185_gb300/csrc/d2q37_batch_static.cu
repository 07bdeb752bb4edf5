// Batched stepping without any device allocation (lbm_batch_step_static,
// declared in include/d2q37.h).
//
// lbm_batch_create keeps the lattices' tile table in memory it gets from
// cudaMalloc.  Some callers cannot allocate device memory: programs whose
// device memory all belongs to a caching allocator or a pre-registered pool
// (a stray cudaMalloc breaks their budget or fails when the device is full),
// and loops that cannot afford the device synchronisation cudaMalloc/cudaFree
// may imply.  This entry point keeps the table in a fixed file-scope device
// array instead; the lattices' own memory is the caller's, as always.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "d2q37_handle.h"

namespace {

// The table lives here: LBM_STATIC_BATCH_MAX entries, loaded with the
// library on every GPU that uses it and held until the process exits.
__device__ __align__(256) BatchEntry g_static_tab[LBM_STATIC_BATCH_MAX];

std::mutex g_static_mutex;               // guards the host staging table and set-up
BatchEntry g_static_host[LBM_STATIC_BATCH_MAX];
BatchEntry* g_static_dev[256];           // address of g_static_tab per device, once set up

// Device address of g_static_tab on the current device.  In host code the
// name g_static_tab is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
int static_table(BatchEntry** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return LBM_ECUDA;
  if (!g_static_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_tab) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ECUDA;
    }
    g_static_dev[dev] = (BatchEntry*)p;
  }
  *out = g_static_dev[dev];
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_step_static(int n, lbm_t* const* lattices, int steps, void* cuda_stream) {
  if (!lattices || n <= 0 || steps < 0) return LBM_EINVAL;
  if (n > LBM_STATIC_BATCH_MAX) return LBM_ETOOBIG;
  for (int i = 0; i < n; ++i) {
    if (!lattices[i] || lattices[i]->prec != lattices[0]->prec) return LBM_EINVAL;
    if (!lattices[i]->have_state) return LBM_ESTATE;
    for (int j = 0; j < i; ++j)
      if (lattices[j] == lattices[i]) return LBM_EINVAL;
  }
  if (steps == 0) return LBM_OK;
  const cudaStream_t stream = (cudaStream_t)cuda_stream;
  // The lattices' current buffers are switched here, on the host, and the
  // table is copied from host memory that the next call rewrites: work
  // recorded into a graph would replay with stale buffers and table.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return LBM_EINVAL;
  // every lattice's memory must be on the current device, where the table is
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  for (int i = 0; i < n; ++i) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, lattices[i]->buf[0]) != cudaSuccess) {
      cudaGetLastError();
      return LBM_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice || a.device != dev) return LBM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mutex);
  int rc = handle_device_consts();
  BatchEntry* dev_tab = nullptr;
  if (!rc) rc = static_table(&dev_tab);
  for (int i = 0; i < n && !rc; ++i) rc = handle_prepare_halos(lattices[i], stream);
  if (rc) return rc;
  // the whole table [0, n) is rewritten every call; entries past n are never read
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    BatchEntry& e = g_static_host[i];
    std::memset(&e, 0, sizeof(e));
    e.p = lattices[i]->sp;
    e.buf[0] = lattices[i]->buf[0];
    e.buf[1] = lattices[i]->buf[1];
    e.cur = lattices[i]->cur;
    e.ytiles = (lattices[i]->Ly + 127) / 128;
    e.tile0 = tiles;
    tiles += (long long)lattices[i]->Lx * e.ytiles;
  }
  // pageable source: the runtime stages it before the call returns (so the
  // next call may rewrite it), which waits for the stream's earlier work
  if (cudaMemcpyAsync(dev_tab, g_static_host, n * sizeof(BatchEntry), cudaMemcpyHostToDevice, stream) !=
      cudaSuccess)
    return LBM_ECUDA;
  const int prec = lattices[0]->prec;
  const int grid = (int)(tiles < 2147483647LL ? tiles : 2147483647LL);
  for (int t = 0; t < steps; ++t) {
    const int launched =
        prec == LBM_PRECISION_FP64
            ? launch_batch_fused(dev_tab, nullptr, n, tiles, t & 1, 128, grid, nullptr, stream)
            : launch_batch_fused32(dev_tab, nullptr, n, tiles, t & 1, 128, grid, prec == LBM_PRECISION_FP32_FP64, stream);
    if (launched < 0) return LBM_ECUDA;
  }
  for (int i = 0; i < n; ++i) lattices[i]->cur ^= (steps & 1);
  return LBM_OK;
}

}  // extern "C"
