// Batched stepping of many independent lattices (C ABI declared in
// include/d2q37.h, lbm_batch_*).
//
// The lattices keep their own memory and parameters (lbm_t handles); the
// batch owns a device table of BatchEntry (parameters, both buffers, the
// buffer holding the state, tile range) and a per-tile owner table, and
// advances every lattice by one step per launch:
//  - block_y > 0, blocks_per_sm = 0: one block per tile.  FP64 batches that
//    allow it (walls, one tau and g, at most kBatchGeoMax lattices, 32-bit
//    offsets) run the split form, site tiles and wall tiles of every lattice
//    with each lattice's offsets in the launch's parameters (BatchLaunch);
//    FP32-storage batches of at most kBatchGeo32Max lattices take their
//    parameters from BatchLaunch32; other batches run the table kernel.
//  - block_y > 0, blocks_per_sm > 0: the table kernel on a persistent grid.
//  - block_y = 0: the single-lattice fused kernel once per lattice (its
//    parameters in the constant bank), spread over kAux streams forked from
//    and joined to the batch stream, so that small lattices run side by side.
// lbm_batch_step(n) replays a captured two-step CUDA graph when the stream
// can be captured (with block_y = 0 a graph of parallel branches).
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "d2q37_handle.h"

struct lbm_batch_t {
  int n;
  int prec;
  std::vector<lbm_t*> lat;
  std::vector<BatchEntry> host_tab[3];  // per block_y choice (64, 128, 256)
  BatchEntry* dev_tab[3];
  int* dev_tile_entry[3];  // owning entry of every tile
  bool uniform;            // every lattice has the collision constants of `common` (same tau, g)
  StepParams common;
  // FP64 with walls, shared tau and g, at most kBatchGeoMax lattices whose
  // offsets fit 32 bits: block_y > 0 with blocks_per_sm = 0 runs the split
  // form (site tiles and wall tiles in one launch), parameters per block_y
  bool split_ok;
  BatchLaunch* split[3];
  // FP32 storage, at most kBatchGeo32Max lattices: block_y > 0 with
  // blocks_per_sm = 0 runs one block per tile with parameters in the launch
  bool split32_ok;
  BatchLaunch32* split32[3];
  long long tiles[3];
  int block_y;        // 64, 128 or 256
  int blocks_per_sm;  // 0: one block per tile; else a persistent grid of blocks_per_sm x SMs
  int sms;
  int parity;         // lattice i holds its state in buffer entry.cur ^ parity
  cudaStream_t stream;
  int64_t launches;
  cudaGraphExec_t graph2;  // two steps from parity 0
  int graph_config;        // block_y * 16 + blocks_per_sm the graph was captured with
  int64_t graph_launches;  // kernels in graph2 (2, or 2 n with block_y = 0)
  bool graph_unavailable;
  // block_y = 0: one launch per lattice, largest first, round robin over aux
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux];
  cudaEvent_t fork, join[kAux];
  bool aux_ready;
  std::vector<int> order;  // lattices by decreasing site count
};

namespace {

int check(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

int slot_of(int block_y) { return block_y == 64 ? 0 : block_y == 128 ? 1 : block_y == 256 ? 2 : -1; }

// The streams and events of the per-lattice form (made when the batch is).
int ensure_aux(lbm_batch_t* b) {
  if (b->aux_ready) return LBM_OK;
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < lbm_batch_t::kAux; ++k) {
    b->aux[k] = nullptr;
    b->join[k] = nullptr;
    ok = ok && cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  }
  b->aux_ready = true;  // destroy releases whatever was made
  if (!ok) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

// One step of every lattice with its own fused kernel: forked from the batch
// stream onto the aux streams and joined back to it.
int launch_each(lbm_batch_t* b, int parity) {
  int rc = ensure_aux(b);
  if (rc) return rc;
  rc = check(cudaEventRecord(b->fork, b->stream));
  for (int k = 0; k < lbm_batch_t::kAux && !rc; ++k) rc = check(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
  for (size_t j = 0; j < b->order.size() && !rc; ++j) {
    const int i = b->order[j];
    const lbm_t* h = b->lat[i];
    const int c = b->host_tab[0][i].cur ^ parity;
    cudaStream_t s = b->aux[j % lbm_batch_t::kAux];
    const int n = b->prec == LBM_PRECISION_FP64
                      ? launch_fused((const double*)h->buf[c], (double*)h->buf[c ^ 1], h->sp, s)
                      : launch_fused32((const float*)h->buf[c], (float*)h->buf[c ^ 1], h->sp,
                                       b->prec == LBM_PRECISION_FP32_FP64, s);
    if (n < 0) rc = LBM_ECUDA;
    else b->launches += n;
  }
  for (int k = 0; k < lbm_batch_t::kAux && !rc; ++k) {
    rc = check(cudaEventRecord(b->join[k], b->aux[k]));
    if (!rc) rc = check(cudaStreamWaitEvent(b->stream, b->join[k], 0));
  }
  return rc;
}

int max_blocks_per_sm(const lbm_batch_t* b, int block_y) {
  return b->prec == LBM_PRECISION_FP64 ? batch_blocks_per_sm(block_y)
                                       : batch32_blocks_per_sm(block_y, b->prec == LBM_PRECISION_FP32_FP64);
}

long long grid_of(const lbm_batch_t* b, int block_y, int blocks_per_sm) {
  const long long tiles = b->tiles[slot_of(block_y)];
  long long g = blocks_per_sm > 0 ? (long long)blocks_per_sm * b->sms : tiles;
  g = std::min(g, tiles);
  return std::min(std::max(g, 1LL), 2147483647LL);
}

int launch(lbm_batch_t* b, int block_y, int blocks_per_sm, int parity) {
  if (block_y == 0) return launch_each(b, parity);
  const int s = slot_of(block_y);
  if (blocks_per_sm == 0 && (b->split_ok || b->split32_ok)) {
    const int n = b->split_ok ? launch_batch_split(*b->split[s], b->dev_tab[s], b->dev_tile_entry[s], parity,
                                                   block_y, b->stream)
                              : launch_batch_split32(*b->split32[s], b->dev_tile_entry[s], (int)b->tiles[s], parity,
                                                     block_y, b->prec == LBM_PRECISION_FP32_FP64, b->stream);
    if (n < 0) return LBM_ECUDA;
    b->launches += n;
    return LBM_OK;
  }
  const int grid = (int)grid_of(b, block_y, blocks_per_sm);
  const int n = b->prec == LBM_PRECISION_FP64
                    ? launch_batch_fused(b->dev_tab[s], b->dev_tile_entry[s], b->n, b->tiles[s], parity, block_y,
                                         grid, b->uniform ? &b->common : nullptr, b->stream)
                    : launch_batch_fused32(b->dev_tab[s], b->dev_tile_entry[s], b->n, b->tiles[s], parity, block_y, grid,
                                           b->prec == LBM_PRECISION_FP32_FP64, b->stream);
  if (n < 0) return LBM_ECUDA;
  b->launches += n;
  return LBM_OK;
}

// Record the parity of the lattices' current buffers in their handles.
void publish_parity(lbm_batch_t* b) {
  for (int i = 0; i < b->n; ++i) b->lat[i]->cur = b->host_tab[0][i].cur ^ b->parity;
}

bool pair_graph(lbm_batch_t* b, cudaGraphExec_t* out) {
  if (b->graph_unavailable) return false;
  const int cfg = b->block_y * 16 + b->blocks_per_sm;
  if (b->graph2 && b->graph_config != cfg) {
    cudaGraphExecDestroy(b->graph2);
    b->graph2 = nullptr;
  }
  if (!b->graph2) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      b->graph_unavailable = true;
      return false;
    }
    const int64_t before = b->launches;
    const int r0 = launch(b, b->block_y, b->blocks_per_sm, 0);
    const int r1 = launch(b, b->block_y, b->blocks_per_sm, 1);
    b->graph_launches = b->launches - before;
    b->launches = before;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || r0 || r1 || cudaGraphInstantiate(&b->graph2, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      b->graph2 = nullptr;
      b->graph_unavailable = true;
      return false;
    }
    cudaGraphDestroy(g);
    b->graph_config = cfg;
  }
  *out = b->graph2;
  return true;
}

bool fits32(long long v) { return v >= -2147483647LL - 1 && v <= 2147483647LL; }

// The FP32 one-block-per-tile form's launch parameters (the lattices'
// entries of the device table dev_tab hold their wall constants).
void build_split32(lbm_batch_t* b) {
  b->split32_ok = b->prec != LBM_PRECISION_FP64 && b->n <= kBatchGeo32Max;
  for (int s = 0; s < 3 && b->split32_ok; ++s) {
    if (b->tiles[s] > 2147483647LL) {
      b->split32_ok = false;
      break;
    }
    BatchLaunch32* L = new BatchLaunch32();
    std::memset(L, 0, sizeof(*L));
    L->n = b->n;
    for (int i = 0; i < b->n; ++i) {
      const lbm_t* h = b->lat[i];
      const StepParams& q = h->sp;
      // device addresses inside the entry's parameters (addresses only: no access on the host)
      const char* dq = (const char*)b->dev_tab[s] + i * sizeof(BatchEntry) + offsetof(BatchEntry, p);
      BatchGeo32& g = L->g[i];
      g.Lx = h->Lx;
      g.Ly = h->Ly;
      g.NY = q.NY;
      g.Hy = q.Hy;
      g.periodic_y = q.periodic_y;
      g.tile0 = (int)b->host_tab[s][i].tile0;
      g.cur = b->host_tab[s][i].cur;
      g.plane = q.plane;
      g.buf[0] = h->buf[0];
      g.buf[1] = h->buf[1];
      g.omega_f = q.omega_f;
      g.keep_f = q.keep_f;
      g.uy_shift_df[0] = q.uy_shift_df[0];
      g.uy_shift_df[1] = q.uy_shift_df[1];
      g.theta_shift_df[0] = q.theta_shift_df[0];
      g.theta_shift_df[1] = q.theta_shift_df[1];
      g.theta_shift = q.theta_shift;
      g.fw32 = (const float(*)[kQ])(dq + offsetof(StepParams, fw32));
      g.fwmw32 = (const float(*)[kQ])(dq + offsetof(StepParams, fwmw32));
      g.wall_e32 = (const float(*)[2])(dq + offsetof(StepParams, wall_e32));
      g.wall_inv32 = (const float(*)[2])(dq + offsetof(StepParams, wall_inv32));
    }
    b->split32[s] = L;
  }
}

// The split form's launch parameters for every block_y, if the batch allows it.
void build_split(lbm_batch_t* b) {
  b->split_ok = b->prec == LBM_PRECISION_FP64 && b->uniform && b->n <= kBatchGeoMax;
  for (int i = 0; i < b->n && b->split_ok; ++i) {
    const StepParams& q = b->lat[i]->sp;
    b->split_ok = !q.periodic_y;
    for (int l = 0; l < kQ && b->split_ok; ++l) b->split_ok = fits32(q.pull_off[l]) && fits32(q.plane_off[l]);
  }
  if (!b->split_ok) return;
  const int bys[3] = {64, 128, 256};
  for (int s = 0; s < 3; ++s) {
    BatchLaunch* L = new BatchLaunch();
    std::memset(L, 0, sizeof(*L));
    L->common = b->common;
    L->n = b->n;
    long long t0 = 0, w0 = 0;
    const int per_wall_tile = batch_wall_groups_per_tile(bys[s]);
    for (int i = 0; i < b->n; ++i) {
      const lbm_t* h = b->lat[i];
      BatchGeo& g = L->g[i];
      for (int l = 0; l < kQ; ++l) {
        g.pull_off[l] = (int)h->sp.pull_off[l];
        g.plane_off[l] = (int)h->sp.plane_off[l];
      }
      g.Lx = h->Lx;
      g.Ly = h->Ly;
      g.NY = h->sp.NY;
      g.Hy = h->sp.Hy;
      g.ytiles = (h->Ly + bys[s] - 1) / bys[s];
      g.tile0 = (int)t0;
      g.wtile0 = (int)w0;
      g.cur = b->host_tab[s][i].cur;
      g.entry = i;
      g.plane = h->sp.plane;
      g.buf[0] = h->buf[0];
      g.buf[1] = h->buf[1];
      g.inv_denom[0] = h->sp.inv_denom[0];
      g.inv_denom[1] = h->sp.inv_denom[1];
      t0 += (long long)h->Lx * g.ytiles;
      w0 += (2LL * h->Lx + per_wall_tile - 1) / per_wall_tile;
    }
    if (t0 + w0 > 2147483647LL) {
      delete L;
      b->split_ok = false;
      return;
    }
    L->site_tiles = (int)t0;
    L->wall_tiles = (int)w0;
    b->split[s] = L;
  }
}

}  // namespace

extern "C" {

int lbm_batch_create(int n, lbm_t* const* lattices, void* cuda_stream, lbm_batch_t** out) {
  if (!out || n <= 0 || !lattices) return LBM_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!lattices[i]) return LBM_EINVAL;
    if (lattices[i]->prec != lattices[0]->prec) return LBM_EINVAL;
    if (!lattices[i]->have_state) return LBM_ESTATE;
    for (int j = 0; j < i; ++j)
      if (lattices[j] == lattices[i]) return LBM_EINVAL;
  }
  int rc = handle_device_consts();
  if (rc) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LBM_ECUDA;
  lbm_batch_t* b = new lbm_batch_t();
  b->n = n;
  b->prec = lattices[0]->prec;
  b->lat.assign(lattices, lattices + n);
  b->sms = sms;
  b->stream = (cudaStream_t)cuda_stream;
  b->block_y = 128;
  b->blocks_per_sm = 0;
  b->common = lattices[0]->sp;
  b->uniform = true;
  for (int i = 1; i < n; ++i) {
    const StepParams& q = lattices[i]->sp;
    b->uniform = b->uniform && q.omega == b->common.omega && q.uy_shift == b->common.uy_shift &&
                 q.theta_shift == b->common.theta_shift;
  }
  // the lattices' own pending work comes first; their halos must mirror the state
  for (int i = 0; i < n && !rc; ++i) {
    rc = check(cudaStreamSynchronize(lattices[i]->stream));
    if (!rc) rc = handle_prepare_halos(lattices[i], b->stream);
  }
  const int bys[3] = {64, 128, 256};
  for (int s = 0; s < 3 && !rc; ++s) {
    long long t0 = 0;
    b->host_tab[s].resize(n);
    for (int i = 0; i < n; ++i) {
      BatchEntry& e = b->host_tab[s][i];
      std::memset(&e, 0, sizeof(e));
      e.p = lattices[i]->sp;
      e.buf[0] = lattices[i]->buf[0];
      e.buf[1] = lattices[i]->buf[1];
      e.cur = lattices[i]->cur;
      e.ytiles = (lattices[i]->Ly + bys[s] - 1) / bys[s];
      e.tile0 = t0;
      t0 += (long long)lattices[i]->Lx * e.ytiles;
    }
    b->tiles[s] = t0;
    if (t0 > 2147483647LL) {
      rc = LBM_ETOOBIG;
      break;
    }
    std::vector<int> owner((size_t)t0);
    for (int i = 0; i < n; ++i)
      std::fill(owner.begin() + b->host_tab[s][i].tile0,
                owner.begin() + b->host_tab[s][i].tile0 + (long long)lattices[i]->Lx * b->host_tab[s][i].ytiles, i);
    if (cudaMalloc(&b->dev_tab[s], n * sizeof(BatchEntry)) != cudaSuccess ||
        cudaMalloc(&b->dev_tile_entry[s], owner.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      rc = LBM_ENOMEM;
      break;
    }
    rc = check(cudaMemcpyAsync(b->dev_tab[s], b->host_tab[s].data(), n * sizeof(BatchEntry),
                               cudaMemcpyHostToDevice, b->stream));
    if (!rc)
      rc = check(cudaMemcpyAsync(b->dev_tile_entry[s], owner.data(), owner.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, b->stream));
    // the host vector must outlive the asynchronous copy
    if (!rc) rc = check(cudaStreamSynchronize(b->stream));
  }
  if (!rc) rc = check(cudaStreamSynchronize(b->stream));
  if (!rc) {
    build_split(b);
    build_split32(b);
  }
  if (rc) {
    lbm_batch_destroy(b);
    return rc;
  }
  // the per-lattice form's streams now, never inside a stream capture
  rc = ensure_aux(b);
  if (rc) {
    lbm_batch_destroy(b);
    return rc;
  }
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int i, int j) {
    return (long long)lattices[i]->Lx * lattices[i]->Ly > (long long)lattices[j]->Lx * lattices[j]->Ly;
  });
  *out = b;
  return LBM_OK;
}

int lbm_batch_set_config(lbm_batch_t* b, int block_y, int blocks_per_sm) {
  if (!b || blocks_per_sm < 0) return LBM_EINVAL;
  if (block_y == 0 ? blocks_per_sm != 0 : slot_of(block_y) < 0) return LBM_EINVAL;
  if (blocks_per_sm > 0 && blocks_per_sm > max_blocks_per_sm(b, block_y)) return LBM_EINVAL;
  b->block_y = block_y;
  b->blocks_per_sm = blocks_per_sm;
  return LBM_OK;
}

int lbm_batch_get_config(const lbm_batch_t* b, int* block_y, int* blocks_per_sm) {
  if (!b || !block_y || !blocks_per_sm) return LBM_EINVAL;
  *block_y = b->block_y;
  *blocks_per_sm = b->blocks_per_sm;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch_t* b, int n) {
  const TraceRange trace("lbm_batch_step");
  if (!b || n < 0) return LBM_EINVAL;
  int t = 0;
  if (n >= 4) {
    if (b->parity) {
      const int rc = launch(b, b->block_y, b->blocks_per_sm, b->parity);
      if (rc) return rc;
      b->parity ^= 1;
      ++t;
    }
    cudaGraphExec_t g;
    while (n - t >= 2 && pair_graph(b, &g)) {
      if (cudaGraphLaunch(g, b->stream) != cudaSuccess) return LBM_ECUDA;
      b->launches += b->graph_launches;
      t += 2;
    }
  }
  for (; t < n; ++t) {
    const int rc = launch(b, b->block_y, b->blocks_per_sm, b->parity);
    if (rc) return rc;
    b->parity ^= 1;
  }
  publish_parity(b);
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_t* b, int trial_steps, int* block_y, int* blocks_per_sm, double* best_ms) {
  const TraceRange trace("lbm_batch_autotune");
  if (!b || trial_steps <= 0) return LBM_EINVAL;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LBM_ECUDA;
  }
  int rc = LBM_OK;
  float best = 1e30f;
  int best_by = b->block_y, best_bps = b->blocks_per_sm;
  const int bys[4] = {64, 128, 256, 0};  // 0: one launch per lattice
  const int64_t launches0 = b->launches;
  for (int s = 0; s < 4 && !rc; ++s) {
    const int occ = bys[s] ? max_blocks_per_sm(b, bys[s]) : 0;
    for (int bps = 0; bps <= occ && !rc; ++bps) {
      // the same parity every launch: each trial recomputes the same step into
      // the other buffer, so the lattices' state does not advance
      rc = launch(b, bys[s], bps, b->parity);
      if (!rc) rc = check(cudaEventRecord(e0, b->stream));
      for (int k = 0; k < trial_steps && !rc; ++k) rc = launch(b, bys[s], bps, b->parity);
      if (!rc) rc = check(cudaEventRecord(e1, b->stream));
      if (!rc) rc = check(cudaEventSynchronize(e1));
      float ms = 0.0f;
      if (!rc) rc = check(cudaEventElapsedTime(&ms, e0, e1));
      if (!rc && ms < best) {
        best = ms;
        best_by = bys[s];
        best_bps = bps;
      }
    }
  }
  b->launches = launches0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->block_y = best_by;
  b->blocks_per_sm = best_bps;
  if (block_y) *block_y = best_by;
  if (blocks_per_sm) *blocks_per_sm = best_bps;
  if (best_ms) *best_ms = best / trial_steps;
  return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch_t* b) {
  if (!b) return LBM_EINVAL;
  return check(cudaStreamSynchronize(b->stream));
}

int64_t lbm_batch_launch_count(const lbm_batch_t* b) { return b ? b->launches : 0; }

void lbm_batch_destroy(lbm_batch_t* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph2) cudaGraphExecDestroy(b->graph2);
  if (b->aux_ready) {
    for (int k = 0; k < lbm_batch_t::kAux; ++k) {
      if (b->aux[k]) {
        cudaStreamSynchronize(b->aux[k]);
        cudaStreamDestroy(b->aux[k]);
      }
      if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
  }
  for (BatchEntry* t : b->dev_tab)
    if (t) cudaFree(t);
  for (int* t : b->dev_tile_entry)
    if (t) cudaFree(t);
  for (BatchLaunch* L : b->split) delete L;
  for (BatchLaunch32* L : b->split32) delete L;
  delete b;
}

}  // extern "C"
