// Host-side launchers of the sm_103a kernels (d2q37_kernels.cu), used by the
// C ABI (d2q37_api.cu).  Each launcher enqueues on `stream` and returns the
// number of kernels it launched, or -1 if a launch failed.
#pragma once

#include <cuda_runtime.h>

#include "d2q37_lattice.cuh"

namespace d2q37 {

// Copy the quadrature constants to the current device's constant memory.
cudaError_t upload_shell_consts(const ShellConsts& c);

int launch_wrap(double* buf, const StepParams& p, cudaStream_t stream);
int launch_propagate(const double* src, double* dst, const StepParams& p, cudaStream_t stream);
int launch_bc(const double* src, double* dst, const StepParams& p, cudaStream_t stream);
int launch_collide(double* buf, const StepParams& p, cudaStream_t stream);
// overlap: the wall-band kernel (walls only) is launched as a programmatic
// dependent of the sites kernel and starts in its tail; false: after it.
int launch_fused(const double* src, double* dst, const StepParams& p, cudaStream_t stream, bool overlap = true);
int launch_fields(const double* buf, double* rho, double* u, double* T, const StepParams& p, cudaStream_t stream);
int launch_init_equilibrium(double* buf, const double* T, const StepParams& p, cudaStream_t stream);

// FP32 deviation storage (d2q37_kernels_fp32.cu; init in d2q37_kernels.cu).
// wide_fp64 selects FP64 (true) or double-float (false) for the wide terms.
cudaError_t upload_shell_consts32(const ShellConsts32& c);
int launch_wrap32(float* buf, const StepParams& p, cudaStream_t stream);
int launch_propagate32(const float* src, float* dst, const StepParams& p, cudaStream_t stream);
int launch_bc32(const float* src, float* dst, const StepParams& p, cudaStream_t stream);
int launch_collide32(float* buf, const StepParams& p, bool wide_fp64, cudaStream_t stream);
int launch_fused32(const float* src, float* dst, const StepParams& p, bool wide_fp64, cudaStream_t stream);
int launch_fields32(const float* buf, double* rho, double* u, double* T, const StepParams& p, cudaStream_t stream);
int launch_init_equilibrium32(float* buf, const double* T, const StepParams& p, cudaStream_t stream);
// Batched fused step over a table of n lattices (BatchEntry, device memory),
// tiles of block_y rows; block_y in {64, 128, 256}; grid = number of blocks
// of the grid-stride loop.  *_blocks_per_sm: resident blocks per SM.
// tile_entry: owning entry of every tile (device, tiles values), or null
// for a binary search over the table's tile0.  common (FP64): when every
// lattice shares tau and g, a StepParams holding their collision constants
// (passed as a kernel argument), else null.
int launch_batch_fused(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity,
                       int block_y, int grid, const StepParams* common, cudaStream_t stream);
int batch_blocks_per_sm(int block_y);
// The split form of the batched FP64 step (one launch: site tiles, then wall
// tiles; see BatchLaunch); the (column, wall) groups one wall tile holds.
// tile_entry: owning lattice of every site tile (the batch's per-tile table).
int launch_batch_split(const BatchLaunch& L, const BatchEntry* tab, const int* tile_entry, int parity, int block_y,
                       cudaStream_t stream);
int batch_wall_groups_per_tile(int block_y);
int launch_batch_fused32(const BatchEntry* tab, const int* tile_entry, int n, long long tiles, int parity,
                         int block_y, int grid, bool wide_fp64, cudaStream_t stream);
int batch32_blocks_per_sm(int block_y, bool wide_fp64);
// FP32 storage, one block per tile with every lattice's parameters in the
// launch's parameter space (BatchLaunch32); tiles: grid size.
int launch_batch_split32(const BatchLaunch32& L, const int* tile_entry, int tiles, int parity, int block_y,
                         bool wide_fp64, cudaStream_t stream);

// One population plane between a contiguous FP64 [Lx][Ly] array (f) and the
// FP32 deviation frame (d = f - w_l).
int launch_plane_to_frame32(float* frame, const double* plane, int l, const StepParams& p, cudaStream_t stream);
int launch_frame32_to_plane(double* plane, const float* frame, int l, const StepParams& p, cudaStream_t stream);

}  // namespace d2q37
