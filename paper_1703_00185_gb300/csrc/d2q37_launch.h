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
int launch_fused(const double* src, double* dst, const StepParams& p, cudaStream_t stream);
int launch_fields(const double* buf, double* rho, double* u, double* T, const StepParams& p, cudaStream_t stream);
int launch_init_equilibrium(double* buf, const double* T, const StepParams& p, cudaStream_t stream);

}  // namespace d2q37
