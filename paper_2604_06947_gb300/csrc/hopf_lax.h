// hopf_lax.h -- the Hopf-Lax entropy reference of Burgers (k_hopf_lax.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fqnm {

// u_i = (x_i - y_j*) / t with j* = argmin_j U0y_j + (x_i - y_j)^2 / (2t), ties
// to the smallest j, for nx points from ny candidates (device arrays); idx
// (may be null) receives j*.
cudaError_t launch_hopf_lax(const double* x, int64_t nx, const double* y, const double* U0y,
                            int64_t ny, double t, double* u, int64_t* idx, cudaStream_t st);

}  // namespace fqnm
