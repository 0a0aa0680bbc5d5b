// forecast_ns2d.h -- 2-D compressible Navier-Stokes forecast launcher (internal).
#pragma once

#include <cuda_runtime.h>

namespace mgk {

// NULL if grids of n_whole (one member per CTA group) and n_split points per
// side can be advanced, else the reason.
const char *ns2d_check_size(int n_whole, int n_split);

// Scratch (elements of T) the forecast needs for its two stage buffers.
size_t ns2d_scratch_elems(int n_whole, int n_whole_probs, int n_split, int n_split_probs);

// Advance n_whole_probs grids of n_whole^2 x 4 and n_split_probs grids of
// n_split^2 x 4 conserved variables by nsteps SSP-RK3 steps, with caller
// scratch of ns2d_scratch_elems() elements.
template <typename T>
cudaError_t ns2d_forecast_scratch(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                                  int n_split_probs, double length, double dt, double mu,
                                  double gamma, double prandtl, int nsteps, T *scratch,
                                  cudaStream_t stream);

// Same, with stream-ordered temporary scratch (cudaMallocAsync / cudaFreeAsync).
template <typename T>
cudaError_t ns2d_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                          int n_split_probs, double length, double dt, double mu, double gamma,
                          double prandtl, int nsteps, cudaStream_t stream);

}  // namespace mgk
