// forecast_ns2d.h -- 2-D compressible Navier-Stokes forecast launcher (internal).
#pragma once

#include <cuda_runtime.h>

namespace mgk {

// NULL if grids of n_whole (one member per CTA group) and n_split points per
// side can be advanced, else the reason.
const char *ns2d_check_size(int n_whole, int n_split);

// Advance n_whole_probs grids of n_whole^2 x 4 and n_split_probs grids of
// n_split^2 x 4 conserved variables by nsteps SSP-RK3 steps.
template <typename T>
cudaError_t ns2d_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                          int n_split_probs, double length, double dt, double mu, double gamma,
                          double prandtl, int nsteps, cudaStream_t stream);

}  // namespace mgk
