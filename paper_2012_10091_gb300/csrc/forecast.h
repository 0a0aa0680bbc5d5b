// forecast.h -- model forecast launchers (internal to the library).
#pragma once

#include <cuda_runtime.h>

namespace mgk {

constexpr int kBurgersMaxPtsPerCta = 4096;

// CTAs per Burgers grid of n points (0 if n cannot be split within the limits).
int burgers_split_factor(int n);

// Advance n_whole_probs grids of n_whole points (one CTA each, n_whole <= 4096)
// and n_split_probs grids of n_split points (a cluster of CTAs each) by nsteps
// SSP-RK3 steps of periodic viscous Burgers, in one launch.
template <typename T>
cudaError_t burgers_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                             int n_split_probs, double length, double dt, double nu, int nsteps,
                             cudaStream_t stream);

}  // namespace mgk
