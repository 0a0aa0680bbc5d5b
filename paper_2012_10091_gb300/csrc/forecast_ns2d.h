// forecast_ns2d.h -- 2-D compressible Navier-Stokes forecast launcher (internal).
#pragma once

#include <cuda_runtime.h>

namespace mgk {

// one set of grids of the same size advanced by a stage launch
template <typename T>
struct NsGroup {
    T *u0, *s1, *s2;       // nprob states of 4 n^2 values each, and two scratch buffers of the same size
                           // (FP64: the stage buffers; FP32: s1 is the second state of the alternating steps)
    int n, nprob, tx, ty;  // points per side, grids, tiles per side
    int tile_begin;        // first tile of this group in a launch over several groups
    T inv_h, inv_2h, dt;
};

// tile shapes of the batched FP32 step kernel (points per tile, x by y):
// 0 = 32 x 32, 1 = 16 x 32, 2 = 32 x 16
constexpr int kNsTileShapes = 3;
int ns2d_tile_x(int shape);
int ns2d_tile_y(int shape);

// nsteps SSP-RK3 steps of every group of a device table (tile_begin ascending,
// all tiles of the given shape), FP32 states.
cudaError_t ns2d_forecast_table(const NsGroup<float> *d_groups, int ngroups, int tiles, int shape, int nsteps,
                                double gamma, double mu, double prandtl, cudaStream_t s);

// NULL if grids of n_whole (one member per CTA group) and n_split points per
// side can be advanced, else the reason.
const char *ns2d_check_size(int n_whole, int n_split);

// Scratch (elements of T) the forecast needs for its two stage buffers (FP32
// uses the first of the two).
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

// one step from u0 into s1 (it leaves the states untouched): timing probe of the autotuner
cudaError_t ns2d_probe_step(const NsGroup<float> *d_groups, int ngroups, int tiles, int shape, double gamma,
                                double mu, double prandtl, cudaStream_t s);

}  // namespace mgk
