// forecast_ns2d.h -- 2-D compressible Navier-Stokes forecast launcher (internal).
#pragma once

#include <cuda_runtime.h>

namespace mgk {

// one set of grids of the same size advanced by a launch
template <typename T>
struct NsGroup {
    T *u0, *s1, *s2;       // nprob states of 4 n^2 values each, and two scratch buffers of the same size
                           // (FP64: the stage buffers; FP32: s1 is the second state of the alternating steps)
    int n, nprob, tx, ty;  // points per side, grids; FP32: bands and row segments per grid (FP64: tiles per side)
    int tile_begin;        // FP32: first unit of this group in a launch over several groups
    T inv_h, inv_2h, dt;
};

// Choices of the FP32 step (the batch's tuned "tile shape" per grid size):
// rows per segment of the march (shape mod 8: 0 = 32, 1 = 16, 2 = 64,
// 3 = 128, 4 = 256, 5 = 24, 6 = 48, 7 = 20; a grid of n rows is cut into
// ceil(n / rows) segments of equal length but the last) and the band width
// (shape / 8: 0 = the whole width up to 512 columns, 1 = bands of at most 122
// columns, 64 threads per CTA).
constexpr int kNsSegChoices = 8;
constexpr int kNsTileShapes = 2 * kNsSegChoices;
int ns2d_seg_rows(int shape);
bool ns2d_narrow(int shape);
// default choice for `grids` n x n grids stepped on their own: narrow bands
// above 256 points per side, the longest segments that still give two units
// per SM (`sms` SMs), else 16 rows
int ns2d_default_choice(int n, int grids, int sms);
// bands, row segments and threads per CTA of the FP32 step on an n x n grid
void ns2d_march_layout(int n, int shape, int *bands, int *segs, int *threads);

// nsteps SSP-RK3 steps of every group of a device table (tile_begin ascending,
// all groups of grid size n, units = bands x segments x grids in total), FP32
// states.
cudaError_t ns2d_forecast_table(const NsGroup<float> *d_groups, int ngroups, int units, int n, int nsteps,
                                double gamma, double mu, double prandtl, int shape, cudaStream_t s);

// NULL if grids of n_whole (one member per CTA group) and n_split points per
// side can be advanced, else the reason.
const char *ns2d_check_size(int n_whole, int n_split);

// Scratch (elements of T) the forecast needs for its two stage buffers (FP32
// uses the first of the two).
size_t ns2d_scratch_elems(int n_whole, int n_whole_probs, int n_split, int n_split_probs);

// Advance n_whole_probs grids of n_whole^2 x 4 and n_split_probs grids of
// n_split^2 x 4 conserved variables by nsteps SSP-RK3 steps, with caller
// scratch of ns2d_scratch_elems() elements.  FP32: with both groups (a
// handle's members and fine run, when its layout choice is -1) one launch of
// the tile kernel per step, with one group the column march.  (A handle's
// default steps each grid with ns2d_forecast_table on its own stream.)
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
cudaError_t ns2d_probe_step(const NsGroup<float> *d_groups, int ngroups, int units, int n, double gamma,
                            double mu, double prandtl, int shape, cudaStream_t s);

}  // namespace mgk
