// batch_analysis.h -- grouped analysis of many independent NS-2D mixed-precision
// problems (internal to the library): each step of the analysis and correction
// (Algorithm 4 steps 4-5 with Algorithm 3 steps 2-3 and 7-8 inside) is one
// launch over all problems.  A launch's blocks are mapped to (problem, block of
// that problem) by a table, and every block runs the same kernel body as the
// single-problem launch, so a problem's results do not depend on the batch.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "analysis.h"
#include "update_tc.h"

namespace mgk {

// one problem of the grouped analysis (device table entry)
struct GroupProb {
    float *fine, *members, *xstar, *dC;
    const int32_t *tap_idx;  // H^C taps [ny][taps]
    const double *tap_w;
    const float *tap_wh, *tap_wl;  // the weights split into FP32 pairs (double-FP32 sums)
    const double *yo_in;  // this problem's observations (read by the innovation step)
    double *yo;           // copy of them in the problem's own buffer
    double *yf, *ybar, *eps, *Y, *Z;
    double *S, *Lt, *Bt;  // S = I + Y^T R^-1 Y and its factor; T (column c contiguous) in Bt
    double *part;         // split-K partial sums of the gain products
    DfOperands df;        // double-FP32 copies of Y and Z (the gain products' operands)
    double *innov;        // RMS of d* = y^o - H^C x^C*
    __nv_bfloat16 *Tt;
    int *status;
    uint64_t *cycle;  // analysis counter (keys the perturbations)
    uint64_t seed;
    double sigma, s2, inv_ne, isq;
    int nc, r, ne, ny, taps, ldx, nx;
    int splits, kchunk;              // gain products: K chunks (1: no split)
    int kblocks, ntile, tmem_cols;   // tensor-core update
    long long wait_limit;            // its operand wait, SM clock cycles
    ProlongWeights pw;
};

// steps of the grouped analysis, in launch order
enum GroupStep {
    kGsRestrict,     // x^C* = Pi_C(x^F), dC = 0
    kGsObsApply,     // H^C of the members and of x^C*
    kGsObsMean,      // observation means, d*, y^o check and copy
    kGsPerturb,      // perturbed observations, Y, Z
    kGsInnov,        // RMS of d*
    kGsGemm,         // S and Y^T R^-1 [D | d*] in double-FP32 arithmetic (tiles or K chunks)
    kGsReduce,       // sum of the K chunks
    kGsCholCluster,  // Cholesky of S, 8-CTA clusters (32 <= Ne <= 256)
    kGsChol,         // Cholesky of S, one CTA (Ne < 32)
    kGsSolve,        // T = S^-1 [Y^T R^-1 D | Y^T R^-1 d*], BF16 copy
    kGsUpdate,       // anomalies X, members += X T_i, dC = X T_ne (tensor cores)
    kGsProlong,      // x^F += Pi_F(dC), analysis counter + 1
    kGsSteps
};

constexpr int kSolveColsPerCta = 8;  // right-hand sides per CTA of the grouped solve

// host side of a grouped analysis: the device table, the block maps of every
// step and the launch shapes
struct GroupPlan {
    GroupProb *d_probs = nullptr;
    int2 *d_maps = nullptr;  // all steps' maps, one allocation: entry = (problem, block of the problem)
    int nprob = 0;
    int map_off[kGsSteps] = {}, nblocks[kGsSteps] = {};
    size_t chol_cluster_smem = 0, chol_smem = 0, solve_smem = 0;
    int solve_maxr = 4;
    // update: one launch per class of problems that fit the same number of
    // CTAs per SM (at most kUpdateLaunchMax problems each), over the tiles
    // [map_begin, map_end) of the update map (entry = (index in probs, tile))
    struct UpdateLaunch {
        std::vector<int> probs;
        int map_begin = 0, map_end = 0;
    };
    std::vector<UpdateLaunch> upd;
    std::vector<CUtensorMap> upd_maps;  // 2 per problem: T, members
    std::vector<UpdateProb> upd_probs;  // per problem
};

// Fills `plan` for the problems `probs` (host copies; pointers are device
// pointers) with their tensor maps and uploads the table and maps on stream s
// (synchronised before return).  Returns false if the problems do not fit the
// grouped kernels (the caller runs them one by one).
bool group_plan_build(GroupPlan *plan, const std::vector<GroupProb> &probs, const std::vector<CUtensorMap> &maps,
                      cudaStream_t s);
void group_plan_free(GroupPlan *plan);
// the whole grouped analysis and correction on stream s
cudaError_t group_analyse(const GroupPlan &plan, cudaStream_t s);
// whether a problem of Ne members, Ny observations fits the grouped kernels
bool group_supported(int ne, int ny);

}  // namespace mgk
