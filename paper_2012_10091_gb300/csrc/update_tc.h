// update_tc.h -- tensor-core (tcgen05) member update, internal to the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace mgk {

// TMA descriptors and launch shape of the update for one handle's buffers.
struct UpdateTcPlan {
    CUtensorMap map_t;  // T^T, [ntpad][ldx] bf16, K-major, box 64 x ntpad
    CUtensorMap map_m;  // members, [ne][nx] fp32, box 128 points x ne members
    const float *members;
    int kblocks, ntile, tmem_cols, nx, ne;
    size_t smem;
    long long wait_limit;  // SM clock cycles the kernel waits for its operands (default about a second)
    bool ready;
};

// one problem of an update launch (the kernel's view)
struct UpdateProb {
    float *members, *dC;
    int *status;
    int nx, ne, kblocks, ntile;
    long long wait_limit;  // operand waits, SM clock cycles
    double inv_ne, isq;    // 1/Ne, 1/sqrt(Ne - 1) (host values)
};
constexpr int kUpdateLaunchMax = 96;  // problems per launch (tensor maps and scalars as parameters)

bool update_tc_supported(int ne, int ldx, int ntpad, int nx);
bool update_tc_prepare(UpdateTcPlan *plan, int ldx, int nx, const __nv_bfloat16 *Tt, int ntpad, int ne,
                       const float *members);
// members[c][p] += sum_a X[p][a] T[c][a] (c < ne), dC[p] = sum_a X[p][a] T[ne][a],
// with X the BF16 normalised anomalies of the members as they are on entry
// (formed in the kernel); `members` must be the buffer the plan was prepared for
cudaError_t launch_update_tc(const UpdateTcPlan &plan, float *members, float *dC, int *status, cudaStream_t s);
// the launch view of a handle's update
UpdateProb update_tc_prob(const UpdateTcPlan &plan, float *dC, int *status);
// dynamic shared memory of the update (operands and nbuf member tiles), and
// what a launch asks for so that its CTAs never oversubscribe TMEM
size_t update_tc_smem(int kblocks, int ntpad, int ne, int nbuf);
size_t update_tc_launch_smem(size_t smem, int tmem_cols);

// the update step of a grouped analysis (every problem of the plan)
struct GroupPlan;
cudaError_t launch_update_tc_group(const GroupPlan &plan, cudaStream_t s);

}  // namespace mgk
