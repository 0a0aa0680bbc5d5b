// conv_tc.h -- tensor-core 3x3 convolutions of the learned correction,
// internal to the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mgk {

// elements of the packed weights of one CIN -> COUT layer ([9][groups][COUT][8])
int conv_packed_elems(int cin, int cout);
// W in [COUT][CIN][9] order -> the packed B operands of launch_conv_fwd_tc
cudaError_t launch_pack_conv_weights(const __nv_bfloat16 *W, int cin, int cout, __nv_bfloat16 *packed,
                                     cudaStream_t s);
// out = conv3x3_periodic(in, W) + bias (ReLU if RELU) for `batch` n x n maps;
// in: BF16 C8 layout; out: BF16 C8 (OUT_BF16) or FP32 [batch][COUT][n][n].
// A wait that expires records MGENKF_ERR_TIMEOUT in *status (may be NULL).
template <int CIN, int COUT, bool RELU, bool OUT_BF16>
cudaError_t launch_conv_fwd_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *wp, const float *bias, void *out, int n,
                               int batch, int *status, cudaStream_t s);

}  // namespace mgk
