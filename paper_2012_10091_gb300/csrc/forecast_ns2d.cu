// forecast_ns2d.cu -- 2-D compressible Navier-Stokes forecast (placeholder until
// the stencil kernel lands).
#include "forecast_ns2d.h"

namespace mgk {

const char *ns2d_check_size(int, int) { return "the NS-2D forecast kernel is not built in this version"; }

template <typename T>
cudaError_t ns2d_forecast(T *, int, int, T *, int, int, double, double, double, double, double, int,
                          cudaStream_t) {
    return cudaErrorNotSupported;
}

template cudaError_t ns2d_forecast<float>(float *, int, int, float *, int, int, double, double, double,
                                          double, double, int, cudaStream_t);
template cudaError_t ns2d_forecast<double>(double *, int, int, double *, int, int, double, double,
                                           double, double, double, int, cudaStream_t);

}  // namespace mgk
