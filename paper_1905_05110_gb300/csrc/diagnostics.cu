// Diagnostic entry point: the FP32 reciprocal of the step kernels on an
// array, so that its error can be measured against the correctly rounded
// 1/x (the step kernels take 1/rho with it for u = j / rho, Eq. 22).
#include <stdio.h>

#include "vplbm_node.cuh"

namespace vplbm {
vplbm_status report_error(vplbm_status st, const char *msg);

namespace {

__global__ void recip_kernel(const float *__restrict__ x, float *__restrict__ y, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) y[k] = recip(x[k]);
}

}  // namespace
}  // namespace vplbm

extern "C" vplbm_status vplbm_eval_recip_f32(const float *x_dev, float *y_dev, long long n, void *cuda_stream)
{
    using namespace vplbm;
    if (n < 0 || (n > 0 && (!x_dev || !y_dev))) return report_error(VPLBM_EINVAL, "x_dev, y_dev and n >= 0 required");
    if ((uintptr_t)x_dev % 4 || (uintptr_t)y_dev % 4) return report_error(VPLBM_EINVAL, "x_dev, y_dev must be 4-byte aligned");
    if (n == 0) return VPLBM_OK;
    const long long blocks = (n + 255) / 256;
    recip_kernel<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, (cudaStream_t)cuda_stream>>>(x_dev, y_dev, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "vplbm_eval_recip_f32 launch failed: %s", cudaGetErrorString(e));
        return report_error(VPLBM_ECUDA, msg);
    }
    return VPLBM_OK;
}
