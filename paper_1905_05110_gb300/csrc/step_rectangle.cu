// Instantiations of the fused step kernel for a rectangular body (the disk's
// are in step_kernels.cu, the ellipse's in step_ellipse.cu).
#include "step_scalar.cuh"

namespace vplbm {

cudaError_t launch_step_rectangle(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb)
{
    return launch_step_shape<VPLBM_SHAPE_RECTANGLE>(precision, p, bx, by, stream, minb);
}

}  // namespace vplbm
