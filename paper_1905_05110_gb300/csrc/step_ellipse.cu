// Instantiations of the fused step kernel for an elliptic body (the disk's
// are in step_kernels.cu): a separate translation unit, so the two compile
// in parallel and the disk kernels keep their own register allocation.
#include "step_scalar.cuh"

namespace vplbm {

cudaError_t launch_step_ellipse(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb)
{
    return launch_step_shape<VPLBM_SHAPE_ELLIPSE>(precision, p, bx, by, stream, minb);
}

}  // namespace vplbm
