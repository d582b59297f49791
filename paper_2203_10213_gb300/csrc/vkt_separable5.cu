// vkt_separable5.cu -- the single-volume separable kernels for k = 5 (vkt_separable.cuh).
#include "vkt_separable.cuh"

namespace vkt {

vktError launch_separable_k5(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx)
{
    return sepk::launch_k<5>(job, gx, gy, gz, ctx);
}

}  // namespace vkt
