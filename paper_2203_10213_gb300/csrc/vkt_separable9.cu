// vkt_separable9.cu -- the single-volume separable kernels for k = 9 (vkt_separable.cuh).
#include "vkt_separable.cuh"

namespace vkt {

vktError launch_separable_k9(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx)
{
    return sepk::launch_k<9>(job, gx, gy, gz, ctx);
}

}  // namespace vkt
