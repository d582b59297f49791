// vkt_separable.cu -- ApplyFilter for a rank-1 filter w[c][b][a] = gz[c] gy[b] gx[a]
// (the Gaussian blur of Sec. 4.3 is one), as three fused 1-D passes; one launch per
// volume, one brick per CTA.  The brick pipeline lives in vkt_sep_brick.cuh, the kernels
// and their launcher in vkt_separable.cuh; this unit holds k = 1 and 3 and the dispatch.
#include "vkt_separable.cuh"

namespace vkt {

vktError launch_separable_k1(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx)
{
    return sepk::launch_k<1>(job, gx, gy, gz, ctx);
}

vktError launch_separable_k3(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx)
{
    return sepk::launch_k<3>(job, gx, gy, gz, ctx);
}

vktError launch_separable(const Job& job, const float* gx, const float* gy, const float* gz,
                          int k, const Ctx& ctx)
{
    switch (k) {
    case 1: return launch_separable_k1(job, gx, gy, gz, ctx);
    case 3: return launch_separable_k3(job, gx, gy, gz, ctx);
    case 5: return launch_separable_k5(job, gx, gy, gz, ctx);
    case 7: return launch_separable_k7(job, gx, gy, gz, ctx);
    case 9: return launch_separable_k9(job, gx, gy, gz, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

}  // namespace vkt
