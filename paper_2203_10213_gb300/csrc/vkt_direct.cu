// vkt_direct.cu -- the direct kernels with float accumulation (forward, any destination
// whose FP32 error bound keeps its codes exact, and the adjoint of the backward pass); the
// kernel template lives in vkt_direct.cuh.
#include "vkt_direct.cuh"

namespace vkt {

vktError launch_direct(const Job& job, const float* w, int k, const Ctx& ctx)
{
    if (job.comp) return launch_direct_comp(job, w, k, ctx);
    switch (k) {
    case 1: return dir::launch_k<1, false>(job, w, ctx);
    case 3:
        return dir::direct_small(job, ctx.sms) ? dir::launch_k<3, false, false, 1>(job, w, ctx)
                                      : dir::launch_k<3, false>(job, w, ctx);
    case 5: return dir::launch_k<5, false>(job, w, ctx);
    case 7: return dir::launch_k<7, false>(job, w, ctx);
    case 9: return dir::launch_k<9, false>(job, w, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

vktError launch_adjoint(const Job& job, const float* w, int k, const Ctx& ctx)
{
    switch (k) {
    case 1: return dir::launch_k<1, true>(job, w, ctx);
    case 3: return dir::launch_k<3, true>(job, w, ctx);
    case 5: return dir::launch_k<5, true>(job, w, ctx);
    case 7: return dir::launch_k<7, true>(job, w, ctx);
    case 9: return dir::launch_k<9, true>(job, w, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

}  // namespace vkt
