// vkt_direct_comp.cu -- the direct kernels with compensated accumulation (Dot2 pairs and
// a double-float rounding decision), for integer destinations whose FP32 error bound could
// flip a code; the kernel template lives in vkt_direct.cuh.
#include "vkt_direct.cuh"

namespace vkt {

vktError launch_direct_comp(const Job& job, const float* w, int k, const Ctx& ctx)
{
    switch (k) {
    case 1: return dir::launch_k<1, false, true>(job, w, ctx);
    case 3: return dir::launch_k<3, false, true>(job, w, ctx);
    case 5: return dir::launch_k<5, false, true>(job, w, ctx);
    case 7: return dir::launch_k<7, false, true>(job, w, ctx);
    case 9: return dir::launch_k<9, false, true>(job, w, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

}  // namespace vkt
