// vkt_tc.cu -- tensor-core evaluation path (placeholder until the tcgen05 kernel lands).
#include "vkt_internal.h"

namespace vkt {

vktError tensor_available(const vktStructuredVolume_impl*, const vktStructuredVolume_impl*,
                          const vktFilter_impl*)
{
    return VKT_ERROR_UNSUPPORTED;
}

vktError launch_tensor(const Job&, const float*, int, const Ctx&) { return VKT_ERROR_UNSUPPORTED; }

}  // namespace vkt
