// Batched and backward entry points (placeholders until their kernels land).
#include "vkt_internal.h"

extern "C" {

vktError vktApplyFilterBatchSV(int32_t, vktStructuredVolume*, vktStructuredVolume*, vktFilter*)
{
    return VKT_ERROR_UNSUPPORTED;
}

vktError vktApplyFilterBackwardSV(vktStructuredVolume, float*, vktStructuredVolume,
                                  vktStructuredVolume, vktFilter)
{
    return VKT_ERROR_UNSUPPORTED;
}

}
