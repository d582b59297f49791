// Batched entry point (placeholder until its kernel lands).
#include "vkt_internal.h"

extern "C" {

vktError vktApplyFilterBatchSV(int32_t, vktStructuredVolume*, vktStructuredVolume*, vktFilter*)
{
    return VKT_ERROR_UNSUPPORTED;
}

}
