// K3 (tensor-core path): placeholder until the tcgen05 kernel lands.
#include "ie_internal.h"

namespace ie {

int tc_tile_columns() { return 128; }

ie_status prepare_translate_tc() { return IE_OK; }

ie_status launch_translate_tc(ie_plan, int, float2 *, int, cudaStream_t, const int *) {
    set_error("tensor-core translation not built");
    return IE_ERR_UNSUPPORTED;
}

}  // namespace ie
