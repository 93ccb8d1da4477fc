// tc_conv.cu - tensor-core (tcgen05) fused teacher path. (in progress)
#include "internal.h"

namespace mb {
mb_status tc_prepare(mb_net*) { return MB_OK; }
void tc_release(mb_net*) {}
mb_status tc_infer_blocks(mb_net*, const mb_block*, int, const int64_t*, const int64_t*, const int64_t*,
                          const int64_t*, mb_out_type, cudaStream_t, bool) {
    set_error("tensor-core path not built yet");
    return MB_ERR_UNSUPPORTED;
}
}  // namespace mb

extern "C" mb_status mb_autotune(mb_net*, int64_t, int64_t, int64_t, const char*, int32_t*, void*) {
    mb::set_error("autotuner not built yet");
    return MB_ERR_UNSUPPORTED;
}
