// student.cu - distilled student: training kernels and the multi-pass cascade. (in progress)
#include "internal.h"

namespace mb {
mb_status student_loss_grad(mb_net*, const uint8_t*, const float*, int64_t, int64_t, int64_t, double*, float*,
                            cudaStream_t) {
    set_error("student training not built yet");
    return MB_ERR_UNSUPPORTED;
}
mb_status student_train(mb_net*, const uint8_t*, const float*, int64_t, int64_t, int64_t, const mb_train_cfg*,
                        const char*, float*, cudaStream_t) {
    set_error("student training not built yet");
    return MB_ERR_UNSUPPORTED;
}
mb_status cascade(mb_net*, mb_net*, const uint8_t*, int64_t, int64_t, int64_t, float*, int, float, float, float,
                  double*, uint8_t*, cudaStream_t) {
    set_error("cascade not built yet");
    return MB_ERR_UNSUPPORTED;
}
}  // namespace mb
