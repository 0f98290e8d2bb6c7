// Entry points whose kernels are not built yet: they report QTS_ERR_UNSUPPORTED.
#include "qts_internal.h"

using namespace qts;

extern "C" {

qts_status qts_batched_fwd_bwd(int32_t, const qts_request*, int32_t, qts_stream_t) {
    return fail(QTS_ERR_UNSUPPORTED, "qts_batched_fwd_bwd is not built yet");
}

qts_status qts_autotune(qts_ensemble*, const float*, int64_t, int32_t, const char*, qts_stream_t) {
    return fail(QTS_ERR_UNSUPPORTED, "qts_autotune is not built yet");
}

}
