// exw_batched.cu -- persistent batched path (placeholder until the persistent kernel lands).
#include "exw_internal.h"

struct exw_tuner {
    int dummy;
};

extern "C" {

exw_tuner *exw_tuner_create(void) { return new exw_tuner{0}; }
void exw_tuner_destroy(exw_tuner *t) { delete t; }
size_t exw_tuner_report(const exw_tuner *, char *buf, size_t len) {
    if (buf && len) buf[0] = '\0';
    return 1;
}
size_t exw_batched_workspace_bytes(const exw_stream_desc *, int, int) { return 0; }
exw_status exw_extrapolate_batched(const exw_stream_desc *, int, int, unsigned, void *, size_t, exw_tuner *,
                                   exw_stream_t) {
    return EXW_ERR_UNSUPPORTED;
}

}  // extern "C"
