// serve.cu -- request loop (continuous batching).
#include "dsps_internal.cuh"

namespace dsps {

void set_last_error(const char *msg);

int serve_start(Ctx *) { return DSPS_OK; }
void serve_stop(Ctx *) {}
int serve_submit(Ctx *, const dsps_request *, uint64_t *) {
    set_last_error("dsps_submit: not built yet");
    return DSPS_ERR_UNSUPPORTED;
}
int serve_poll(Ctx *, uint64_t, int64_t, double *) {
    set_last_error("dsps_poll: not built yet");
    return DSPS_ERR_UNSUPPORTED;
}

}  // namespace dsps
