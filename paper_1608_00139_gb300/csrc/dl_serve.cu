// dl_serve.cu -- asynchronous requests (dl_submit / dl_poll / dl_cancel).
#include "dl_ctx.h"

using namespace dl;

struct dl_ctx::Serve {};

void dl_serve_shutdown(dl_ctx *) {}

extern "C" {

dl_status dl_submit(dl_ctx *ctx, const dl_request *req, uint64_t *ticket) {
    (void)ctx; (void)req; (void)ticket;
    set_error("serving is not available in this build");
    return DL_ENOTIMPL;
}

dl_status dl_poll(dl_ctx *ctx, uint64_t ticket, int64_t timeout_us, dl_stats *stats) {
    (void)ctx; (void)ticket; (void)timeout_us; (void)stats;
    set_error("serving is not available in this build");
    return DL_ENOTIMPL;
}

dl_status dl_cancel(dl_ctx *ctx, uint64_t ticket) {
    (void)ctx; (void)ticket;
    set_error("serving is not available in this build");
    return DL_ENOTIMPL;
}

}  // extern "C"
