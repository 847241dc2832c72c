// server.cpp -- continuous-batching field-query server (declared in include/nebem.h).
#include <cstring>

#include "context.h"

using namespace nb;

extern "C" {

int nebem_server_default_options(nebem_server_options* opt) {
    if (!opt) return fail(NEBEM_INVALID_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->arena_points = 4194304;
    opt->chunk_points = 1024;
    opt->max_requests = 256;
    opt->workers = 0;
    opt->idle_us = 2000;
    return NEBEM_OK;
}

int nebem_server_create(nebem_server** out, nebem_ctx* const* ctxs, int32_t n_ctx, const nebem_server_options* opt) {
    (void)out; (void)ctxs; (void)n_ctx; (void)opt;
    return fail(NEBEM_BAD_STATE, "server not built yet");
}
int nebem_server_submit(nebem_server*, int32_t, const double*, int64_t, double*, double*, int32_t, int64_t*) {
    return fail(NEBEM_BAD_STATE, "server not built yet");
}
int nebem_server_poll(nebem_server*, int64_t, int32_t*) { return fail(NEBEM_BAD_STATE, "server not built yet"); }
int nebem_server_wait(nebem_server*, int64_t, int64_t) { return fail(NEBEM_BAD_STATE, "server not built yet"); }
int nebem_server_request_times(nebem_server*, int64_t, double*, double*, double*) {
    return fail(NEBEM_BAD_STATE, "server not built yet");
}
int nebem_server_destroy(nebem_server*) { return NEBEM_OK; }

}  // extern "C"
