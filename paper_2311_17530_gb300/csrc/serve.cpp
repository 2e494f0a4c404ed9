// Serving entry points (continuous batching); filled in by the serving loop.
#include "api_internal.h"

using namespace msadp;

extern "C" {

int msa_submit(const msa_request *req, uint64_t *out_handle) {
    (void)req;
    (void)out_handle;
    return set_error(MSA_EINVAL, "serving loop not built yet");
}

int msa_poll(uint64_t handle, int32_t *out_score, char *out_alignment) {
    (void)handle;
    (void)out_score;
    (void)out_alignment;
    return set_error(MSA_EBADHANDLE, "unknown handle");
}

int msa_cancel(uint64_t handle) {
    (void)handle;
    return set_error(MSA_EBADHANDLE, "unknown handle");
}

int msa_drain(void) { return MSA_OK; }

}  // extern "C"
