// Batched persistent launch and autotuner (not yet available in this build).
#include "internal.cuh"

using namespace gbsp;

extern "C" {

gbsp_status gbsp_batch_plan(int32_t, const gbsp_batch_item *, int32_t, int64_t *) {
    set_error("batched launch not available in this build");
    return GBSP_ERR_UNSUPPORTED;
}
gbsp_status gbsp_batch_create(int32_t, const gbsp_batch_item *, int32_t, void *, int64_t, void *,
                              gbsp_batch *) {
    set_error("batched launch not available in this build");
    return GBSP_ERR_UNSUPPORTED;
}
gbsp_status gbsp_batch_run(gbsp_batch, int32_t *, void *) { return GBSP_ERR_UNSUPPORTED; }
gbsp_status gbsp_batch_destroy(gbsp_batch) { return GBSP_OK; }
gbsp_status gbsp_autotune(gbsp_handle, int32_t, const void *, void *, void *, gbsp_kernel_opts *,
                          float *) {
    set_error("autotuner not available in this build");
    return GBSP_ERR_UNSUPPORTED;
}

}  // extern "C"
