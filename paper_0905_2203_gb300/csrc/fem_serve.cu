// fem_serve.cu -- serving loop (placeholder until the loop lands).
#include "fem_internal.cuh"

extern "C" int fem_server_create(int, size_t, int, fem_server **out) {
    if (out) *out = nullptr;
    return FEM_ERR_INVAL;
}
extern "C" int fem_server_submit(fem_server *, const uint16_t *, const int32_t *, int64_t, uint32_t, const int32_t *,
                                 const int32_t *, int, uint32_t, int, uint64_t *) {
    return FEM_ERR_INVAL;
}
extern "C" int fem_server_wait(fem_server *, uint64_t, int, fem_result **, fem_job_info *) { return FEM_ERR_INVAL; }
extern "C" void fem_server_destroy(fem_server *) {}
