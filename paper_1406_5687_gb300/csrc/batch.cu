// batch.cu -- batched counting (placeholder until the packed path lands).
#include "graph.cuh"

extern "C" {
tc_status tc_batch_create(const tc_graph_t*, int32_t, const tc_options*, tc_stream_t, tc_batch_t* out) {
    if (out) *out = nullptr;
    return TC_ERR_UNSUPPORTED;
}
tc_status tc_batch_run(tc_batch_t, tc_stream_t, uint64_t*) { return TC_ERR_UNSUPPORTED; }
void tc_batch_free(tc_batch_t) {}
tc_status tc_batch_count(const tc_graph_t*, int32_t, tc_stream_t, uint64_t*) { return TC_ERR_UNSUPPORTED; }
tc_status tc_build_batch(const int32_t* const*, const int32_t* const*, const int64_t*, const int32_t*, int32_t,
                         const tc_options*, tc_stream_t, tc_graph_t*) {
    return TC_ERR_UNSUPPORTED;
}
tc_status tc_server_create(int64_t, int32_t, const tc_options*, tc_server_t* out) {
    if (out) *out = nullptr;
    return TC_ERR_UNSUPPORTED;
}
tc_status tc_server_submit(tc_server_t, const int32_t*, const int32_t*, int64_t, int32_t, uint64_t) {
    return TC_ERR_UNSUPPORTED;
}
tc_status tc_server_poll(tc_server_t, tc_result*, int32_t, int32_t*) { return TC_ERR_UNSUPPORTED; }
tc_status tc_server_drain(tc_server_t, int64_t) { return TC_ERR_UNSUPPORTED; }
void tc_server_destroy(tc_server_t) {}
}
