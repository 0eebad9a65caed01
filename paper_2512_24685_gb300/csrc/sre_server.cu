// sre_server.cu -- continuous-batching M2 server (placeholder until built).
#include <cuda_runtime.h>

#include "sre.h"

extern "C" {

void sre_server_cfg_default(sre_server_cfg_t *cfg) {
    if (!cfg) return;
    cfg->hbm_budget_bytes = 8ull << 30;
    cfg->max_inflight = 32;
    cfg->max_queue = 4096;
    cfg->max_N = 20;
    cfg->mode = SRE_MODE_FP32;
    cfg->wait_limit_ns = 5000000000ull;
    cfg->device = 0;
}

sre_status_t sre_server_create(const sre_server_cfg_t *, sre_server_t *) { return SRE_EUNSUPPORTED; }
sre_status_t sre_server_submit(sre_server_t, const void *, int, int, sre_dtype_t, uint64_t *) {
    return SRE_EUNSUPPORTED;
}
sre_status_t sre_server_poll(sre_server_t, uint64_t, int *, double *) { return SRE_EUNSUPPORTED; }
sre_status_t sre_server_wait(sre_server_t, uint64_t, double, double *) { return SRE_EUNSUPPORTED; }
sre_status_t sre_server_stats(sre_server_t, sre_server_stats_t *) { return SRE_EUNSUPPORTED; }
sre_status_t sre_server_destroy(sre_server_t) { return SRE_OK; }

}  // extern "C"
