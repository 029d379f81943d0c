// pending.cpp -- entry points whose implementation lands in a later unit.
#include "../../include/hrm.h"

extern "C" {
int hrm_autotune(int, int, int, int, int, int, unsigned, void*, hrm_plan*) { return HRM_ENOTSUP; }
int hrm_server_create(void*, size_t, int, int, hrm_server**) { return HRM_ENOTSUP; }
int hrm_submit(hrm_server*, const hrm_request*, uint64_t*) { return HRM_ENOTSUP; }
int hrm_poll(hrm_server*, uint64_t, int) { return HRM_ENOTSUP; }
double hrm_ticket_latency_us(hrm_server*, uint64_t) { return -1.0; }
int hrm_server_stats_get(hrm_server*, hrm_server_stats*) { return HRM_ENOTSUP; }
int hrm_server_destroy(hrm_server*) { return HRM_ENOTSUP; }
}
