// server.cpp -- continuous-batching server (ata_server_*, ata_submit, ata_poll).
#include "runtime.h"

using namespace ata;

struct ata_server_s {};

extern "C" {

ata_status ata_server_create(ata_server* out, size_t budget, ata_dtype dtype, int max_inflight) {
    (void)budget;
    (void)dtype;
    (void)max_inflight;
    if (out) *out = nullptr;
    return fail(ATA_EUNSUPPORTED, "server not built");
}

ata_status ata_submit(ata_server, int64_t, int64_t, const void*, int64_t, double*, ata_ticket*) {
    return fail(ATA_EUNSUPPORTED, "server not built");
}

ata_status ata_poll(ata_server, ata_ticket, int) { return fail(ATA_EUNSUPPORTED, "server not built"); }

ata_status ata_server_stats(ata_server, double*, double*, int64_t*) {
    return fail(ATA_EUNSUPPORTED, "server not built");
}

void ata_server_destroy(ata_server) {}

}  // extern "C"
