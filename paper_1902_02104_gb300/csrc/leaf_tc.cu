// leaf_tc.cu -- tensor-core leaf products (bf16x3 / TF32 / FP64 emulation).
#include "runtime.h"

namespace ata {

bool leaf_supported(LeafKind k) { return k == LEAF_F64; }

ata_status launch_leaf_tc(const DeviceTables& t, const Bind* binds, int nb, cudaStream_t s) {
    (void)t;
    (void)binds;
    (void)nb;
    (void)s;
    return fail(ATA_EUNSUPPORTED, "tensor-core leaves are not built into this library");
}

}  // namespace ata
