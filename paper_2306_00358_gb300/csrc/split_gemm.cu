// Split-precision GEMM (TRG_SPLIT_BF16) -- placeholder until the tcgen05 kernel lands.
#include "internal.h"

namespace trg {

void gemm_split(Ctx& ctx, const GemmDesc& g) {
    (void)ctx;
    (void)g;
    fail(TRG_ENOTSUP, "split-precision GEMM not built yet");
}

}  // namespace trg
