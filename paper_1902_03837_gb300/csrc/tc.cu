// Split-precision tensor-core contraction for the mixed mode (placeholder
// until the tcgen05 kernel lands).
#include "ctx.cuh"

namespace chi0 {

chi0_status tc_build_chi0(chi0_ctx* c, const void*, const double*, int64_t, int, int, double2*) {
  return ctx_fail(c, CHI0_EUNSUPPORTED, "mixed-precision contraction not built yet");
}

void tc_release(chi0_ctx*) {}

}  // namespace chi0
