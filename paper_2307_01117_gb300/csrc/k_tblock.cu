// k_tblock.cu -- form HEAT_FORM_TBLOCK (placeholder until the temporal-blocking kernel lands).
#include "heat_internal.cuh"
namespace heat {
int run_tblock(heat_ctx *, int64_t) { return HEAT_ENOTSUP; }
}  // namespace heat
