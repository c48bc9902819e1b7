// Reverse-time adjoint of the stream-collide step (placeholder until the adjoint kernels land).
#include "lbem_internal.cuh"

namespace lbk {
void adjoint_free(lbem_t *h) { (void)h; }
}  // namespace lbk

using namespace lbk;
extern "C" {
lbem_status lbem_forward_record(lbem_t *h, int nsteps, int checkpoint_every) {
    (void)h; (void)nsteps; (void)checkpoint_every;
    return fail(LBEM_ERR_STATE, "lbem_forward_record: not available in this build");
}
lbem_status lbem_adjoint(lbem_t *h, const float *trace_cot, float *grad_eps, double *grad_cL2) {
    (void)h; (void)trace_cot; (void)grad_eps; (void)grad_cL2;
    return fail(LBEM_ERR_STATE, "lbem_adjoint: not available in this build");
}
}
