// Batched stepping of independent media (placeholder until the batched kernel lands).
#include "lbem_internal.cuh"

using namespace lbk;
extern "C" {
lbem_status lbem_batch_create(int n, lbem_t *const *members, void *stream, lbem_batch_t **out) {
    (void)n; (void)members; (void)stream; (void)out;
    return fail(LBEM_ERR_STATE, "lbem_batch_create: not available in this build");
}
lbem_status lbem_batch_step(lbem_batch_t *b, int nsteps) { (void)b; (void)nsteps; return fail(LBEM_ERR_STATE, "not available"); }
lbem_status lbem_batch_autotune(lbem_batch_t *b, int trial_steps, int *best) {
    (void)b; (void)trial_steps; (void)best;
    return fail(LBEM_ERR_STATE, "not available");
}
void lbem_batch_destroy(lbem_batch_t *b) { (void)b; }
}
