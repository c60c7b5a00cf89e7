// ems_krylov.cu -- rational Krylov reduced model (Sec. IV-E, Alg. 1).
#include "ems_internal.cuh"

using namespace ems;

extern "C" ems_status ems_krylov_reduce(ems_ctx *c, int q, double eta, int *n_reduced, int *n_fallback) {
    if (!c) return EMS_E_INVAL;
    (void)q; (void)eta;
    if (n_reduced) *n_reduced = 0;
    if (n_fallback) *n_fallback = 0;
    return fail(c, EMS_E_STATE, "Krylov reduction is not available in this build");
}
