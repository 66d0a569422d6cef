// Forces and vector-Jacobian products of Phi.
#include "mbm_internal.h"

extern "C" mbm_status mbm_forces(mbm_ctx*, const double*, int64_t, double, double, int, double*,
                                 mbm_stream_t) {
    return mbm_fail(MBM_ENOTSUP, "forces not built yet");
}

extern "C" mbm_status mbm_potential_vjp(mbm_ctx*, const double*, int64_t, const double*, int,
                                        double*, mbm_stream_t) {
    return mbm_fail(MBM_ENOTSUP, "vjp not built yet");
}
