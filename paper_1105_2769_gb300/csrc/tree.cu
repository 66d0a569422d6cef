// Multi-tree approximation (Algorithm 2 with the p = 0 rules of Sec. 4).
#include "mbm_tree_api.h"

mbm_status mbm_tree_potential(mbm_ctx*, const double*, int64_t, double, double, bool,
                              const mbm_config&, mbm_tree*, double*, mbm_stats*, cudaStream_t) {
    return mbm_fail(MBM_ENOTSUP, "tree path not built yet");
}
