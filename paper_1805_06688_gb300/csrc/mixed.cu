// Mixed-precision MGRIT (tensor-core inner V-cycles with FP64 iterative refinement).
#include "sfde_internal.cuh"

sfde_status sfde_mgrit_mixed(sfde_ctx* c, const mgrit_opts* o, mgrit_stats* st) {
    (void)c; (void)o; (void)st;
    return SFDE_EUNSUPPORTED;
}

void sfde_free_mixed(sfde_ctx* c) { (void)c; }
