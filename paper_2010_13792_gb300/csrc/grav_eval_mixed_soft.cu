// Adaptive-softening instantiations of the mixed-precision force kernel (K5):
// per-element supports, pair-averaged kernels and the correction term, one
// per tile configuration (single-system launch); the table that points at
// them is built in grav_eval_mixed.cu.
#include "grav_eval_mixed_cfg.cuh"

namespace grav {

#define GRAV_MIXED_DEFINE(NT, KT, S, MINB, U, SACC, PAIR) \
    GRAV_MIXED_MODE_FNS(template, kModeSoft, NT, KT, S, MINB, U, SACC, PAIR)
GRAV_MIXED_CONFIG_LIST(GRAV_MIXED_DEFINE)

}  // namespace grav
