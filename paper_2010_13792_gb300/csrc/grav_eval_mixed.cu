// Instantiations of the mixed-precision force kernel (K5) for the tile
// configurations the autotuner chooses from.
#include "grav_eval.cuh"

namespace grav {

#define GRAV_MIXED_CFG(NT, KT, S, MINB, U, SACC)                                              \
    {GRAV_MIXED, NT, KT, S,                                                                       \
     {launch_mixed<NT, KT, S, MINB, U, false, SACC>, launch_mixed<NT, KT, S, MINB, U, true, SACC>}, \
     {occupancy_mixed<NT, KT, S, MINB, U, false, SACC>,                                           \
      occupancy_mixed<NT, KT, S, MINB, U, true, SACC>},                                           \
     launch_pack<S, true, true>}

// threads, targets per thread, sources per tile, min CTAs per SM (register
// budget), unroll depth of the Newtonian loop, accumulators in shared memory
static const EvalConfig kMixedConfigs[] = {
    GRAV_MIXED_CFG(128, 1, 256, 4, 8, false),
    GRAV_MIXED_CFG(128, 1, 256, 6, 4, true),
    GRAV_MIXED_CFG(128, 2, 256, 4, 4, true),
    GRAV_MIXED_CFG(128, 2, 256, 4, 2, true),
    GRAV_MIXED_CFG(256, 1, 256, 3, 4, true),
    GRAV_MIXED_CFG(64, 2, 256, 8, 2, true),
    GRAV_MIXED_CFG(128, 1, 256, 5, 8, true),
    GRAV_MIXED_CFG(256, 1, 256, 2, 4, false),
};

const EvalConfig *mixed_configs(int *count)
{
    *count = (int)(sizeof(kMixedConfigs) / sizeof(kMixedConfigs[0]));
    return kMixedConfigs;
}

}  // namespace grav
