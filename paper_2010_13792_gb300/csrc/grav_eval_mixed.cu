// Instantiations of the mixed-precision force kernel (K5) for the tile
// configurations the autotuner chooses from.
#include "grav_eval.cuh"

namespace grav {

#define GRAV_MIXED_CFG(NT, KT, S, MINB)                                                       \
    {GRAV_MIXED, NT, KT, S,                                                                   \
     {launch_mixed<NT, KT, S, MINB, false>, launch_mixed<NT, KT, S, MINB, true>},             \
     {occupancy_mixed<NT, KT, S, MINB, false>, occupancy_mixed<NT, KT, S, MINB, true>},       \
     launch_pack<S, true>}

static const EvalConfig kMixedConfigs[] = {
    GRAV_MIXED_CFG(128, 1, 256, 4),
    GRAV_MIXED_CFG(128, 2, 256, 3),
    GRAV_MIXED_CFG(256, 1, 256, 2),
    GRAV_MIXED_CFG(64, 2, 256, 6),
    GRAV_MIXED_CFG(128, 2, 128, 3),
};

const EvalConfig *mixed_configs(int *count)
{
    *count = (int)(sizeof(kMixedConfigs) / sizeof(kMixedConfigs[0]));
    return kMixedConfigs;
}

}  // namespace grav
