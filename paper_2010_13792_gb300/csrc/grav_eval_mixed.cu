// Instantiations of the mixed-precision force kernel (K5) for the tile
// configurations the autotuner chooses from.
#include "grav_eval.cuh"

namespace grav {

#define GRAV_MIXED_CFG(NT, KT, S, MINB, U, SACC, PAIR)                                        \
    {GRAV_MIXED, NT, KT, S, U, SACC,                                                              \
     {launch_mixed<NT, KT, S, MINB, U, false, SACC, PAIR>,                                        \
      launch_mixed<NT, KT, S, MINB, U, true, SACC, PAIR>},                                        \
     {occupancy_mixed<NT, KT, S, MINB, U, false, SACC, PAIR>,                                     \
      occupancy_mixed<NT, KT, S, MINB, U, true, SACC, PAIR>},                                     \
     launch_pack<S, true, true, PAIR>,                                                            \
     {launch_mixed_batched<NT, KT, S, MINB, U, false, SACC, PAIR>,                                \
      launch_mixed_batched<NT, KT, S, MINB, U, true, SACC, PAIR>},                                \
     {occupancy_mixed_batched<NT, KT, S, MINB, U, false, SACC, PAIR>,                             \
      occupancy_mixed_batched<NT, KT, S, MINB, U, true, SACC, PAIR>},                             \
     launch_pack_batched<S, true, true, PAIR>, PAIR}

// threads, targets per thread, sources per tile, min CTAs per SM (register
// budget), unroll depth of the Newtonian loop, accumulators in shared memory,
// paired source layout (two sources per packed FP32x2 instruction)
static const EvalConfig kMixedConfigs[] = {
    GRAV_MIXED_CFG(128, 1, 256, 4, 8, false, false),
    GRAV_MIXED_CFG(128, 1, 256, 6, 4, true, false),
    GRAV_MIXED_CFG(128, 2, 256, 4, 4, true, false),
    GRAV_MIXED_CFG(128, 2, 256, 4, 2, true, false),
    GRAV_MIXED_CFG(256, 1, 256, 3, 4, true, false),
    GRAV_MIXED_CFG(64, 2, 256, 8, 2, true, false),
    GRAV_MIXED_CFG(128, 1, 256, 4, 2, false, true),
    GRAV_MIXED_CFG(128, 1, 256, 4, 4, false, true),
    GRAV_MIXED_CFG(128, 1, 256, 6, 2, true, true),
    GRAV_MIXED_CFG(256, 1, 256, 2, 2, false, true),
    GRAV_MIXED_CFG(128, 1, 256, 5, 4, true, true),
    GRAV_MIXED_CFG(256, 1, 256, 3, 2, true, true),
};
// (512-source tiles were measured 2% faster but their longer FP32 partial
// sums take the jerk's worst-case error past 1e-4 on dense inputs.)

const EvalConfig *mixed_configs(int *count)
{
    *count = (int)(sizeof(kMixedConfigs) / sizeof(kMixedConfigs[0]));
    return kMixedConfigs;
}

}  // namespace grav
