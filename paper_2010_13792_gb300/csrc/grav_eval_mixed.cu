// Instantiations of the mixed-precision force kernel (K5) for the tile
// configurations the autotuner chooses from (open boundaries here; the
// periodic-box and adaptive-softening kernels are instantiated in
// grav_eval_mixed_periodic.cu and grav_eval_mixed_soft.cu).
#include "grav_eval_mixed_cfg.cuh"

namespace grav {

#define GRAV_MIXED_EXTERN(NT, KT, S, MINB, U, SACC, PAIR)                                   \
    GRAV_MIXED_MODE_FNS(extern template, kModePeriodic, NT, KT, S, MINB, U, SACC, PAIR)        \
    GRAV_MIXED_BATCHED_FNS(extern template, kModePeriodic, NT, KT, S, MINB, U, SACC, PAIR)     \
    GRAV_MIXED_MODE_FNS(extern template, kModeSoft, NT, KT, S, MINB, U, SACC, PAIR)
GRAV_MIXED_CONFIG_LIST(GRAV_MIXED_EXTERN)

#define GRAV_MIXED_FN3(FN, NT, KT, S, MINB, U, SACC, PAIR)                                  \
    {{FN<NT, KT, S, MINB, U, false, SACC, PAIR, kModeOpen>,                                  \
      FN<NT, KT, S, MINB, U, true, SACC, PAIR, kModeOpen>},                                  \
     {FN<NT, KT, S, MINB, U, false, SACC, PAIR, kModePeriodic>,                              \
      FN<NT, KT, S, MINB, U, true, SACC, PAIR, kModePeriodic>},                              \
     {FN<NT, KT, S, MINB, U, false, SACC, PAIR, kModeSoft>,                                  \
      FN<NT, KT, S, MINB, U, true, SACC, PAIR, kModeSoft>}}

#define GRAV_MIXED_FN2(FN, NT, KT, S, MINB, U, SACC, PAIR)                                  \
    {{FN<NT, KT, S, MINB, U, false, SACC, PAIR, kModeOpen>,                                  \
      FN<NT, KT, S, MINB, U, true, SACC, PAIR, kModeOpen>},                                  \
     {FN<NT, KT, S, MINB, U, false, SACC, PAIR, kModePeriodic>,                              \
      FN<NT, KT, S, MINB, U, true, SACC, PAIR, kModePeriodic>}}

#define GRAV_MIXED_CFG(NT, KT, S, MINB, U, SACC, PAIR)                                      \
    {GRAV_MIXED, NT, KT, S, U, SACC,                                                          \
     GRAV_MIXED_FN3(launch_mixed, NT, KT, S, MINB, U, SACC, PAIR),                            \
     GRAV_MIXED_FN3(occupancy_mixed, NT, KT, S, MINB, U, SACC, PAIR),                         \
     launch_pack<S, true, true, PAIR>,                                                        \
     GRAV_MIXED_FN2(launch_mixed_batched, NT, KT, S, MINB, U, SACC, PAIR),                    \
     GRAV_MIXED_FN2(occupancy_mixed_batched, NT, KT, S, MINB, U, SACC, PAIR),                 \
     launch_pack_batched<S, true, true, PAIR>, PAIR},

static const EvalConfig kMixedConfigs[] = {GRAV_MIXED_CONFIG_LIST(GRAV_MIXED_CFG)};
static_assert(sizeof(kMixedConfigs) / sizeof(kMixedConfigs[0]) <= kMaxTileConfigs,
              "more tile configurations than the host caches hold");

const EvalConfig *mixed_configs(int *count)
{
    *count = (int)(sizeof(kMixedConfigs) / sizeof(kMixedConfigs[0]));
    return kMixedConfigs;
}

}  // namespace grav
