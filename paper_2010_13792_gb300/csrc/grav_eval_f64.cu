// Instantiations of the FP64 force kernel (K4) and of the split reduction (K9).
#include "grav_eval.cuh"

namespace grav {

#define GRAV_F64_FN3(FN, NT, S)                                                                   \
    {{FN<NT, S, false, kModeOpen>, FN<NT, S, true, kModeOpen>},                                      \
     {FN<NT, S, false, kModePeriodic>, FN<NT, S, true, kModePeriodic>},                              \
     {FN<NT, S, false, kModeSoft>, FN<NT, S, true, kModeSoft>}}

#define GRAV_F64_FN2(FN, NT, S)                                                                   \
    {{FN<NT, S, false, kModeOpen>, FN<NT, S, true, kModeOpen>},                                      \
     {FN<NT, S, false, kModePeriodic>, FN<NT, S, true, kModePeriodic>}}

#define GRAV_F64_CFG(NT, S)                                                                       \
    {GRAV_F64, NT, 1, S, 4, 0, GRAV_F64_FN3(launch_f64, NT, S), GRAV_F64_FN3(occupancy_f64, NT, S), \
     launch_pack<S, false, false, false>, GRAV_F64_FN2(launch_f64_batched, NT, S),                 \
     GRAV_F64_FN2(occupancy_f64_batched, NT, S), launch_pack_batched<S, false, false, false>, false}

static const EvalConfig kF64Configs[] = {
    GRAV_F64_CFG(128, 128),
    GRAV_F64_CFG(64, 128),
    GRAV_F64_CFG(256, 64),
};

const EvalConfig *f64_configs(int *count)
{
    *count = (int)(sizeof(kF64Configs) / sizeof(kF64Configs[0]));
    return kF64Configs;
}

void launch_reduce(const EvalArgs &a, int32_t BT, bool pot, bool etrace, int blocks, cudaStream_t st)
{
    if (pot && etrace)
        reduce_partials_kernel<true, true><<<blocks, 256, 0, st>>>(a, BT);
    else if (pot)
        reduce_partials_kernel<true, false><<<blocks, 256, 0, st>>>(a, BT);
    else if (etrace)
        reduce_partials_kernel<false, true><<<blocks, 256, 0, st>>>(a, BT);
    else
        reduce_partials_kernel<false, false><<<blocks, 256, 0, st>>>(a, BT);
}

}  // namespace grav
