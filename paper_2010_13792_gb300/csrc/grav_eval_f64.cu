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
     launch_pack<S, false, true, false>, GRAV_F64_FN2(launch_f64_batched, NT, S),                  \
     GRAV_F64_FN2(occupancy_f64_batched, NT, S), launch_pack_batched<S, false, true, false>, false}

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

void launch_reduce(const EvalArgs &a, int32_t BT, bool pot, bool etrace, int64_t n_targets,
                   cudaStream_t st)
{
    const int tpb = pot ? reduce_targets_per_block<true>() : reduce_targets_per_block<false>();
    int sms = 0;
    if (device_sm_count(&sms) != GRAV_OK || sms <= 0) sms = 1;
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_targets + tpb - 1) / tpb, 8LL * sms));
    if (pot && etrace)
        reduce_partials_kernel<true, true><<<blocks, kReduceThreads, 0, st>>>(a, BT);
    else if (pot)
        reduce_partials_kernel<true, false><<<blocks, kReduceThreads, 0, st>>>(a, BT);
    else if (etrace)
        reduce_partials_kernel<false, true><<<blocks, kReduceThreads, 0, st>>>(a, BT);
    else
        reduce_partials_kernel<false, false><<<blocks, kReduceThreads, 0, st>>>(a, BT);
}

}  // namespace grav
