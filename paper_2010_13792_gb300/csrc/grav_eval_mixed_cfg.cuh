// Tile configurations of the mixed-precision force kernel (K5), listed once
// for the translation units that instantiate them: open boundaries in
// grav_eval_mixed.cu, the periodic box in grav_eval_mixed_periodic.cu and
// per-element adaptive softening in grav_eval_mixed_soft.cu (each mode is a
// separate instantiation, so the open kernels carry none of the other modes'
// code and keep their register allocation).
#pragma once

#include "grav_eval.cuh"

// X(threads, targets per thread, sources per tile, min CTAs per SM (register
//   budget), unroll depth of the Newtonian loop, accumulators in shared
//   memory, paired source layout (two sources per packed FP32x2 instruction))
#define GRAV_MIXED_CONFIG_LIST(X)          \
    X(128, 1, 256, 4, 8, false, false)     \
    X(128, 1, 256, 6, 4, true, false)      \
    X(128, 2, 256, 4, 4, true, false)      \
    X(128, 2, 256, 4, 2, true, false)      \
    X(256, 1, 256, 3, 4, true, false)      \
    X(64, 2, 256, 8, 2, true, false)       \
    X(128, 1, 256, 4, 2, false, true)      \
    X(128, 1, 256, 4, 4, false, true)      \
    X(128, 1, 256, 6, 2, true, true)       \
    X(256, 1, 256, 2, 2, false, true)      \
    X(128, 1, 256, 5, 4, true, true)       \
    X(256, 1, 256, 3, 2, true, true)       \
    X(128, 2, 256, 4, 1, true, true)       \
    X(128, 2, 256, 4, 2, true, true)       \
    X(64, 2, 256, 8, 1, true, true)        \
    X(256, 2, 256, 2, 1, true, true)       \
    X(384, 1, 256, 2, 4, true, true)       \
    X(768, 1, 256, 1, 4, true, true)       \
    X(768, 1, 256, 1, 8, true, true)       \
    X(384, 1, 256, 2, 8, true, true)
// (512-source tiles were measured 2% faster but their longer FP32 partial
// sums take the jerk's worst-case error past 1e-4 on dense inputs.)

// The launchers of one configuration in one mode (kModePeriodic with the
// batched launch, kModeSoft without): declared `extern` where the table is
// built, defined in the mode's own translation unit.
#define GRAV_MIXED_MODE_FNS(PREFIX, MODE, NT, KT, S, MINB, U, SACC, PAIR)                           \
    PREFIX void launch_mixed<NT, KT, S, MINB, U, false, SACC, PAIR, MODE>(const EvalArgs &, int,      \
                                                                           cudaStream_t);             \
    PREFIX void launch_mixed<NT, KT, S, MINB, U, true, SACC, PAIR, MODE>(const EvalArgs &, int,       \
                                                                          cudaStream_t);              \
    PREFIX int occupancy_mixed<NT, KT, S, MINB, U, false, SACC, PAIR, MODE>(int *);                   \
    PREFIX int occupancy_mixed<NT, KT, S, MINB, U, true, SACC, PAIR, MODE>(int *);

#define GRAV_MIXED_BATCHED_FNS(PREFIX, MODE, NT, KT, S, MINB, U, SACC, PAIR)                        \
    PREFIX void launch_mixed_batched<NT, KT, S, MINB, U, false, SACC, PAIR, MODE>(                     \
        const EvalArgs &, const BatchView &, int, cudaStream_t);                                      \
    PREFIX void launch_mixed_batched<NT, KT, S, MINB, U, true, SACC, PAIR, MODE>(                      \
        const EvalArgs &, const BatchView &, int, cudaStream_t);                                      \
    PREFIX int occupancy_mixed_batched<NT, KT, S, MINB, U, false, SACC, PAIR, MODE>(int *);           \
    PREFIX int occupancy_mixed_batched<NT, KT, S, MINB, U, true, SACC, PAIR, MODE>(int *);
