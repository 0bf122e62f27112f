// Shared device helpers and host plumbing of libgrav (sm_103a).
//
// Device side: SFU reciprocal square root, error-free FP32/FP64 addition
// (TwoSum), the 1-D TMA bulk copy (cp.async.bulk) into shared memory with an
// mbarrier transaction count, and bounded mbarrier waits that report a timeout
// through the caller's flag word instead of spinning forever.
//
// Host side: thread-local error string, status helpers and cached device
// attributes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "grav.h"

namespace grav {

// ---------------------------------------------------------------------------
// Host plumbing
// ---------------------------------------------------------------------------

void set_error(const char *fmt, ...);
void clear_error();
int fail(int code, const char *fmt, ...);
// Returns GRAV_OK or GRAV_ECUDA (with the CUDA error text) for `e`.
int check_cuda(cudaError_t e, const char *what);
// Returns GRAV_OK or GRAV_ECUDA for the last launch error.
int check_launch(const char *what);
int device_sm_count(int *out);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Iteration bound of every mbarrier wait: far beyond any healthy copy
// (each try_wait may also suspend in hardware for a while).
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ void flag_or(int32_t *flags, int32_t bit)
{
    if (flags) atomicOr(flags, bit);
}

// SFU approximate 1/sqrt(x) (MUFU.RSQ), flush-to-zero.
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Knuth's TwoSum: hi + lo absorbs x exactly (lo accumulates the rounding
// errors).  Plain IEEE adds; the compiler may neither reassociate nor fuse.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    float t = __fadd_rn(hi, x);
    float z = __fsub_rn(t, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(x, z));
    lo = __fadd_rn(lo, e);
    hi = t;
}

__device__ __forceinline__ void two_sum_acc(double &hi, double &lo, double x)
{
    double t = __dadd_rn(hi, x);
    double z = __dsub_rn(t, hi);
    double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(t, z)), __dsub_rn(x, z));
    lo = __dadd_rn(lo, e);
    hi = t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier shared-memory accesses (generic proxy) before
// bulk copies it issues afterwards (async proxy) into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One elected thread: arm `bar` for `bytes` and start the 1-D bulk copy
// global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                            uint64_t *bar)
{
    uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(b)
        : "memory");
}

// One elected thread: arm `bar` for both copies' bytes and start two 1-D
// bulk copies global -> shared that complete on it.
__device__ __forceinline__ void tma_load_1d_two(void *dst1, const void *src1, uint32_t bytes1,
                                                void *dst2, const void *src2, uint32_t bytes2,
                                                uint64_t *bar)
{
    uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                 "r"(bytes1 + bytes2)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst1)),
        "l"(src1), "r"(bytes1), "r"(b)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst2)),
        "l"(src2), "r"(bytes2), "r"(b)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false (and GRAV_FLAG_TIMEOUT) if
// `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *flags,
                                                  uint32_t limit = kWaitLimit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    flag_or(flags, GRAV_FLAG_TIMEOUT);
    return false;
}

__device__ __forceinline__ bool finite3(double a, double b, double c)
{
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Tidal timestep, Eq. (tidaltimestep): sqrt(eta) * (||T||_F^2 / 6)^(-1/4),
// ||T||^2 summed in the fixed order xx, yy, zz, then 2xy^2, 2xz^2, 2yz^2,
// every operation correctly rounded (no contraction); +inf for T = 0.
__device__ __forceinline__ double tidal_dt(const double t[6], double sqrt_eta)
{
    double s = __dmul_rn(t[0], t[0]);
    s = __dadd_rn(s, __dmul_rn(t[1], t[1]));
    s = __dadd_rn(s, __dmul_rn(t[2], t[2]));
    s = __dadd_rn(s, __dmul_rn(2.0, __dmul_rn(t[3], t[3])));
    s = __dadd_rn(s, __dmul_rn(2.0, __dmul_rn(t[4], t[4])));
    s = __dadd_rn(s, __dmul_rn(2.0, __dmul_rn(t[5], t[5])));
    if (s == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
    return __ddiv_rn(sqrt_eta, __dsqrt_rn(__dsqrt_rn(__ddiv_rn(s, 6.0))));
}

}  // namespace grav
