// Selection side of the adaptive-force-update path (Grudic 2020, Sections 2-3):
//   K1 select_due   -- Eq. (3) counter update and Eq. (updatecondition) test
//   K2 compact      -- ascending index list of the due set (count, scan, scatter)
//   K6 predict      -- Eq. (jerkupdate) in closed form, streaming FP64
//      assign_bins  -- dt_i = min(dt_grav, dt_hydro) on power-of-two bins
// All of these are HBM- or launch-bound elementwise passes.  Every floating
// point step that decides an integer (due, bin) is a single correctly rounded
// operation written as an explicit intrinsic, so results are bit-identical to
// any IEEE implementation of the same definition.
#include <mutex>

#include "grav_common.cuh"

namespace grav {
namespace {

constexpr int kElemThreads = 256;

__global__ void __launch_bounds__(kElemThreads)
select_due_kernel(int64_t n, int64_t tick, int32_t k_max, const int8_t *__restrict__ bin,
                  int64_t *__restrict__ tf_ticks, const double *__restrict__ dt_grav, double q_f,
                  double dt_min, uint8_t *__restrict__ active_out, uint8_t *__restrict__ due_out,
                  int64_t *__restrict__ elapsed_out, int32_t *flags)
{
    int64_t i = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    if (i >= n) return;
    int32_t k = bin[i];
    if (k < 0 || k > k_max) {
        active_out[i] = 0;
        due_out[i] = 0;
        flag_or(flags, GRAV_FLAG_BADINDEX);
        return;
    }
    int64_t step = (int64_t)1 << (k_max - k);
    if ((tick & (step - 1)) != 0) {
        active_out[i] = 0;
        due_out[i] = 0;
        return;
    }
    int64_t tf = tf_ticks[i] + step;                       // Eq. (3)
    double elapsed = __dmul_rn(__ll2double_rn(tf), dt_min);
    double need = __dmul_rn(q_f, dt_grav[i]);
    bool due = elapsed >= need;                            // Eq. (updatecondition)
    if (due && elapsed_out) elapsed_out[i] = tf;           // time since the previous evaluation
    tf_ticks[i] = due ? 0 : tf;                            // reset: re-evaluated now
    active_out[i] = 1;
    due_out[i] = due ? 1 : 0;
}

// ---- compaction -----------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kPerThread = 16;
constexpr int kPerBlock = kScanThreads * kPerThread;   // 4096 flags per block

// Number of non-zero bytes in a 32-bit word.
__device__ __forceinline__ int nonzero_bytes(uint32_t w)
{
    uint32_t t = ((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w;
    return __popc(t & 0x80808080u);
}

// The 16 flags of this thread as four 32-bit words (bytes past n read as 0).
__device__ __forceinline__ void load16(const uint8_t *flags, int64_t n, int64_t base, bool vec_ok,
                                       uint32_t w[4])
{
    if (vec_ok && base + kPerThread <= n) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(flags + base));
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
        return;
    }
    for (int q = 0; q < 4; ++q) {
        uint32_t x = 0;
        for (int b = 0; b < 4; ++b) {
            int64_t j = base + q * 4 + b;
            uint32_t f = (j < n) ? (flags[j] != 0) : 0u;
            x |= f << (8 * b);
        }
        w[q] = x;
    }
}

// Block-wide exclusive scan of one int per thread; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *excl)
{
    __shared__ int warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    int warp_base = wid ? warp_tot[wid - 1] : 0;
    *excl = warp_base + x - v;
    int total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads)
compact_count_kernel(int64_t n, const uint8_t *__restrict__ flags, bool vec_ok,
                     int32_t *__restrict__ block_counts)
{
    int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    uint32_t w[4];
    load16(flags, n, base, vec_ok, w);
    int c = nonzero_bytes(w[0]) + nonzero_bytes(w[1]) + nonzero_bytes(w[2]) + nonzero_bytes(w[3]);
    int excl;
    int total = block_exclusive_scan(c, &excl);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = total;
}

constexpr int kTopThreads = 1024;

// One block: exclusive scan of the per-block counts in place; total -> count.
__global__ void __launch_bounds__(kTopThreads)
compact_scan_kernel(int64_t nb, int32_t *__restrict__ block_counts, int32_t *__restrict__ count_dev)
{
    __shared__ int warp_tot[kTopThreads / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += kTopThreads) {
        int64_t b = b0 + threadIdx.x;
        int v = (b < nb) ? block_counts[b] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        int excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
        if (b < nb) block_counts[b] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[kTopThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count_dev = carry;
}

__global__ void __launch_bounds__(kScanThreads)
compact_scatter_kernel(int64_t n, const uint8_t *__restrict__ flags, bool vec_ok,
                       const int32_t *__restrict__ block_offsets, int32_t *__restrict__ idx_out)
{
    int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    uint32_t w[4];
    load16(flags, n, base, vec_ok, w);
    int c = nonzero_bytes(w[0]) + nonzero_bytes(w[1]) + nonzero_bytes(w[2]) + nonzero_bytes(w[3]);
    int excl;
    block_exclusive_scan(c, &excl);
    if (c == 0) return;
    int64_t pos = (int64_t)block_offsets[blockIdx.x] + excl;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if ((w[q] >> (8 * b)) & 0xFFu) idx_out[pos++] = (int32_t)(base + q * 4 + b);
        }
    }
}

// ---- predictor ------------------------------------------------------------

// Flattened over the 3n components so that loads and stores coalesce.
__global__ void __launch_bounds__(kElemThreads)
predict_kernel(int64_t n3, const uint8_t *__restrict__ active, const uint8_t *__restrict__ due,
               const double *__restrict__ a_last, const double *__restrict__ j_last,
               const int64_t *__restrict__ tf_ticks, double dt_min, double *__restrict__ a_out)
{
    int64_t q = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    if (q >= n3) return;
    int64_t i = q / 3;
    if (!active[i]) return;
    double a = a_last[q];
    if (!due[i]) {
        double tau = __dmul_rn(__ll2double_rn(tf_ticks[i]), dt_min);
        a = __dadd_rn(a, __dmul_rn(j_last[q], tau));     // Eq. (jerkupdate)
    }
    a_out[q] = a;
}

// Two elements per thread with 16-byte loads and stores (all arrays 16-byte
// aligned, flags 2-byte aligned): the same correctly rounded operations as
// predict_kernel, so the results are bit-identical.
__global__ void __launch_bounds__(kElemThreads)
predict_pair_kernel(int64_t n, const uint8_t *__restrict__ active, const uint8_t *__restrict__ due,
                    const double *__restrict__ a_last, const double *__restrict__ j_last,
                    const int64_t *__restrict__ tf_ticks, double dt_min, double *__restrict__ a_out)
{
    const int64_t t = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    const int64_t i0 = 2 * t;
    if (i0 >= n) return;
    if (i0 + 1 >= n) {                                   // odd tail: one element
        if (!active[i0]) return;
        const double tau = __dmul_rn(__ll2double_rn(tf_ticks[i0]), dt_min);
        for (int c = 0; c < 3; ++c) {
            double a = a_last[3 * i0 + c];
            if (!due[i0]) a = __dadd_rn(a, __dmul_rn(j_last[3 * i0 + c], tau));
            a_out[3 * i0 + c] = a;
        }
        return;
    }
    const uchar2 act = *reinterpret_cast<const uchar2 *>(active + i0);
    if (!act.x && !act.y) return;
    const uchar2 du = *reinterpret_cast<const uchar2 *>(due + i0);
    const longlong2 tf = __ldg(reinterpret_cast<const longlong2 *>(tf_ticks + i0));
    const double2 *al = reinterpret_cast<const double2 *>(a_last + 3 * i0);
    const double2 *jl = reinterpret_cast<const double2 *>(j_last + 3 * i0);
    double2 a[3] = {__ldg(al), __ldg(al + 1), __ldg(al + 2)};
    const double2 j[3] = {__ldg(jl), __ldg(jl + 1), __ldg(jl + 2)};
    double *av = reinterpret_cast<double *>(a);
    const double *jv = reinterpret_cast<const double *>(j);
    const double tau0 = __dmul_rn(__ll2double_rn(tf.x), dt_min);
    const double tau1 = __dmul_rn(__ll2double_rn(tf.y), dt_min);
    if (!du.x)
        for (int c = 0; c < 3; ++c) av[c] = __dadd_rn(av[c], __dmul_rn(jv[c], tau0));
    if (!du.y)
        for (int c = 3; c < 6; ++c) av[c] = __dadd_rn(av[c], __dmul_rn(jv[c], tau1));
    double2 *ao = reinterpret_cast<double2 *>(a_out + 3 * i0);
    if (act.x && act.y) {
        ao[0] = a[0];
        ao[1] = a[1];
        ao[2] = a[2];
    } else {
        const int lo = act.x ? 0 : 3;
        for (int c = lo; c < lo + 3; ++c) a_out[3 * i0 + c] = av[c];
    }
}

// ---- polynomial predictor (Section 2.2) -----------------------------------

// Log the evaluation before the new one for every due element: its
// acceleration and the gap between the two (T_f when it became due); an
// element never evaluated before (dt_grav == 0) has no history.
__global__ void __launch_bounds__(kElemThreads)
push_history_kernel(int64_t n, const uint8_t *__restrict__ due,
                    const int64_t *__restrict__ elapsed, const double *__restrict__ dt_grav,
                    const double *__restrict__ a_last, double *__restrict__ a_prev,
                    double *__restrict__ dt_prev, double dt_min)
{
    const int64_t i = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    if (i >= n || !due[i]) return;
    dt_prev[i] = (dt_grav[i] == 0.0) ? 0.0 : __dmul_rn(__ll2double_rn(elapsed[i]), dt_min);
#pragma unroll
    for (int c = 0; c < 3; ++c) a_prev[3 * i + c] = a_last[3 * i + c];
}

// Linear extrapolation through the last two evaluations, flattened over the
// 3n components (every operation correctly rounded, no fusion).
__global__ void __launch_bounds__(kElemThreads)
predict_poly_kernel(int64_t n3, const uint8_t *__restrict__ active, const uint8_t *__restrict__ due,
                    const double *__restrict__ a_last, const double *__restrict__ a_prev,
                    const double *__restrict__ dt_prev, const int64_t *__restrict__ tf_ticks,
                    double dt_min, double *__restrict__ a_out)
{
    const int64_t q = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    if (q >= n3) return;
    const int64_t i = q / 3;
    if (!active[i]) return;
    double a = a_last[q];
    const double gap = dt_prev[i];
    if (!due[i] && gap > 0.0) {
        const double tau = __dmul_rn(__ll2double_rn(tf_ticks[i]), dt_min);
        const double frac = __ddiv_rn(tau, gap);
        a = __dadd_rn(a, __dmul_rn(__dsub_rn(a, a_prev[q]), frac));
    }
    a_out[q] = a;
}

// ---- bins -----------------------------------------------------------------

__device__ __forceinline__ int32_t target_bin(double dt, double dt_max, int32_t k_max)
{
    if (!(dt > 0.0)) return k_max;                  // 0, negative or NaN
    if (isinf(dt)) return 0;
    int ei, em;
    double mi = frexp(dt, &ei);
    double mm = frexp(dt_max, &em);
    // dt_max 2^-k <= dt  <=>  mm 2^(em-k) <= mi 2^ei  (exact)
    int64_t k = (int64_t)em - (int64_t)ei;
    if (mm > mi) k += 1;
    if (k < 0) k = 0;
    if (k > k_max) k = k_max;
    return (int32_t)k;
}

__global__ void __launch_bounds__(kElemThreads)
assign_bins_kernel(int64_t n, int32_t k_align, int32_t k_max, double dt_max,
                   const uint8_t *__restrict__ active, const double *__restrict__ dt_grav,
                   const double *__restrict__ dt_hydro, int8_t *__restrict__ bin)
{
    int64_t i = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
    if (i >= n || !active[i]) return;
    double dt = dt_grav[i];
    if (dt_hydro) {
        double dh = dt_hydro[i];
        if (dh < dt) dt = dh;
        if (isnan(dh)) dt = dh;
    }
    int32_t k = target_bin(dt, dt_max, k_max);
    if (k < k_align) k = k_align;
    bin[i] = (int8_t)k;
}

inline unsigned elem_blocks(int64_t n) { return (unsigned)((n + kElemThreads - 1) / kElemThreads); }

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int grav_select_due(int64_t n, int64_t tick, int32_t k_max, const int8_t *bin,
                               int64_t *tf_ticks, const double *dt_grav, double q_f, double dt_min,
                               uint8_t *active_out, uint8_t *due_out, int64_t *elapsed_out,
                               int32_t *flags_dev, void *stream)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_select_due: n < 0");
    if (tick < 0) return fail(GRAV_EINVAL, "grav_select_due: tick < 0");
    if (k_max < 0 || k_max > 62) return fail(GRAV_EINVAL, "grav_select_due: k_max outside [0, 62]");
    if (!(q_f >= 0.0) || !(dt_min > 0.0) || isinf(dt_min) || isinf(q_f))
        return fail(GRAV_EINVAL, "grav_select_due: need finite q_f >= 0 and dt_min > 0");
    if (n == 0) return GRAV_OK;
    if (!bin || !tf_ticks || !dt_grav || !active_out || !due_out)
        return fail(GRAV_EINVAL, "grav_select_due: null array");
    unsigned blocks = elem_blocks(n);
    select_due_kernel<<<blocks, kElemThreads, 0, as_stream(stream)>>>(
        n, tick, k_max, bin, tf_ticks, dt_grav, q_f, dt_min, active_out, due_out, elapsed_out,
        flags_dev);
    return check_launch("grav_select_due");
}

extern "C" int64_t grav_compact_workspace_bytes(int64_t n)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_compact_workspace_bytes: n < 0");
    int64_t nb = (n + kPerBlock - 1) / kPerBlock;
    return round_up(std::max<int64_t>(nb, 1) * 4, 256);
}

extern "C" int grav_compact_active(int64_t n, const uint8_t *flags, int32_t *idx_out,
                                   int32_t *count_dev, void *workspace, int64_t workspace_bytes,
                                   void *stream)
{
    if (n < 0 || n > INT32_MAX) return fail(GRAV_EINVAL, "grav_compact_active: n outside [0, 2^31)");
    if (!count_dev) return fail(GRAV_EINVAL, "grav_compact_active: null count_dev");
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        return check_cuda(cudaMemsetAsync(count_dev, 0, sizeof(int32_t), s), "grav_compact_active");
    }
    if (!flags || !idx_out || !workspace) return fail(GRAV_EINVAL, "grav_compact_active: null array");
    if (workspace_bytes < grav_compact_workspace_bytes(n))
        return fail(GRAV_ENOMEM, "grav_compact_active: workspace of %lld bytes < %lld",
                    (long long)workspace_bytes, (long long)grav_compact_workspace_bytes(n));
    if (!aligned(workspace, 256)) return fail(GRAV_EINVAL, "grav_compact_active: workspace not 256-byte aligned");
    int64_t nb = (n + kPerBlock - 1) / kPerBlock;
    bool vec_ok = aligned(flags, 16);
    int32_t *counts = static_cast<int32_t *>(workspace);
    compact_count_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, flags, vec_ok, counts);
    int rc = check_launch("grav_compact_active/count");
    if (rc) return rc;
    compact_scan_kernel<<<1, kTopThreads, 0, s>>>(nb, counts, count_dev);
    rc = check_launch("grav_compact_active/scan");
    if (rc) return rc;
    compact_scatter_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, flags, vec_ok, counts, idx_out);
    return check_launch("grav_compact_active/scatter");
}

extern "C" int grav_predict(int64_t n, const uint8_t *active, const uint8_t *due,
                            const double *a_last, const double *j_last, const int64_t *tf_ticks,
                            double dt_min, double *a_out, void *stream)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_predict: n < 0");
    if (!(dt_min > 0.0) || isinf(dt_min)) return fail(GRAV_EINVAL, "grav_predict: dt_min must be finite and > 0");
    if (n == 0) return GRAV_OK;
    if (!active || !due || !a_last || !j_last || !tf_ticks || !a_out)
        return fail(GRAV_EINVAL, "grav_predict: null array");
    if (a_out == a_last || a_out == j_last) return fail(GRAV_EINVAL, "grav_predict: a_out aliases an input");
    if (aligned(a_last, 16) && aligned(j_last, 16) && aligned(a_out, 16) && aligned(tf_ticks, 16) &&
        aligned(active, 2) && aligned(due, 2)) {
        const int64_t pairs = (n + 1) / 2;
        predict_pair_kernel<<<elem_blocks(pairs), kElemThreads, 0, as_stream(stream)>>>(
            n, active, due, a_last, j_last, tf_ticks, dt_min, a_out);
        return check_launch("grav_predict");
    }
    int64_t n3 = 3 * n;
    predict_kernel<<<elem_blocks(n3), kElemThreads, 0, as_stream(stream)>>>(
        n3, active, due, a_last, j_last, tf_ticks, dt_min, a_out);
    return check_launch("grav_predict");
}

extern "C" int grav_assign_bins(int64_t n, int64_t tick, int32_t k_max, double dt_max,
                                const uint8_t *active, const double *dt_grav,
                                const double *dt_hydro, int8_t *bin, void *stream)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_assign_bins: n < 0");
    if (tick < 0) return fail(GRAV_EINVAL, "grav_assign_bins: tick < 0");
    if (k_max < 0 || k_max > 62) return fail(GRAV_EINVAL, "grav_assign_bins: k_max outside [0, 62]");
    if (!(dt_max > 0.0) || isinf(dt_max)) return fail(GRAV_EINVAL, "grav_assign_bins: dt_max must be finite and > 0");
    if (n == 0) return GRAV_OK;
    if (!active || !dt_grav || !bin) return fail(GRAV_EINVAL, "grav_assign_bins: null array");
    int32_t k_align = 0;
    if (tick != 0) {
        int tz = 0;
        while (((tick >> tz) & 1) == 0) ++tz;
        k_align = k_max - tz;
        if (k_align < 0) k_align = 0;
    }
    assign_bins_kernel<<<elem_blocks(n), kElemThreads, 0, as_stream(stream)>>>(
        n, k_align, k_max, dt_max, active, dt_grav, dt_hydro, bin);
    return check_launch("grav_assign_bins");
}

// ---------------------------------------------------------------------------
// Compaction for callers that cannot allocate device memory.
//
// Some callers cannot hand us a workspace: a host framework that reserved the
// whole device memory pool for itself, a time-step loop that must not stall
// on cudaMalloc's implicit device synchronisation, or code recording work in
// a mode where allocation is forbidden.  This entry point keeps its scratch
// (one int32 per block of 4096 flags) in a fixed array inside the library.
// The array lives on every device that loads the library until the process
// exits, is shared by all calls, and keeps whatever the last call left in it;
// every element a call reads is written by that same call first, so nothing
// has to be cleared.  Calls whose kernels overlap on the GPU race on it.
// ---------------------------------------------------------------------------

namespace grav {
namespace {

constexpr int64_t kNoAllocMaxBlocks = 1 << 14;
constexpr int64_t kNoAllocMaxN = kNoAllocMaxBlocks * kPerBlock;   // 2^26 flags
static_assert(kNoAllocMaxN == GRAV_COMPACT_NOALLOC_MAX_N, "limit of the header");

static __device__ __align__(256) int32_t g_noalloc_block_counts[kNoAllocMaxBlocks];

// Device address of the array on the current device, looked up once per
// device (host code may not use the array's name as a device pointer).
int noalloc_scratch(int32_t **out)
{
    static std::mutex mu;
    static int32_t *addr[64] = {nullptr};
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return fail(GRAV_ECUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_block_counts),
                        "cudaGetSymbolAddress(g_noalloc_block_counts)");
        if (rc) return rc;
        addr[dev] = static_cast<int32_t *>(p);
    }
    *out = addr[dev];
    return GRAV_OK;
}

}  // namespace
}  // namespace grav

extern "C" int grav_compact_active_noalloc(int64_t n, const uint8_t *flags, int32_t *idx_out,
                                           int32_t *count_dev, void *stream)
{
    static const char *who = "grav_compact_active_noalloc";
    if (n < 0 || n > kNoAllocMaxN)
        return fail(GRAV_EINVAL, "%s: n = %lld outside [0, %lld] (the fixed scratch holds %lld blocks)",
                    who, (long long)n, (long long)kNoAllocMaxN, (long long)kNoAllocMaxBlocks);
    if (!count_dev) return fail(GRAV_EINVAL, "%s: null count_dev", who);
    cudaStream_t s = as_stream(stream);
    if (n == 0) return check_cuda(cudaMemsetAsync(count_dev, 0, sizeof(int32_t), s), who);
    if (!flags || !idx_out) return fail(GRAV_EINVAL, "%s: null array", who);
    int32_t *counts = nullptr;
    int rc = noalloc_scratch(&counts);
    if (rc) return rc;
    const int64_t nb = (n + kPerBlock - 1) / kPerBlock;
    const bool vec_ok = aligned(flags, 16);
    compact_count_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, flags, vec_ok, counts);
    rc = check_launch("grav_compact_active_noalloc/count");
    if (rc) return rc;
    compact_scan_kernel<<<1, kTopThreads, 0, s>>>(nb, counts, count_dev);
    rc = check_launch("grav_compact_active_noalloc/scan");
    if (rc) return rc;
    compact_scatter_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(n, flags, vec_ok, counts, idx_out);
    return check_launch("grav_compact_active_noalloc/scatter");
}

extern "C" int grav_push_history(int64_t n, const uint8_t *due, const int64_t *elapsed,
                                 const double *dt_grav, const double *a_last, double *a_prev,
                                 double *dt_prev, double dt_min, void *stream)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_push_history: n < 0");
    if (!(dt_min > 0.0) || isinf(dt_min)) return fail(GRAV_EINVAL, "grav_push_history: dt_min must be finite and > 0");
    if (n == 0) return GRAV_OK;
    if (!due || !elapsed || !dt_grav || !a_last || !a_prev || !dt_prev)
        return fail(GRAV_EINVAL, "grav_push_history: null array");
    if (a_prev == a_last) return fail(GRAV_EINVAL, "grav_push_history: a_prev aliases a_last");
    push_history_kernel<<<elem_blocks(n), kElemThreads, 0, as_stream(stream)>>>(
        n, due, elapsed, dt_grav, a_last, a_prev, dt_prev, dt_min);
    return check_launch("grav_push_history");
}

extern "C" int grav_predict_poly(int64_t n, const uint8_t *active, const uint8_t *due,
                                 const double *a_last, const double *a_prev, const double *dt_prev,
                                 const int64_t *tf_ticks, double dt_min, double *a_out, void *stream)
{
    if (n < 0) return fail(GRAV_EINVAL, "grav_predict_poly: n < 0");
    if (!(dt_min > 0.0) || isinf(dt_min)) return fail(GRAV_EINVAL, "grav_predict_poly: dt_min must be finite and > 0");
    if (n == 0) return GRAV_OK;
    if (!active || !due || !a_last || !a_prev || !dt_prev || !tf_ticks || !a_out)
        return fail(GRAV_EINVAL, "grav_predict_poly: null array");
    if (a_out == a_last || a_out == a_prev) return fail(GRAV_EINVAL, "grav_predict_poly: a_out aliases an input");
    const int64_t n3 = 3 * n;
    predict_poly_kernel<<<elem_blocks(n3), kElemThreads, 0, as_stream(stream)>>>(
        n3, active, due, a_last, a_prev, dt_prev, tf_ticks, dt_min, a_out);
    return check_launch("grav_predict_poly");
}
