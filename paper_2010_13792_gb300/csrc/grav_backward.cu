// K7: adjoint of the force evaluation (reverse mode), all n elements targets.
//
// For a loss L(a, W) with a_bar = dL/da and w_bar = dL/dW (W = 1/2 sum m Phi):
//   pos_bar_k  = T_k a_bar_k + G m_k sum_{i!=k} [ f a_bar_i + g d (d . a_bar_i) ]
//                - w_bar m_k a_k
//   mass_bar_k = -G sum_{i!=k} f (d . a_bar_i) + w_bar Phi_k,      d = x_i - x_k,
// obtained by differentiating a_i = G sum_j m_j f(r) d (Eq. 4's acceleration)
// with respect to x_k and m_k; T_k = d a_k / d x_k is the forward tidal tensor.
// The paper has no adjoint.  The kernels are the forward direct sum with the
// source attribute a_bar_i in place of (v_i, m_i) (FP64: backward_kernel;
// mixed: backward_pair_kernel on the forward's paired FP32x2 tile layout and
// per-warp TMA ring): per pair they accumulate
//   X1 += f a_bar_i,   X2 += g' (d . a_bar_i) d,   MB += f (d . a_bar_i)
// with g' = -g/3, recomputing every pair term instead of storing any, and the
// epilogue forms pos_bar = T a_bar + G m (X1 - 3 X2) - w_bar m a.
#include <cmath>
#include <mutex>

#include "grav_eval.cuh"

namespace grav {
namespace {

constexpr int kNB = 7;
enum { X10 = 0, X20 = 3, MBS = 6 };

struct BwdArgs {
    int64_t n;
    const TileGeom *geo;
    const void *src;
    int32_t n_tiles;
    int32_t max_split;
    int32_t grid;
    int32_t pad0;
    double *part;
    int64_t part_cap_rows;
    const double *pos, *mass, *a_bar;
    double w_bar;
    const double *acc, *tidal, *pot;
    double G, h;
    float h2f_up, hinvf;
    double *pos_bar, *mass_bar;
    int32_t *flags;
};

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T sqrt_t(T x) { return sqrt(x); }

template <typename T>
struct Src;
template <>
struct Src<double> { using type = D4; };

template <typename T, int KT, int S, bool NEAR>
__device__ __forceinline__ void bwd_loop(const typename Src<T>::type *__restrict__ sp,
                                         const typename Src<T>::type *__restrict__ sa,
                                         const T tx[KT][3], const int64_t tk[KT], int64_t jbase,
                                         T h2, T hinv, T acc[KT][kNB])
{
    const T hinv3 = hinv * hinv * hinv;
    const T hinv5 = hinv3 * hinv * hinv;
#pragma unroll 4
    for (int j = 0; j < S; ++j) {
        const auto p = sp[j];
        const auto ab = sa[j];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            T dx = p.x - tx[q][0], dy = p.y - tx[q][1], dz = p.z - tx[q][2];
            T r2 = dx * dx + dy * dy + dz * dz;
            T ri = rsqrt_t<T>(r2);
            T ri2 = ri * ri;
            T f = ri * ri2;
            T gp = f * ri2;
            if (NEAR && r2 < h2) {
                T F, Gp, P;
                spline_kernel<T>(sqrt_t<T>(r2) * hinv, F, Gp, P);
                f = F * hinv3;
                gp = Gp * hinv5;
                if (jbase + j == tk[q]) {
                    f = T(0);
                    gp = T(0);
                }
            }
            T da = dx * ab.x + dy * ab.y + dz * ab.z;
            acc[q][X10 + 0] += f * ab.x;
            acc[q][X10 + 1] += f * ab.y;
            acc[q][X10 + 2] += f * ab.z;
            T gd = gp * da;
            acc[q][X20 + 0] += gd * dx;
            acc[q][X20 + 1] += gd * dy;
            acc[q][X20 + 2] += gd * dz;
            acc[q][MBS] += f * da;
        }
    }
}

__device__ __forceinline__ void bwd_write(const BwdArgs &a, int64_t k, const double s[kNB])
{
    const double m = a.mass[k];
    double px[3] = {0.0, 0.0, 0.0};
    double pm = 0.0;
    if (a.a_bar) {
        const double *t6 = a.tidal + 6 * k;
        const double *ak = a.a_bar + 3 * k;
        px[0] = t6[0] * ak[0] + t6[3] * ak[1] + t6[4] * ak[2];
        px[1] = t6[3] * ak[0] + t6[1] * ak[1] + t6[5] * ak[2];
        px[2] = t6[4] * ak[0] + t6[5] * ak[1] + t6[2] * ak[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) px[c] += a.G * m * (s[X10 + c] - 3.0 * s[X20 + c]);
        pm = -a.G * s[MBS];
    }
    if (a.w_bar != 0.0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) px[c] -= a.w_bar * m * a.acc[3 * k + c];
        pm += a.w_bar * a.pot[k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a.pos_bar[3 * k + c] = px[c];
    a.mass_bar[k] = pm;
}

// The direct-sum adjoint on scalar (x, a_bar) tiles; instantiated for FP64
// (the mixed adjoint is backward_pair_kernel below).
template <typename T, int NT, int KT, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB)
backward_kernel(const BwdArgs a)
{
    using E = typename Src<T>::type;
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int BT = NT * KT;
    constexpr int NSTAGE = 2;
    constexpr uint32_t kTileBytes = S * 2 * sizeof(E);
    __shared__ __align__(128) E stage[NSTAGE][2 * S];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    __shared__ float blo[3], bhi[3];
    __shared__ int abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t parity = 0, pending = 0;

    const int64_t n_tb = (a.n + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    const int64_t items = n_tb * split;
    const int64_t rows = n_tb * BT;
    const E *src = static_cast<const E *>(a.src);
    const T h2 = MIXED ? (T)a.h2f_up : (T)(a.h * a.h);
    const T hinv = MIXED ? (T)a.hinvf : (T)(1.0 / a.h);

    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        const int t_begin = (int)((int64_t)sp * a.n_tiles / split);
        const int t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);

        double xk[KT][3];
        int64_t tk[KT];
        float lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = __int_as_float(0x7f800000);
            hi[c] = -__int_as_float(0x7f800000);
        }
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const int64_t k = tb * BT + (int64_t)q * NT + threadIdx.x;
            tk[q] = k < a.n ? k : -1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xk[q][c] = tk[q] >= 0 ? a.pos[3 * k + c] : 0.0;
                if (tk[q] >= 0) {
                    lo[c] = fminf(lo[c], __double2float_rd(xk[q][c]));
                    hi[c] = fmaxf(hi[c], __double2float_ru(xk[q][c]));
                }
            }
        }
        block_bbox<NT>(lo, hi, blo, bhi);
        // each warp tests tiles against its own targets' box (lo/hi now hold
        // it): the near and far loops synchronise nothing
        const float blo_r[3] = {lo[0], lo[1], lo[2]};
        const float bhi_r[3] = {hi[0], hi[1], hi[2]};

        T shi[KT][kNB], slo[KT][kNB];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNB; ++c) {
                shi[q][c] = T(0);
                slo[q][c] = T(0);
            }
        if (threadIdx.x == 0) {
            for (int s = 0; s < NSTAGE; ++s) {
                int t = t_begin + s;
                if (t < t_end) {
                    tma_load_1d(stage[s], src + (int64_t)t * 2 * S, kTileBytes, &bar[s]);
                    pending |= 1u << s;
                }
            }
        }
        for (int t = t_begin; t < t_end; ++t) {
            const int s = (t - t_begin) % NSTAGE;
            const TileGeom g = a.geo[t];
            const bool near = tile_is_near(blo_r, bhi_r, g, a.h2f_up);
            T tx[KT][3];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (MIXED)
                        tx[q][c] = (T)__double2float_rn(__dsub_rn(xk[q][c], g.c[c]));
                    else
                        tx[q][c] = (T)xk[q][c];
                }
            const bool got = mbar_wait_bounded(&bar[s], (parity >> s) & 1u, a.flags);
            if (got)
                parity ^= 1u << s;
            else
                atomicExch(&abort_flag, 1);
            T acc[KT][kNB];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNB; ++c) acc[q][c] = T(0);
            if (!near)
                bwd_loop<T, KT, S, false>(stage[s], stage[s] + S, tx, tk, g.first, h2, hinv, acc);
            else
                bwd_loop<T, KT, S, true>(stage[s], stage[s] + S, tx, tk, g.first, h2, hinv, acc);
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNB; ++c) two_sum_acc(shi[q][c], slo[q][c], acc[q][c]);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (got) pending &= ~(1u << s);
                if (t + NSTAGE < t_end && !abort_flag) {
                    tma_load_1d(stage[s], src + (int64_t)(t + NSTAGE) * 2 * S, kTileBytes, &bar[s]);
                    pending |= 1u << s;
                }
            }
            if (abort_flag) break;
        }
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            double sum[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c) sum[c] = (double)shi[q][c] + (double)slo[q][c];
            const int64_t slot = tb * BT + (int64_t)q * NT + threadIdx.x;
            if (split == 1) {
                if (tk[q] >= 0) bwd_write(a, tk[q], sum);
            } else {
#pragma unroll
                for (int c = 0; c < kNB; ++c) a.part[((int64_t)sp * kNB + c) * rows + slot] = sum[c];
            }
        }
        if (abort_flag) break;
        __syncthreads();
    }
    if (threadIdx.x == 0 && pending) {
        for (int s = 0; s < NSTAGE; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bar[s], (parity >> s) & 1u, a.flags);
    }
}

// Mixed adjoint on the paired source layout of the forward kernel (the
// packer's velocity slots carry a_bar_i, its mass slots are unused): two
// sources per packed FP32x2 instruction in the Newtonian loop, 20 such
// instructions per source pair (the scalar loop's 20 per source).
template <int KT, int S, int U>
__device__ __forceinline__ void bwd_far_pair(const float *__restrict__ tile, const float tx[KT][3],
                                             float2 acc[KT][kNB])
{
    const float4 *P0 = reinterpret_cast<const float4 *>(tile);
    const float4 *P1 = P0 + S / 2;
    const float4 *V0 = P1 + S / 2;
    const float2 *V1 = reinterpret_cast<const float2 *>(V0 + S / 2);
    float2 ntx[KT], nty[KT], ntz[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        ntx[q] = make_float2(-tx[q][0], -tx[q][0]);
        nty[q] = make_float2(-tx[q][1], -tx[q][1]);
        ntz[q] = make_float2(-tx[q][2], -tx[q][2]);
    }
#pragma unroll U
    for (int k = 0; k < S / 2; ++k) {
        const float4 p0 = P0[k], p1 = P1[k], v0 = V0[k];
        const float2 bz = V1[k];
        const float2 bx = make_float2(v0.x, v0.y), by = make_float2(v0.z, v0.w);
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float2 dx = __fadd2_rn(make_float2(p0.x, p0.y), ntx[q]);
            const float2 dy = __fadd2_rn(make_float2(p0.z, p0.w), nty[q]);
            const float2 dz = __fadd2_rn(make_float2(p1.x, p1.y), ntz[q]);
            float2 r2 = __fmul2_rn(dz, dz);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dx, dx, r2);
            const float2 ri = make_float2(rsqrt_sfu(r2.x), rsqrt_sfu(r2.y));
            const float2 ri2 = __fmul2_rn(ri, ri);
            const float2 f = __fmul2_rn(ri, ri2);
            const float2 gp = __fmul2_rn(f, ri2);
            float2 da = __fmul2_rn(dz, bz);
            da = __ffma2_rn(dy, by, da);
            da = __ffma2_rn(dx, bx, da);
            acc[q][X10 + 0] = __ffma2_rn(f, bx, acc[q][X10 + 0]);
            acc[q][X10 + 1] = __ffma2_rn(f, by, acc[q][X10 + 1]);
            acc[q][X10 + 2] = __ffma2_rn(f, bz, acc[q][X10 + 2]);
            const float2 gd = __fmul2_rn(gp, da);
            acc[q][X20 + 0] = __ffma2_rn(gd, dx, acc[q][X20 + 0]);
            acc[q][X20 + 1] = __ffma2_rn(gd, dy, acc[q][X20 + 1]);
            acc[q][X20 + 2] = __ffma2_rn(gd, dz, acc[q][X20 + 2]);
            acc[q][MBS] = __ffma2_rn(f, da, acc[q][MBS]);
        }
    }
}

// Softened loop on the paired layout, one source at a time (lane x of the
// accumulators), the self pair excluded by index.
template <int KT, int S>
__device__ __forceinline__ void bwd_near_pair(const float *__restrict__ tile, const float tx[KT][3],
                                              const int64_t tk[KT], int64_t jbase, float h2, float hinv,
                                              float2 acc[KT][kNB])
{
    const float hinv3 = hinv * hinv * hinv;
    const float hinv5 = hinv3 * hinv * hinv;
#pragma unroll 2
    for (int j = 0; j < S; ++j) {
        const int k = j >> 1, h = j & 1;
        const float x = tile[4 * k + h], y = tile[4 * k + 2 + h];
        const float z = tile[2 * S + 4 * k + h];
        const float bx = tile[4 * S + 4 * k + h], by = tile[4 * S + 4 * k + 2 + h];
        const float bz = tile[6 * S + 2 * k + h];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float dx = x - tx[q][0], dy = y - tx[q][1], dz = z - tx[q][2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_sfu(r2);
            const float ri2 = ri * ri;
            float f = ri * ri2;
            float gp = f * ri2;
            if (r2 < h2) {
                float F, Gp, P;
                spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
                f = F * hinv3;
                gp = Gp * hinv5;
                if (jbase + j == tk[q]) {
                    f = 0.0f;
                    gp = 0.0f;
                }
            }
            const float da = fmaf(dx, bx, fmaf(dy, by, dz * bz));
            acc[q][X10 + 0].x = fmaf(f, bx, acc[q][X10 + 0].x);
            acc[q][X10 + 1].x = fmaf(f, by, acc[q][X10 + 1].x);
            acc[q][X10 + 2].x = fmaf(f, bz, acc[q][X10 + 2].x);
            const float gd = gp * da;
            acc[q][X20 + 0].x = fmaf(gd, dx, acc[q][X20 + 0].x);
            acc[q][X20 + 1].x = fmaf(gd, dy, acc[q][X20 + 1].x);
            acc[q][X20 + 2].x = fmaf(gd, dz, acc[q][X20 + 2].x);
            acc[q][MBS].x = fmaf(f, da, acc[q][MBS].x);
        }
    }
}

// Shared memory of the mixed adjoint: a three-stage ring of paired tiles.
template <int S>
struct BwdPairSmem {
    static constexpr int kStages = 3;
    float4 stage[kStages][7 * S / 4];
    uint64_t bar[kStages];
    int done[kStages];           // warps finished with the tile in each stage
    unsigned issued[kStages];    // copies issued into each stage
    float blo[3], bhi[3];
    int abort_flag;
};

// The mixed adjoint kernel: the structure of the forward mixed kernel (work
// items of target blocks x source chunks, a three-stage TMA ring in which
// each warp releases a stage on its own and the last warp to release it
// issues the refill, each warp's near/far test against its own targets'
// box), with the adjoint's pair terms.  Per-tile FP32 sums are carried across
// tiles as compensated FP32 pairs (TwoSum); the result is FP64.
template <int NT, int KT, int S, int MINB, int U>
__global__ void __launch_bounds__(NT, MINB) backward_pair_kernel(const BwdArgs a)
{
    using Sm = BwdPairSmem<S>;
    constexpr int NSTAGE = Sm::kStages;
    constexpr int BT = NT * KT;
    constexpr uint32_t kTileBytes = S * 28;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&sm.bar[s], 1);
            sm.done[s] = 0;
            sm.issued[s] = 0;
        }
        sm.abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t parity = 0;

    const int64_t n_tb = (a.n + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    const int64_t items = n_tb * split;
    const int64_t rows = n_tb * BT;
    const float4 *src = static_cast<const float4 *>(a.src);
    const float h2 = a.h2f_up, hinv = a.hinvf;

    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        const int t_begin = (int)((int64_t)sp * a.n_tiles / split);
        const int t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);

        double xk[KT][3];
        int64_t tk[KT];
        float lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = __int_as_float(0x7f800000);
            hi[c] = -__int_as_float(0x7f800000);
        }
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const int64_t k = tb * BT + (int64_t)q * NT + threadIdx.x;
            tk[q] = k < a.n ? k : -1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xk[q][c] = tk[q] >= 0 ? a.pos[3 * k + c] : 0.0;
                if (tk[q] >= 0) {
                    lo[c] = fminf(lo[c], __double2float_rd(xk[q][c]));
                    hi[c] = fmaxf(hi[c], __double2float_ru(xk[q][c]));
                }
            }
        }
        // lo/hi become the warp's box; tiles are tested against it
        block_bbox<NT>(lo, hi, sm.blo, sm.bhi);

        float shi[KT][kNB], slo[KT][kNB];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNB; ++c) {
                shi[q][c] = 0.0f;
                slo[q][c] = 0.0f;
            }
        if (threadIdx.x == 0) {
            for (int s = 0; s < NSTAGE; ++s) {
                const int t = t_begin + s;
                if (t < t_end) {
                    tma_load_1d(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes, &sm.bar[s]);
                    sm.issued[s] += 1u;
                }
            }
        }
        for (int t = t_begin; t < t_end; ++t) {
            const int s = (t - t_begin) % NSTAGE;
            const TileGeom g = a.geo[t];
            const bool near = tile_is_near(lo, hi, g, h2);
            float tx[KT][3];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) tx[q][c] = __double2float_rn(__dsub_rn(xk[q][c], g.c[c]));
            const bool got = mbar_wait_bounded(&sm.bar[s], (parity >> s) & 1u, a.flags);
            if (got)
                parity ^= 1u << s;
            else
                atomicExch(&sm.abort_flag, 1);
            float2 acc[KT][kNB];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNB; ++c) acc[q][c] = make_float2(0.0f, 0.0f);
            const float *tf = reinterpret_cast<const float *>(sm.stage[s]);
            if (!near)
                bwd_far_pair<KT, S, U>(tf, tx, acc);
            else
                bwd_near_pair<KT, S>(tf, tx, tk, g.first, h2, hinv, acc);
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNB; ++c) two_sum_acc(shi[q][c], slo[q][c], acc[q][c].x + acc[q][c].y);
            // this warp is done reading stage s; the last warp refills it
            __syncwarp();
            if ((threadIdx.x & 31) == 0) {
                __threadfence_block();
                const int prev = atomicAdd(&sm.done[s], 1);
                if (prev == NT / 32 - 1) {
                    sm.done[s] = 0;
                    __threadfence_block();
                    if (t + NSTAGE < t_end && !*(volatile int *)&sm.abort_flag) {
                        fence_proxy_async_smem();
                        tma_load_1d(sm.stage[s], src + (int64_t)(t + NSTAGE) * 2 * S, kTileBytes,
                                    &sm.bar[s]);
                        sm.issued[s] += 1u;
                    }
                }
            }
            __syncwarp();
            if (*(volatile int *)&sm.abort_flag) break;
        }
        __syncthreads();   // every warp is out of the tile loop: a uniform status
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            double sum[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c) sum[c] = (double)shi[q][c] + (double)slo[q][c];
            const int64_t slot = tb * BT + (int64_t)q * NT + threadIdx.x;
            if (split == 1) {
                if (tk[q] >= 0) bwd_write(a, tk[q], sum);
            } else {
#pragma unroll
                for (int c = 0; c < kNB; ++c) a.part[((int64_t)sp * kNB + c) * rows + slot] = sum[c];
            }
        }
        if (sm.abort_flag) break;
        __syncthreads();
    }
    // copies still in flight (only after a timed-out wait): a stage holds one
    // exactly when thread 0 has seen fewer completions there than were issued
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s)
            if ((sm.issued[s] & 1u) != ((parity >> s) & 1u))
                mbar_wait_bounded(&sm.bar[s], (parity >> s) & 1u, a.flags);
    }
}

__global__ void __launch_bounds__(256) backward_reduce_kernel(const BwdArgs a, int32_t BT)
{
    const int64_t n_tb = (a.n + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    if (split <= 1) return;
    const int64_t rows = n_tb * BT;
    const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (k >= a.n) return;
    double hi[kNB], lo[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
        hi[c] = 0.0;
        lo[c] = 0.0;
    }
    for (int sp = 0; sp < split; ++sp)
#pragma unroll
        for (int c = 0; c < kNB; ++c) two_sum_acc(hi[c], lo[c], a.part[((int64_t)sp * kNB + c) * rows + k]);
    double sum[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) sum[c] = hi[c] + lo[c];
    bwd_write(a, k, sum);
}

// a_bar == NULL: only the potential-energy terms, elementwise.
__global__ void __launch_bounds__(256) backward_pot_only_kernel(const BwdArgs a)
{
    const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (k >= a.n) return;
    double zero[kNB] = {0, 0, 0, 0, 0, 0, 0};
    bwd_write(a, k, zero);
}

// Fixed tile shapes of the adjoint.
constexpr int kBwdNTf = 768, kBwdKTf = 1, kBwdSf = 256, kBwdMinBf = 1, kBwdUf = 4;
constexpr size_t kBwdSmemf = sizeof(BwdPairSmem<kBwdSf>);
constexpr int kBwdNTd = 128, kBwdKTd = 1, kBwdSd = 128, kBwdMinBd = 2;

struct BwdLayout {
    int64_t n_tiles, geo_off, src_off, part_off, total, part_cap_rows;
    int32_t max_split, S, BT;
};

int bwd_layout(const grav_params *p, int64_t n, BwdLayout *L)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    const bool mixed = p->precision == GRAV_MIXED;
    L->S = mixed ? kBwdSf : kBwdSd;
    L->BT = mixed ? kBwdNTf * kBwdKTf : kBwdNTd * kBwdKTd;
    const int64_t elem = mixed ? 16 : 32;
    L->max_split = p->max_split > 0 ? p->max_split : kDefaultMaxSplit;
    L->n_tiles = (n + L->S - 1) / L->S;
    L->geo_off = 0;
    L->src_off = round_up(L->n_tiles * (int64_t)sizeof(TileGeom), 256);
    L->part_off = L->src_off + round_up(L->n_tiles * 2 * L->S * elem, 256);
    const int64_t n_tb = (n + L->BT - 1) / L->BT;
    int64_t blocks = 0;
    if (L->max_split > 1 && L->n_tiles > 1) blocks = std::min<int64_t>(n_tb * L->max_split, 16LL * sms);
    L->part_cap_rows = blocks * L->BT;
    L->total = std::max<int64_t>(256, L->part_off + round_up(L->part_cap_rows * kNB * 8, 256));
    return GRAV_OK;
}

int bwd_grid(bool mixed, int *grid)
{
    static std::mutex mu;
    static int cache[64][2];
    int dev = 0, sms = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    rc = device_sm_count(&sms);
    if (rc) return rc;
    if (dev >= 64) return fail(GRAV_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][mixed ? 1 : 0];
    if (slot == 0) {
        int b = 0;
        cudaError_t e = cudaSuccess;
        if (mixed) {
            auto k = backward_pair_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf>;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmemf);
        }
        if (e == cudaSuccess)
            e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &b, backward_pair_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf>,
                                    kBwdNTf, kBwdSmemf)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &b, backward_kernel<double, kBwdNTd, kBwdKTd, kBwdSd, kBwdMinBd>, kBwdNTd, 0);
        rc = check_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (rc) return rc;
        if (b < 1) return fail(GRAV_ECUDA, "adjoint kernel cannot be resident on an SM");
        slot = b * sms;
    }
    *grid = slot;
    return GRAV_OK;
}

int check_bwd_params(const grav_params *p, const char *who)
{
    if (!p) return fail(GRAV_EINVAL, "%s: null params", who);
    if (!(p->G > 0.0) || !std::isfinite(p->G)) return fail(GRAV_EINVAL, "%s: G must be finite and > 0", who);
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(GRAV_EINVAL, "%s: h must be finite and > 0", who);
    if (p->precision != GRAV_F64 && p->precision != GRAV_MIXED)
        return fail(GRAV_EINVAL, "%s: precision must be GRAV_F64 or GRAV_MIXED", who);
    if (p->max_split < 0) return fail(GRAV_EINVAL, "%s: max_split < 0", who);
    if (p->box != 0.0) return fail(GRAV_EINVAL, "%s: the adjoint supports open boundaries only", who);
    return GRAV_OK;
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int64_t grav_backward_workspace_bytes(const grav_params *p, int64_t n)
{
    int rc = check_bwd_params(p, "grav_backward_workspace_bytes");
    if (rc) return rc;
    if (n < 0 || n > INT32_MAX) return fail(GRAV_EINVAL, "grav_backward_workspace_bytes: n outside [0, 2^31)");
    BwdLayout L;
    rc = bwd_layout(p, n, &L);
    if (rc) return rc;
    return L.total;
}

extern "C" int grav_eval_backward(const grav_params *p, int64_t n, const double *pos,
                                  const double *mass, const double *a_bar, double w_bar,
                                  const double *acc, const double *tidal, const double *pot,
                                  double *pos_bar, double *mass_bar, int32_t *flags_dev,
                                  void *workspace, int64_t workspace_bytes, void *stream)
{
    static const char *who = "grav_eval_backward";
    int rc = check_bwd_params(p, who);
    if (rc) return rc;
    if (n < 0 || n > INT32_MAX) return fail(GRAV_EINVAL, "%s: n outside [0, 2^31)", who);
    if (!std::isfinite(w_bar)) return fail(GRAV_EINVAL, "%s: w_bar not finite", who);
    if (n == 0) return GRAV_OK;
    if (!pos || !mass || !pos_bar || !mass_bar) return fail(GRAV_EINVAL, "%s: null array", who);
    if (a_bar && !tidal) return fail(GRAV_EINVAL, "%s: a_bar given but tidal is NULL", who);
    if (w_bar != 0.0 && (!acc || !pot)) return fail(GRAV_EINVAL, "%s: w_bar != 0 needs acc and pot", who);
    const bool mixed = p->precision == GRAV_MIXED;
    BwdLayout L;
    rc = bwd_layout(p, n, &L);
    if (rc) return rc;
    if (a_bar) {
        if (!workspace) return fail(GRAV_EINVAL, "%s: null workspace", who);
        if (!aligned(workspace, 256)) return fail(GRAV_EINVAL, "%s: workspace not 256-byte aligned", who);
        if (workspace_bytes < L.total)
            return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                        (long long)L.total);
    }
    int grid = 0;
    rc = bwd_grid(mixed, &grid);
    if (rc) return rc;
    char *ws = static_cast<char *>(workspace);
    BwdArgs a;
    a.n = n;
    a.geo = reinterpret_cast<const TileGeom *>(ws + L.geo_off);
    a.src = ws + L.src_off;
    a.n_tiles = (int32_t)L.n_tiles;
    a.max_split = L.max_split;
    a.grid = grid;
    a.pad0 = 0;
    a.part = reinterpret_cast<double *>(ws + L.part_off);
    a.part_cap_rows = L.part_cap_rows;
    a.pos = pos;
    a.mass = mass;
    a.a_bar = a_bar;
    a.w_bar = w_bar;
    a.acc = acc;
    a.tidal = tidal;
    a.pot = pot;
    a.G = p->G;
    a.h = p->h;
    double h2 = p->h * p->h;
    float h2f = (float)h2;
    if ((double)h2f < h2) h2f = std::nextafter(h2f, INFINITY);
    a.h2f_up = h2f;
    a.hinvf = (float)(1.0 / p->h);
    a.pos_bar = pos_bar;
    a.mass_bar = mass_bar;
    a.flags = flags_dev;
    cudaStream_t st = as_stream(stream);
    const unsigned eblocks = (unsigned)((n + 255) / 256);
    if (!a_bar) {
        backward_pot_only_kernel<<<eblocks, 256, 0, st>>>(a);
        return check_launch("grav_eval_backward/pot");
    }
    // Pack (x, a_bar) tiles: the forward packer with a_bar in the velocity
    // slot and no mass.
    if (mixed)
        pack_tiles_kernel<kBwdSf, true, false, true><<<(unsigned)L.n_tiles, kBwdSf, 0, st>>>(
            n, pos, a_bar, nullptr, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev);
    else
        pack_tiles_kernel<kBwdSd, false, false><<<(unsigned)L.n_tiles, kBwdSd, 0, st>>>(
            n, pos, a_bar, nullptr, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev);
    rc = check_launch("grav_eval_backward/pack");
    if (rc) return rc;
    if (mixed)
        backward_pair_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf><<<grid, kBwdNTf, kBwdSmemf, st>>>(a);
    else
        backward_kernel<double, kBwdNTd, kBwdKTd, kBwdSd, kBwdMinBd><<<grid, kBwdNTd, 0, st>>>(a);
    rc = check_launch("grav_eval_backward/sum");
    if (rc) return rc;
    const int64_t n_tb = (n + L.BT - 1) / L.BT;
    if (L.part_cap_rows > 0 &&
        choose_split(n_tb, a.n_tiles, grid, a.max_split, a.part_cap_rows, L.BT) > 1) {
        backward_reduce_kernel<<<eblocks, 256, 0, st>>>(a, L.BT);
        rc = check_launch("grav_eval_backward/reduce");
    }
    return rc;
}
