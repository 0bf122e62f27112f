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
    const float *src_lo;   // mixed: per tile, kLoPlanes planes (x, y, z) of the offsets' low parts
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
            // explicit fused multiply-adds: every kernel that inlines this
            // loop forms the same roundings
            T dx = p.x - tx[q][0], dy = p.y - tx[q][1], dz = p.z - tx[q][2];
            T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
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
            T da = fma(dx, ab.x, fma(dy, ab.y, dz * ab.z));
            acc[q][X10 + 0] = fma(f, ab.x, acc[q][X10 + 0]);
            acc[q][X10 + 1] = fma(f, ab.y, acc[q][X10 + 1]);
            acc[q][X10 + 2] = fma(f, ab.z, acc[q][X10 + 2]);
            T gd = gp * da;
            acc[q][X20 + 0] = fma(gd, dx, acc[q][X20 + 0]);
            acc[q][X20 + 1] = fma(gd, dy, acc[q][X20 + 1]);
            acc[q][X20 + 2] = fma(gd, dz, acc[q][X20 + 2]);
            acc[q][MBS] = fma(f, da, acc[q][MBS]);
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
        // (explicit fused multiply-adds: the same roundings in every kernel)
        px[0] = fma(t6[0], ak[0], fma(t6[3], ak[1], t6[4] * ak[2]));
        px[1] = fma(t6[3], ak[0], fma(t6[1], ak[1], t6[5] * ak[2]));
        px[2] = fma(t6[4], ak[0], fma(t6[5], ak[1], t6[2] * ak[2]));
        const double gm = a.G * m;
#pragma unroll
        for (int c = 0; c < 3; ++c) px[c] = fma(gm, fma(-3.0, s[X20 + c], s[X10 + c]), px[c]);
        pm = -a.G * s[MBS];
    }
    if (a.w_bar != 0.0) {
        const double wm = a.w_bar * m;
#pragma unroll
        for (int c = 0; c < 3; ++c) px[c] = fma(-wm, a.acc[3 * k + c], px[c]);
        pm = fma(a.w_bar, a.pot[k], pm);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a.pos_bar[3 * k + c] = px[c];
    a.mass_bar[k] = pm;
}

// One work item of the adjoint: the targets k0 + slot (slot < BT, below
// k_end) against the source tiles [t_begin, t_end).  With split > 1 the sums
// go to partial row slot0 + slot of chunk sp (rows per chunk), else straight
// to the outputs.
struct BwdItem {
    int64_t k0, k_end, slot0, rows;
    int32_t t_begin, t_end, sp, split;
};

// Shared memory of the scalar adjoint: a two-stage ring of (x, a_bar) tiles.
template <typename T, int S>
struct BwdScalarSmem {
    typename Src<T>::type stage[2][2 * S];
    uint64_t bar[2];
    float blo[3], bhi[3];
    int abort_flag;
    long long ticket;
};

template <typename Sm>
__device__ __forceinline__ void bwd_init_ring(Sm &sm, int stages)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&sm.bar[s], 1);
        sm.abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

// One item of the direct-sum adjoint on scalar (x, a_bar) tiles
// (instantiated for FP64; the mixed adjoint is bwd_pair_item below); false
// once a bounded wait gave up.  h2f_up: the FP32 squared support rounded up,
// for the near-tile test.
template <typename T, int NT, int KT, int S>
__device__ __forceinline__ bool bwd_scalar_item(const BwdArgs &a, BwdScalarSmem<T, S> &sm,
                                                uint32_t &parity, uint32_t &pending,
                                                const BwdItem &it, T h2, T hinv, float h2f_up)
{
    using E = typename Src<T>::type;
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int NSTAGE = 2;
    constexpr uint32_t kTileBytes = S * 2 * sizeof(E);
    const E *src = static_cast<const E *>(a.src);
    const int t_begin = it.t_begin, t_end = it.t_end;

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
        const int64_t k = it.k0 + (int64_t)q * NT + threadIdx.x;
        tk[q] = k < it.k_end ? k : -1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xk[q][c] = tk[q] >= 0 ? a.pos[3 * k + c] : 0.0;
            if (tk[q] >= 0) {
                lo[c] = fminf(lo[c], __double2float_rd(xk[q][c]));
                hi[c] = fmaxf(hi[c], __double2float_ru(xk[q][c]));
            }
        }
    }
    block_bbox<NT>(lo, hi, sm.blo, sm.bhi);
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
                tma_load_1d(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes, &sm.bar[s]);
                pending |= 1u << s;
            }
        }
    }
    for (int t = t_begin; t < t_end; ++t) {
        const int s = (t - t_begin) % NSTAGE;
        const TileGeom g = a.geo[t];
        const bool near = tile_is_near(blo_r, bhi_r, g, h2f_up);
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
        const bool got = mbar_wait_bounded(&sm.bar[s], (parity >> s) & 1u, a.flags);
        if (got)
            parity ^= 1u << s;
        else
            atomicExch(&sm.abort_flag, 1);
        T acc[KT][kNB];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNB; ++c) acc[q][c] = T(0);
        if (!near)
            bwd_loop<T, KT, S, false>(sm.stage[s], sm.stage[s] + S, tx, tk, g.first, h2, hinv, acc);
        else
            bwd_loop<T, KT, S, true>(sm.stage[s], sm.stage[s] + S, tx, tk, g.first, h2, hinv, acc);
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNB; ++c) two_sum_acc(shi[q][c], slo[q][c], acc[q][c]);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (got) pending &= ~(1u << s);
            if (t + NSTAGE < t_end && !sm.abort_flag) {
                tma_load_1d(sm.stage[s], src + (int64_t)(t + NSTAGE) * 2 * S, kTileBytes, &sm.bar[s]);
                pending |= 1u << s;
            }
        }
        if (sm.abort_flag) break;
    }
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        double sum[kNB];
#pragma unroll
        for (int c = 0; c < kNB; ++c) sum[c] = (double)shi[q][c] + (double)slo[q][c];
        const int64_t slot = it.slot0 + (int64_t)q * NT + threadIdx.x;
        if (it.split == 1) {
            if (tk[q] >= 0) bwd_write(a, tk[q], sum);
        } else {
#pragma unroll
            for (int c = 0; c < kNB; ++c) a.part[((int64_t)it.sp * kNB + c) * it.rows + slot] = sum[c];
        }
    }
    return !sm.abort_flag;
}

template <typename Sm>
__device__ __forceinline__ void bwd_drain_scalar(Sm &sm, uint32_t parity, uint32_t pending,
                                                 int32_t *flags)
{
    if (threadIdx.x == 0 && pending) {
        for (int s = 0; s < 2; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&sm.bar[s], (parity >> s) & 1u, flags);
    }
}

// The scalar adjoint over all n elements: work items of target blocks x
// source chunks.
template <typename T, int NT, int KT, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB)
backward_kernel(const BwdArgs a)
{
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int BT = NT * KT;
    __shared__ __align__(128) BwdScalarSmem<T, S> sm;
    bwd_init_ring(sm, 2);
    uint32_t parity = 0, pending = 0;

    const int64_t n_tb = (a.n + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    const int64_t items = n_tb * split;
    const int64_t rows = n_tb * BT;
    const T h2 = MIXED ? (T)a.h2f_up : (T)(a.h * a.h);
    const T hinv = MIXED ? (T)a.hinvf : (T)(1.0 / a.h);

    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        BwdItem it;
        it.k0 = tb * BT;
        it.k_end = a.n;
        it.slot0 = tb * BT;
        it.rows = rows;
        it.t_begin = (int)((int64_t)sp * a.n_tiles / split);
        it.t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);
        it.sp = sp;
        it.split = split;
        if (!bwd_scalar_item<T, NT, KT, S>(a, sm, parity, pending, it, h2, hinv, a.h2f_up)) break;
        __syncthreads();
    }
    bwd_drain_scalar(sm, parity, pending, a.flags);
}

// Batched scalar adjoint: the items of all systems from the plan, taken
// through an atomic ticket; each system's targets against its own tiles
// with its own support h (grav_system.h, or the call's h where it is 0).
template <int NT, int KT, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB)
backward_batched_kernel(const BwdArgs a, const BatchView b)
{
    constexpr int BT = NT * KT;
    __shared__ __align__(128) BwdScalarSmem<double, S> sm;
    bwd_init_ring(sm, 2);
    uint32_t parity = 0, pending = 0;
    const int64_t total = b.hdr->total_items;
    for (;;) {
        if (threadIdx.x == 0) sm.ticket = (long long)atomicAdd(&b.hdr->ticket, 1ULL);
        __syncthreads();
        const int64_t ticket = sm.ticket;
        __syncthreads();
        if (ticket >= total) break;
        const int r = item_rank(b, ticket);
        const int s = b.order[r];
        const double h = b.sys[s].h > 0.0 ? b.sys[s].h : a.h;
        float h2f, hinvf;
        softening_f(h, h2f, hinvf);
        BwdItem it;
        it.k0 = (int64_t)b.idx_lo[s] + (ticket - b.item_off[r]) * BT;
        it.k_end = b.idx_hi[s];
        it.slot0 = 0;
        it.rows = 0;
        it.t_begin = b.tile_off[s];
        it.t_end = b.tile_off[s + 1];
        it.sp = 0;
        it.split = 1;
        if (!bwd_scalar_item<double, NT, KT, S>(a, sm, parity, pending, it, h * h, 1.0 / h, h2f)) break;
        __syncthreads();
    }
    bwd_drain_scalar(sm, parity, pending, a.flags);
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

// Pairs of one target summed in FP64 after its tiles (at most this many per
// target; past that a pair stays in the FP32 sums).
constexpr int kBwdCloseList = 64;

// Near and loose tiles on the paired layout, one source at a time (lane x of
// the accumulators), the self pair excluded by index.  Separations are formed
// from both offsets' high and low parts, d = (s - t) + (s_lo - t_lo) (lo: the
// tile's planes of low parts; tl: the targets'), so they are good to a few
// units in the last place of d however far the tile centre lies.  A pair
// within 2h of its target is offered to record(q, j) and, when taken, left
// out of the FP32 sums: it is summed in FP64 after the item's tiles, where
// one such pair can outweigh the rest of the target's sum.
template <int KT, int S, typename Record>
__device__ __forceinline__ void bwd_near_pair(const float *__restrict__ tile,
                                              const float *__restrict__ lo, const float tx[KT][3],
                                              const float tl[KT][3], const int64_t tk[KT],
                                              int64_t jbase, float h2, float hinv,
                                              float2 acc[KT][kNB], Record &record)
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
        const float xl = lo[j], yl = lo[S + j], zl = lo[2 * S + j];
        const int64_t jg = jbase + j;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float dx = (x - tx[q][0]) + (xl - tl[q][0]);
            const float dy = (y - tx[q][1]) + (yl - tl[q][1]);
            const float dz = (z - tx[q][2]) + (zl - tl[q][2]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < 4.0f * h2 && tk[q] >= 0 && jg != tk[q] && record(q, jg)) continue;
            const float ri = rsqrt_sfu(r2);
            const float ri2 = ri * ri;
            float f = ri * ri2;
            float gp = f * ri2;
            if (r2 < h2) {
                float F, Gp, P;
                spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
                f = F * hinv3;
                gp = Gp * hinv5;
                if (jg == tk[q]) {
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

// One listed pair of the mixed adjoint in FP64 (target k at FP64 position
// xk, source i != k), from the FP64 positions and a_bar: added to s[kNB].
__device__ __forceinline__ void bwd_pair_d(const BwdArgs &a, double h, const double xk[3], int64_t i,
                                           double s[kNB])
{
    double d[3], ab[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d[c] = __dsub_rn(a.pos[3 * i + c], xk[c]);
        ab[c] = a.a_bar[3 * i + c];
    }
    const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
    double f, gp;
    if (r2 < h * h) {
        const double hinv = 1.0 / h;
        double F, Gp, P;
        spline_kernel<double>(sqrt(r2) * hinv, F, Gp, P);
        const double hinv3 = hinv * hinv * hinv;
        f = F * hinv3;
        gp = Gp * hinv3 * hinv * hinv;
    } else {
        const double ri = 1.0 / sqrt(r2);
        f = ri * ri * ri;
        gp = f * ri * ri;
    }
    const double da = fma(d[0], ab[0], fma(d[1], ab[1], d[2] * ab[2]));
    const double gd = gp * da;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[X10 + c] = fma(f, ab[c], s[X10 + c]);
        s[X20 + c] = fma(gd, d[c], s[X20 + c]);
    }
    s[MBS] = fma(f, da, s[MBS]);
}

// Shared memory of the mixed adjoint: a three-stage ring of paired tiles.
template <int S>
struct BwdPairSmem {
    static constexpr int kStages = 3;
    // a stage: the paired tile (28 bytes per source), then the low parts of
    // its position offsets (12 bytes per source)
    static constexpr int kTileF4 = 7 * S / 4;
    float4 stage[kStages][kTileF4 + kLoPlanes * S / 4];
    uint64_t bar[kStages];
    int done[kStages];           // warps finished with the tile in each stage
    unsigned issued[kStages];    // copies issued into each stage
    float blo[3], bhi[3];
    int abort_flag;
    long long ticket;
};

template <int S>
__device__ __forceinline__ void bwd_pair_init(BwdPairSmem<S> &sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < BwdPairSmem<S>::kStages; ++s) {
            mbar_init(&sm.bar[s], 1);
            sm.done[s] = 0;
            sm.issued[s] = 0;
        }
        sm.abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

// Copies still in flight (only after a timed-out wait): a stage holds one
// exactly when thread 0 has seen fewer completions there than were issued.
template <int S>
__device__ __forceinline__ void bwd_pair_drain(BwdPairSmem<S> &sm, uint32_t parity, int32_t *flags)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < BwdPairSmem<S>::kStages; ++s)
            if ((sm.issued[s] & 1u) != ((parity >> s) & 1u))
                mbar_wait_bounded(&sm.bar[s], (parity >> s) & 1u, flags);
    }
}

// One item of the mixed adjoint: the structure of the forward mixed kernel
// (a three-stage TMA ring in which each warp releases a stage on its own and
// the last warp to release it issues the refill, each warp's near/far test
// against its own targets' box), with the adjoint's pair terms.  Per-tile
// FP32 sums are carried across tiles as compensated FP32 pairs (TwoSum); the
// result is FP64.  False once a bounded wait gave up.
template <int NT, int KT, int S, int U>
__device__ __forceinline__ bool bwd_pair_item(const BwdArgs &a, BwdPairSmem<S> &sm, uint32_t &parity,
                                              const BwdItem &it, double h, float h2, float hinv)
{
    using Sm = BwdPairSmem<S>;
    constexpr int NSTAGE = Sm::kStages;
    constexpr uint32_t kTileBytes = S * 28;
    const float4 *src = static_cast<const float4 *>(a.src);
    const int t_begin = it.t_begin, t_end = it.t_end;
    // a tile and the low parts of its offsets into stage s
    auto load_stage = [&](int s, int t) {
        tma_load_1d_two(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes, sm.stage[s] + Sm::kTileF4,
                        a.src_lo + (int64_t)t * kLoPlanes * S, 4u * kLoPlanes * S, &sm.bar[s]);
    };

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
        const int64_t k = it.k0 + (int64_t)q * NT + threadIdx.x;
        tk[q] = k < it.k_end ? k : -1;
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
    // pairs within 2h, listed per target for FP64
    int32_t nlist[KT][kBwdCloseList];
    int ncnt[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) ncnt[q] = 0;
    auto record = [&](int q, int64_t j) -> bool {
        if (ncnt[q] >= kBwdCloseList) return false;
        nlist[q][ncnt[q]++] = (int32_t)j;
        return true;
    };

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
                load_stage(s, t);
                sm.issued[s] += 1u;
            }
        }
    }
    for (int t = t_begin; t < t_end; ++t) {
        const int s = (t - t_begin) % NSTAGE;
        const TileGeom g = a.geo[t];
        // near: inside h of the warp's box; loose: within reach of the FP32
        // offsets' rounding (as in the forward kernel); both take the near
        // loop with two-part separations
        const float g2 = box_gap2(lo, hi, g);
        constexpr float kL = kLooseC / (1.0f - kLooseC);
        const bool close = !(g2 >= h2) || g2 < (kL * kL) * box_diag2(g.lo, g.hi);
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
        if (!close) {
            bwd_far_pair<KT, S, U>(tf, tx, acc);
        } else {
            float tl[KT][3];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    tl[q][c] = __double2float_rn(__dsub_rn(__dsub_rn(xk[q][c], g.c[c]), (double)tx[q][c]));
            bwd_near_pair<KT, S>(tf, reinterpret_cast<const float *>(sm.stage[s] + Sm::kTileF4), tx, tl,
                                 tk, g.first, h2, hinv, acc, record);
        }
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
                    load_stage(s, t + NSTAGE);
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
        for (int c = 0; c < kNB; ++c) sum[c] = 0.0;
        if (tk[q] >= 0)
            for (int k = 0; k < ncnt[q]; ++k) bwd_pair_d(a, h, xk[q], nlist[q][k], sum);
#pragma unroll
        for (int c = 0; c < kNB; ++c) sum[c] += (double)shi[q][c] + (double)slo[q][c];
        const int64_t slot = it.slot0 + (int64_t)q * NT + threadIdx.x;
        if (it.split == 1) {
            if (tk[q] >= 0) bwd_write(a, tk[q], sum);
        } else {
#pragma unroll
            for (int c = 0; c < kNB; ++c) a.part[((int64_t)it.sp * kNB + c) * it.rows + slot] = sum[c];
        }
    }
    return !sm.abort_flag;
}

// The mixed adjoint over all n elements: work items of target blocks x
// source chunks.
template <int NT, int KT, int S, int MINB, int U>
__global__ void __launch_bounds__(NT, MINB) backward_pair_kernel(const BwdArgs a)
{
    constexpr int BT = NT * KT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BwdPairSmem<S> &sm = *reinterpret_cast<BwdPairSmem<S> *>(smem_raw);
    bwd_pair_init(sm);
    uint32_t parity = 0;

    const int64_t n_tb = (a.n + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    const int64_t items = n_tb * split;
    const int64_t rows = n_tb * BT;

    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        BwdItem it;
        it.k0 = tb * BT;
        it.k_end = a.n;
        it.slot0 = tb * BT;
        it.rows = rows;
        it.t_begin = (int)((int64_t)sp * a.n_tiles / split);
        it.t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);
        it.sp = sp;
        it.split = split;
        if (!bwd_pair_item<NT, KT, S, U>(a, sm, parity, it, a.h, a.h2f_up, a.hinvf)) break;
        __syncthreads();
    }
    bwd_pair_drain(sm, parity, a.flags);
}

// Batched mixed adjoint: the items of all systems from the plan, taken
// through an atomic ticket; each system's targets against its own tiles with
// its own support h (grav_system.h, or the call's h where it is 0).
template <int NT, int KT, int S, int MINB, int U>
__global__ void __launch_bounds__(NT, MINB) backward_pair_batched_kernel(const BwdArgs a,
                                                                         const BatchView b)
{
    constexpr int BT = NT * KT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BwdPairSmem<S> &sm = *reinterpret_cast<BwdPairSmem<S> *>(smem_raw);
    bwd_pair_init(sm);
    uint32_t parity = 0;
    const int64_t total = b.hdr->total_items;
    for (;;) {
        if (threadIdx.x == 0) sm.ticket = (long long)atomicAdd(&b.hdr->ticket, 1ULL);
        __syncthreads();
        const int64_t ticket = sm.ticket;
        __syncthreads();
        if (ticket >= total) break;
        const int r = item_rank(b, ticket);
        const int s = b.order[r];
        const double h = b.sys[s].h > 0.0 ? b.sys[s].h : a.h;
        float h2f, hinvf;
        softening_f(h, h2f, hinvf);
        BwdItem it;
        it.k0 = (int64_t)b.idx_lo[s] + (ticket - b.item_off[r]) * BT;
        it.k_end = b.idx_hi[s];
        it.slot0 = 0;
        it.rows = 0;
        it.t_begin = b.tile_off[s];
        it.t_end = b.tile_off[s + 1];
        it.sp = 0;
        it.split = 1;
        if (!bwd_pair_item<NT, KT, S, U>(a, sm, parity, it, h, h2f, hinvf)) break;
        __syncthreads();
    }
    bwd_pair_drain(sm, parity, a.flags);
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
    int64_t n_tiles, geo_off, src_off, lo_off, part_off, total, part_cap_rows;
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
    L->lo_off = L->src_off + round_up(L->n_tiles * 2 * L->S * elem, 256);
    L->part_off = L->lo_off + round_up(mixed ? L->n_tiles * kLoPlanes * L->S * 4 : 0, 256);
    const int64_t n_tb = (n + L->BT - 1) / L->BT;
    int64_t blocks = 0;
    if (L->max_split > 1 && L->n_tiles > 1) blocks = std::min<int64_t>(n_tb * L->max_split, 16LL * sms);
    L->part_cap_rows = blocks * L->BT;
    L->total = std::max<int64_t>(256, L->part_off + round_up(L->part_cap_rows * kNB * 8, 256));
    return GRAV_OK;
}

int bwd_grid(bool mixed, bool batched, int *grid)
{
    static std::mutex mu;
    static int cache[64][2][2];
    int dev = 0, sms = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    rc = device_sm_count(&sms);
    if (rc) return rc;
    if (dev >= 64) return fail(GRAV_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][mixed ? 1 : 0][batched ? 1 : 0];
    if (slot == 0) {
        int b = 0;
        cudaError_t e = cudaSuccess;
        if (mixed && !batched) {
            auto k = backward_pair_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf>;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmemf);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kBwdNTf, kBwdSmemf);
        } else if (mixed) {
            auto k = backward_pair_batched_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf>;
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmemf);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kBwdNTf, kBwdSmemf);
        } else if (!batched) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b, backward_kernel<double, kBwdNTd, kBwdKTd, kBwdSd, kBwdMinBd>, kBwdNTd, 0);
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b, backward_batched_kernel<kBwdNTd, kBwdKTd, kBwdSd, kBwdMinBd>, kBwdNTd, 0);
        }
        rc = check_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (rc) return rc;
        if (b < 1) return fail(GRAV_ECUDA, "adjoint kernel cannot be resident on an SM");
        slot = b * sms;
    }
    *grid = slot;
    return GRAV_OK;
}

// Workspace of a batched adjoint: the plan's arrays, then the tiles.
struct BwdBatchLayout {
    int64_t hdr, tile_off, idx_lo, idx_hi, ntb, order, item_off, geo, src, lo, total, max_tiles;
};

BwdBatchLayout bwd_batch_layout(bool mixed, int32_t n_sys, int64_t n_total)
{
    BwdBatchLayout L;
    const int64_t S = mixed ? kBwdSf : kBwdSd;
    const int64_t elem = mixed ? 16 : 32;
    L.max_tiles = (n_total + S - 1) / S + n_sys;
    int64_t o = 0;
    L.hdr = o;
    o += 256;
    L.tile_off = o;
    o += round_up(4 * ((int64_t)n_sys + 1), 256);
    L.idx_lo = o;
    o += round_up(4 * (int64_t)n_sys, 256);
    L.idx_hi = o;
    o += round_up(4 * (int64_t)n_sys, 256);
    L.ntb = o;
    o += round_up(4 * (int64_t)n_sys, 256);
    L.order = o;
    o += round_up(4 * (int64_t)n_sys, 256);
    L.item_off = o;
    o += round_up(8 * ((int64_t)n_sys + 1), 256);
    L.geo = o;
    o += round_up(L.max_tiles * (int64_t)sizeof(TileGeom), 256);
    L.src = o;
    o += round_up(L.max_tiles * 2 * S * elem, 256);
    L.lo = o;
    o += round_up(mixed ? L.max_tiles * kLoPlanes * S * 4 : 0, 256);
    L.total = o;
    return L;
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
    rc = bwd_grid(mixed, false, &grid);
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
    a.src_lo = mixed ? reinterpret_cast<const float *>(ws + L.lo_off) : nullptr;
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
            n, pos, a_bar, nullptr, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev,
            const_cast<float *>(a.src_lo));
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

extern "C" int64_t grav_backward_batched_workspace_bytes(const grav_params *p, int32_t n_sys,
                                                        int64_t n_total)
{
    static const char *who = "grav_backward_batched_workspace_bytes";
    int rc = check_bwd_params(p, who);
    if (rc) return rc;
    if (n_sys < 0 || n_sys > GRAV_BATCH_MAX_SYSTEMS)
        return fail(GRAV_EINVAL, "%s: n_sys outside [0, %d]", who, GRAV_BATCH_MAX_SYSTEMS);
    if (n_total < 0 || n_total > INT32_MAX) return fail(GRAV_EINVAL, "%s: n_total outside [0, 2^31)", who);
    return bwd_batch_layout(p->precision == GRAV_MIXED, n_sys, n_total).total;
}

extern "C" int grav_eval_backward_batched(const grav_params *p, int32_t n_sys,
                                          const grav_system *systems, int64_t n_total,
                                          const double *pos, const double *mass, const double *a_bar,
                                          double w_bar, const double *acc, const double *tidal,
                                          const double *pot, double *pos_bar, double *mass_bar,
                                          int32_t *flags_dev, void *workspace,
                                          int64_t workspace_bytes, void *stream)
{
    static const char *who = "grav_eval_backward_batched";
    int rc = check_bwd_params(p, who);
    if (rc) return rc;
    if (n_sys < 0 || n_sys > GRAV_BATCH_MAX_SYSTEMS)
        return fail(GRAV_EINVAL, "%s: n_sys outside [0, %d]", who, GRAV_BATCH_MAX_SYSTEMS);
    if (n_total < 0 || n_total > INT32_MAX) return fail(GRAV_EINVAL, "%s: n_total outside [0, 2^31)", who);
    if (!std::isfinite(w_bar)) return fail(GRAV_EINVAL, "%s: w_bar not finite", who);
    if (n_sys == 0 || n_total == 0) return GRAV_OK;
    if (!systems || !pos || !mass || !pos_bar || !mass_bar) return fail(GRAV_EINVAL, "%s: null array", who);
    if (a_bar && !tidal) return fail(GRAV_EINVAL, "%s: a_bar given but tidal is NULL", who);
    if (w_bar != 0.0 && (!acc || !pot)) return fail(GRAV_EINVAL, "%s: w_bar != 0 needs acc and pot", who);
    if (!workspace || !aligned(workspace, 256))
        return fail(GRAV_EINVAL, "%s: workspace missing or not 256-byte aligned", who);
    const bool mixed = p->precision == GRAV_MIXED;
    const BwdBatchLayout L = bwd_batch_layout(mixed, n_sys, n_total);
    if (workspace_bytes < L.total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)L.total);
    int grid = 0;
    rc = bwd_grid(mixed, true, &grid);
    if (rc) return rc;
    char *ws = static_cast<char *>(workspace);
    BatchView b;
    b.hdr = reinterpret_cast<BatchHeader *>(ws + L.hdr);
    b.sys = systems;
    b.tile_off = reinterpret_cast<int32_t *>(ws + L.tile_off);
    b.idx_lo = reinterpret_cast<int32_t *>(ws + L.idx_lo);
    b.idx_hi = reinterpret_cast<int32_t *>(ws + L.idx_hi);
    b.ntb = reinterpret_cast<int32_t *>(ws + L.ntb);
    b.order = reinterpret_cast<int32_t *>(ws + L.order);
    b.item_off = reinterpret_cast<int64_t *>(ws + L.item_off);
    b.n_sys = n_sys;
    b.pad = 0;

    BwdArgs a;
    a.n = n_total;
    a.geo = reinterpret_cast<const TileGeom *>(ws + L.geo);
    a.src = ws + L.src;
    a.n_tiles = 0;
    a.max_split = 1;
    a.grid = grid;
    a.pad0 = 0;
    a.part = nullptr;
    a.part_cap_rows = 0;
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
    a.src_lo = mixed ? reinterpret_cast<const float *>(ws + L.lo) : nullptr;
    cudaStream_t st = as_stream(stream);
    if (!a_bar) {
        // only the potential-energy terms, elementwise (no system structure)
        backward_pot_only_kernel<<<(unsigned)((n_total + 255) / 256), 256, 0, st>>>(a);
        return check_launch("grav_eval_backward_batched/pot");
    }
    const int32_t S = mixed ? kBwdSf : kBwdSd;
    const int32_t BT = mixed ? kBwdNTf * kBwdKTf : kBwdNTd * kBwdKTd;
    // every element a target: the plan takes each system's element range
    rc = launch_batch_plan(b, nullptr, nullptr, n_total, n_total, S, BT, 0.0, flags_dev, st);
    if (rc) return rc;
    // (x, a_bar) tiles: the forward's batched packer with a_bar in the
    // velocity slot and no mass
    if (mixed)
        pack_tiles_batched_kernel<kBwdSf, true, false, true><<<(unsigned)L.max_tiles, kBwdSf, 0, st>>>(
            b, pos, a_bar, nullptr, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev,
            const_cast<float *>(a.src_lo));
    else
        pack_tiles_batched_kernel<kBwdSd, false, false, false><<<(unsigned)L.max_tiles, kBwdSd, 0, st>>>(
            b, pos, a_bar, nullptr, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev,
            nullptr);
    rc = check_launch("grav_eval_backward_batched/pack");
    if (rc) return rc;
    if (mixed)
        backward_pair_batched_kernel<kBwdNTf, kBwdKTf, kBwdSf, kBwdMinBf, kBwdUf>
            <<<grid, kBwdNTf, kBwdSmemf, st>>>(a, b);
    else
        backward_batched_kernel<kBwdNTd, kBwdKTd, kBwdSd, kBwdMinBd><<<grid, kBwdNTd, 0, st>>>(a, b);
    return check_launch("grav_eval_backward_batched/sum");
}
