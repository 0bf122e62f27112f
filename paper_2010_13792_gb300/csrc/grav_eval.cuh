// Force evaluation kernels of libgrav (Grudic 2020, Eq. 4 and Section 3).
//
// Direct summation, target-blocked: a CTA owns a block of BT = NT*KT targets
// (KT per thread) and streams source tiles of S elements through shared
// memory with 1-D TMA bulk copies (cp.async.bulk + mbarrier).  Mixed kernels:
// a ring of three stages, each released by every warp on its own and refilled
// by the last warp to release it, so no block barrier separates the tiles and
// each warp tests tiles against its own targets' box; FP64 kernels: two
// stages and a block barrier after every tile.  Every thread evaluates each staged source
// against its KT targets with the SFU reciprocal square root; all lanes read
// the same source (shared-memory broadcast).  This is CUDA-core work, not a
// contraction: no tensor cores.
//
// Accumulated sums per target (d = x_j - x_i, g' = -g/3 = r^-5 beyond h):
//   A  = sum m f d          Tp = sum m g' d d^T       P = sum m phi (optional)
//   J1 = sum m f v          J2 = sum m g' (d.v) d
// and the trace term F = sum m f.  The epilogue forms
//   a = G A,  j = G (J1 - 3 J2),  T = -G (F I - 3 Tp),  Phi = -G P,
// and the tidal timestep of Eq. (tidaltimestep) in FP64.
//
// Mixed precision (K5): positions are FP64; each source tile stores FP32
// offsets from its FP64 bounding-box centre and FP32 velocities relative to
// its velocity centre; each target's offset to the tile centre is formed in
// FP64 and rounded once.  Two identities keep the pair body at 31 FP32
// instructions + 1 MUFU:
//   * beyond h, m f = m r^-3 = m r^-5 r^2, so F = trace(Tp) + E with
//     E = sum (m f - m g' r^2) over softened pairs only;
//   * v = v_j' - v_i' (both relative to the tile's velocity centre), so the
//     per-tile sums J1 = sum m f v_j' - v_i' F_tile and
//     J2 = sum m g' (d.v_j') d - Tp_tile v_i' take the target velocity out of
//     the pair loop.
// Per-tile sums are FP32; they are carried across tiles as compensated FP32
// pairs (TwoSum), in registers or in shared memory, and the final per-target
// result is FP64.  The FP64 path (K4) accumulates the sums in FP64, with the
// second identity (tile-relative velocities) but F summed directly.
//
// Tiles whose bounding box lies at least h from the bounding box of the
// targets of a warp (of the block in the FP64 adaptive-softening kernel) take
// the Newtonian loop (exact there: the cubic spline has compact support); the
// others take the softened loop, which also excludes the self pair by index.
//
// Work items are (target block, source chunk).  A fixed grid of CTAs takes
// items round-robin; when the target set is small the sources are split into
// chunks so that every SM has work, and the chunk partials are reduced by a
// second kernel in a fixed order (deterministic results).
#pragma once

#include "grav_common.cuh"

namespace grav {

constexpr int kNC = 16;            // accumulators without the potential
constexpr int kNCPot = 17;         // with the potential
constexpr int kDefaultMaxSplit = 64;

// Accumulator slots.  Slot 9 holds F (FP64 path) or E (mixed path).
enum { A0 = 0, J10 = 3, J20 = 6, FSUM = 9, ESUM = 9, TXX = 10, TYY, TZZ, TXY, TXZ, TYZ, PSUM = 16 };

struct __align__(16) TileGeom {
    double c[3];    // FP64 bounding-box centre of the positions (offset origin, mixed path)
    float lo[3];    // bounding box, rounded outward to FP32
    float hi[3];
    int32_t first;  // element index of the tile's first source
    float cv[3];    // velocity centre (mixed path; 0 when velocities are stored as they are)
};
static_assert(sizeof(TileGeom) == 64, "TileGeom layout");

struct __align__(16) D4 {
    double x, y, z, w;
};

// Boundary and softening mode of a force-kernel instantiation.
enum : int {
    kModeOpen = 0,       // open boundaries, one support h for every pair
    kModePeriodic = 1,   // nearest periodic image in a cube of side box
    kModeSoft = 2,       // per-element supports and the adaptive-softening correction
};

struct EvalArgs {
    int64_t n_src;
    const int32_t *idx;        // nullable: targets are 0..n_idx_max-1
    const int32_t *n_idx_dev;  // nullable: count is n_idx_max
    int64_t n_idx_max;
    const TileGeom *geo;
    const void *src;           // packed tiles
    int32_t n_tiles;
    int32_t max_split;
    int32_t grid;              // CTAs of the persistent launch (split policy input)
    int32_t pad0;
    double *part;              // split partials
    int64_t part_cap_rows;     // partial rows available (each row NC doubles)
    const double *pos;
    const double *vel;
    const double *mass;           // FP64 masses (the periodic close field reads them)
    double G, h, sqrt_eta;
    float hf, h2f_up, hinvf, pad1;
    double *acc, *jerk, *tidal, *pot, *dt_grav;
    int32_t *flags;
    double box, box_inv;          // periodic cube side and its inverse (box = 0: open)
    double box_tie;               // FP64 path: |d_c| above it re-decides the image by division
    float box_f, box_inv_f;
    float box_tie_f;              // mixed path: |d_c| above it may be an ambiguous image
    float box_lo_f;               // box - box_f, rounded (the low part of the side)
    // mixed path: the low parts of the packed sources' position and velocity
    // offsets, per tile kLoPlanes planes of S (offset = high + low to 2^-48)
    const float *src_lo;

    // adaptive softening (kModeSoft): per-element supports h and correction
    // coefficients zeta (zeta nullable: no correction), FP64 by element; the
    // mixed kernels read them per source as (1/h, zeta) in FP32 from hz and
    // the outward-rounded largest support of each source tile from geo_h
    const double *h_elem;
    const double *zeta;
    const float2 *hz;
    const float *geo_h;
};

// Number of source chunks per target block.  Shared by the host, the eval
// kernel and the reduction kernel, so it must depend only on its arguments.
__host__ __device__ inline int choose_split(int64_t n_tb, int32_t n_tiles, int32_t grid,
                                            int32_t max_split, int64_t part_cap_rows, int32_t BT)
{
    if (n_tb <= 0 || max_split <= 1 || n_tiles <= 1 || grid <= 0) return 1;
    if (n_tb >= 4LL * grid) return 1;
    int64_t s_max = max_split < n_tiles ? max_split : n_tiles;
    int64_t cap = part_cap_rows / (n_tb * (int64_t)BT);
    if (cap < s_max) s_max = cap;
    if (s_max <= 1) return 1;
    int64_t best = 1, best_items = n_tb, best_slots = ((n_tb + grid - 1) / grid) * grid;
    for (int64_t s = 1; s <= s_max; ++s) {
        int64_t items = n_tb * s;
        int64_t slots = ((items + grid - 1) / grid) * grid;
        if (items >= grid && 20 * items >= 19 * slots) return (int)s;
        if (items * best_slots > best_items * slots) {
            best = s;
            best_items = items;
            best_slots = slots;
        }
    }
    return (int)best;
}

__device__ __forceinline__ int64_t active_count(const EvalArgs &a)
{
    int64_t n = a.n_idx_max;
    if (a.n_idx_dev) {
        int64_t c = *a.n_idx_dev;
        if (c < 0) c = 0;
        if (c < n) n = c;
    }
    return n;
}

// Final FP64 outputs of one target from its accumulated sums.  ETRACE: slot 9
// holds E and F = E + trace(Tp) (mixed path); otherwise slot 9 holds F.
// Every operation is an explicit correctly rounded intrinsic, so all kernels
// that end in this epilogue (single-system, batched, reduction) turn the same
// sums into bit-identical outputs whatever the compiler fuses elsewhere.
template <bool POT, bool ETRACE>
__device__ __forceinline__ void write_target(const EvalArgs &a, int64_t i, const double s[kNCPot])
{
    const double G = a.G;
    const double F = ETRACE ? __dadd_rn(s[ESUM], __dadd_rn(__dadd_rn(s[TXX], s[TYY]), s[TZZ]))
                            : s[FSUM];
    const double G3 = __dmul_rn(3.0, G);
    double t6[6];
    t6[0] = __dmul_rn(-G, __dsub_rn(F, __dmul_rn(3.0, s[TXX])));
    t6[1] = __dmul_rn(-G, __dsub_rn(F, __dmul_rn(3.0, s[TYY])));
    t6[2] = __dmul_rn(-G, __dsub_rn(F, __dmul_rn(3.0, s[TZZ])));
    t6[3] = __dmul_rn(G3, s[TXY]);
    t6[4] = __dmul_rn(G3, s[TXZ]);
    t6[5] = __dmul_rn(G3, s[TYZ]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.acc[3 * i + c] = __dmul_rn(G, s[A0 + c]);
        a.jerk[3 * i + c] = __dmul_rn(G, __dsub_rn(s[J10 + c], __dmul_rn(3.0, s[J20 + c])));
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) a.tidal[6 * i + c] = t6[c];
    if (POT) a.pot[i] = __dmul_rn(-G, s[PSUM]);
    if (a.dt_grav) a.dt_grav[i] = tidal_dt(t6, a.sqrt_eta);
}

// Is the source tile within h of the target block (conservative: any doubt
// means "near")?  blo/bhi is the target block's outward-rounded bbox.
__device__ __forceinline__ bool tile_is_near(const float blo[3], const float bhi[3],
                                             const TileGeom &g, float h2_up)
{
    float d2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float gap = fmaxf(0.0f, fmaxf(__fsub_rd(g.lo[c], bhi[c]), __fsub_rd(blo[c], g.hi[c])));
        d2 = __fmaf_rd(gap, gap, d2);
    }
    return !(d2 >= h2_up);
}

// Block reduction of the targets' outward bounding box into shared blo/bhi.
template <int NT>
__device__ __forceinline__ void block_bbox(float lo[3], float hi[3], float *blo, float *bhi)
{
    __shared__ float wlo[3][NT / 32], whi[3][NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
        if (lane == 0) {
            wlo[c][wid] = lo[c];
            whi[c][wid] = hi[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float l = wlo[threadIdx.x][0], h = whi[threadIdx.x][0];
        for (int w = 1; w < NT / 32; ++w) {
            l = fminf(l, wlo[threadIdx.x][w]);
            h = fmaxf(h, whi[threadIdx.x][w]);
        }
        blo[threadIdx.x] = l;
        bhi[threadIdx.x] = h;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tile packing (K3)
// ---------------------------------------------------------------------------

// Block-wide FP64 min/max over S threads.
template <int S>
__device__ __forceinline__ void block_minmax_d(double lo[3], double hi[3], double *slo, double *shi)
{
    __shared__ double wlo[3][S / 32], whi[3][S / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
        if (lane == 0) {
            wlo[c][wid] = lo[c];
            whi[c][wid] = hi[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double l = wlo[threadIdx.x][0], h = whi[threadIdx.x][0];
        for (int w = 1; w < S / 32; ++w) {
            l = fmin(l, wlo[threadIdx.x][w]);
            h = fmax(h, whi[threadIdx.x][w]);
        }
        slo[threadIdx.x] = l;
        shi[threadIdx.x] = h;
    }
    __syncthreads();
}

// Planes of low parts per packed mixed tile: x, y, z.
constexpr int kLoPlanes = 3;

// One CTA of S threads packs one tile holding the sources [first, end).
// MIXED: tile = [S x float4 (offset, m)][S x float4 (v', 0)] (v' = v - cv
// when VOFF, else v); F64: tile = [S x D4 (x, m)][S x D4 (v, 0)].  Padding
// sources have zero mass and sit far away, so they contribute exactly 0.
// `mass` may be NULL (zero masses: the adjoint packs a_bar as "velocity").
template <int S, bool MIXED, bool VOFF, bool PAIR = false>
__device__ __forceinline__ void pack_tile(int t, int64_t first, int64_t end,
                                          const double *__restrict__ pos,
                                          const double *__restrict__ vel,
                                          const double *__restrict__ mass,
                                          TileGeom *__restrict__ geo, void *__restrict__ src,
                                          int32_t *flags, float *__restrict__ src_lo = nullptr)
{
    __shared__ double slo[3], shi[3], svlo[3], svhi[3];
    const int j = threadIdx.x;
    const int64_t gj = first + j;
    const bool ok = gj < end;
    double x[3] = {0, 0, 0}, v[3] = {0, 0, 0}, m = 0.0;
    if (ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = pos[3 * gj + c];
            v[c] = vel[3 * gj + c];
        }
        m = mass ? mass[gj] : 0.0;
        if (!(finite3(x[0], x[1], x[2]) && finite3(v[0], v[1], v[2]) && isfinite(m)))
            flag_or(flags, GRAV_FLAG_NONFINITE);
    }
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = ok ? x[c] : inf;
        hi[c] = ok ? x[c] : -inf;
    }
    block_minmax_d<S>(lo, hi, slo, shi);
    float cvf[3] = {0.0f, 0.0f, 0.0f};
    if (VOFF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = ok ? v[c] : inf;
            hi[c] = ok ? v[c] : -inf;
        }
        block_minmax_d<S>(lo, hi, svlo, svhi);
#pragma unroll
        for (int c = 0; c < 3; ++c) cvf[c] = __double2float_rn(__dmul_rn(0.5, __dadd_rn(svlo[c], svhi[c])));
    }
    double cc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) cc[c] = __dmul_rn(0.5, __dadd_rn(slo[c], shi[c]));
    if (MIXED && src_lo) {
        // low parts of the FP32 position offsets (zero for padding), planes
        // [x y z] of S each
        float *lo_t = src_lo + (int64_t)t * kLoPlanes * S;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float lx = 0.0f;
            if (ok) {
                const double d = __dsub_rn(x[c], cc[c]);
                lx = __double2float_rn(__dsub_rn(d, (double)__double2float_rn(d)));
            }
            lo_t[c * S + j] = lx;
        }
    }
    if (MIXED && PAIR) {
        // paired layout: for source j = 2k + h, floats
        //   [4k + h] x, [4k + 2 + h] y          (S/2 float4: x0 x1 y0 y1)
        //   [2S + 4k + h] z, [2S + 4k + 2 + h] m (S/2 float4: z0 z1 m0 m1)
        //   [4S + 4k + h] vx, [4S + 4k + 2 + h] vy
        //   [6S + 2k + h] vz                     (S/2 float2)
        float *tile = static_cast<float *>(src) + (int64_t)t * 8 * S;
        const int k = j >> 1, h = j & 1;
        float px = 1.0e18f, py = 0.0f, pz = 0.0f, pmv = 0.0f, qx = 0.0f, qy = 0.0f, qz = 0.0f;
        if (ok) {
            px = __double2float_rn(__dsub_rn(x[0], cc[0]));
            py = __double2float_rn(__dsub_rn(x[1], cc[1]));
            pz = __double2float_rn(__dsub_rn(x[2], cc[2]));
            pmv = __double2float_rn(m);
            qx = __double2float_rn(__dsub_rn(v[0], (double)cvf[0]));
            qy = __double2float_rn(__dsub_rn(v[1], (double)cvf[1]));
            qz = __double2float_rn(__dsub_rn(v[2], (double)cvf[2]));
        }
        tile[4 * k + h] = px;
        tile[4 * k + 2 + h] = py;
        tile[2 * S + 4 * k + h] = pz;
        tile[2 * S + 4 * k + 2 + h] = pmv;
        tile[4 * S + 4 * k + h] = qx;
        tile[4 * S + 4 * k + 2 + h] = qy;
        tile[6 * S + 2 * k + h] = qz;
    } else if (MIXED) {
        float4 *tile = static_cast<float4 *>(src) + (int64_t)t * 2 * S;
        float4 pm, pv;
        if (ok) {
            pm = make_float4(__double2float_rn(__dsub_rn(x[0], cc[0])),
                             __double2float_rn(__dsub_rn(x[1], cc[1])),
                             __double2float_rn(__dsub_rn(x[2], cc[2])), __double2float_rn(m));
            pv = make_float4(__double2float_rn(__dsub_rn(v[0], (double)cvf[0])),
                             __double2float_rn(__dsub_rn(v[1], (double)cvf[1])),
                             __double2float_rn(__dsub_rn(v[2], (double)cvf[2])), 0.0f);
        } else {
            pm = make_float4(1.0e18f, 0.0f, 0.0f, 0.0f);
            pv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        tile[j] = pm;
        tile[S + j] = pv;
    } else {
        D4 *tile = static_cast<D4 *>(src) + (int64_t)t * 2 * S;
        D4 pm, pv;
        if (ok) {
            pm = D4{x[0], x[1], x[2], m};
            pv = D4{v[0] - (double)cvf[0], v[1] - (double)cvf[1], v[2] - (double)cvf[2], 0.0};
        } else {
            pm = D4{1.0e150, 0.0, 0.0, 0.0};
            pv = D4{0.0, 0.0, 0.0, 0.0};
        }
        tile[j] = pm;
        tile[S + j] = pv;
    }
    if (j == 0) {
        TileGeom g;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            g.c[c] = cc[c];
            g.lo[c] = __double2float_rd(slo[c]);
            g.hi[c] = __double2float_ru(shi[c]);
            g.cv[c] = cvf[c];
        }
        g.first = (int32_t)first;
        geo[t] = g;
    }
}

// Single system: tile t holds sources [t*S, min((t+1)*S, n_src)).
template <int S, bool MIXED, bool VOFF, bool PAIR = false>
__global__ void __launch_bounds__(S)
pack_tiles_kernel(int64_t n_src, const double *__restrict__ pos, const double *__restrict__ vel,
                  const double *__restrict__ mass, TileGeom *__restrict__ geo, void *__restrict__ src,
                  int32_t *flags, float *__restrict__ src_lo = nullptr)
{
    const int64_t first = (int64_t)blockIdx.x * S;
    const int64_t end = first + S < n_src ? first + S : n_src;
    pack_tile<S, MIXED, VOFF, PAIR>(blockIdx.x, first, end, pos, vel, mass, geo, src, flags,
                                    src_lo);
}

// ---------------------------------------------------------------------------
// Cubic-spline kernel inside the support, u = r/h in [0, 1):
//   F  = h^3 f        (f = M(<r)/(m r^3))
//   Gp = -h^5 g / 3   (g = f'(r)/r; Gp -> u^-5 at u = 1, matching g' = r^-5)
//   P  = h phi        (potential kernel, 2.8 at u = 0, 1 at u = 1)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void spline_kernel(T u, T &F, T &Gp, T &P)
{
    const T u2 = u * u;
    if (u < T(0.5)) {
        F = T(32.0 / 3.0) + u2 * (T(-192.0 / 5.0) + T(32.0) * u);
        Gp = T(128.0 / 5.0) - T(32.0) * u;
        P = T(14.0 / 5.0) + u2 * (T(-16.0 / 3.0) + u2 * (T(48.0 / 5.0) - T(32.0 / 5.0) * u));
    } else {
        const T ui = T(1) / u;
        const T ui3 = ui * ui * ui;
        F = T(64.0 / 3.0) + u * (T(-48.0) + u * (T(192.0 / 5.0) - T(32.0 / 3.0) * u)) -
            ui3 * T(1.0 / 15.0);
        Gp = T(16.0) * ui - T(128.0 / 5.0) + T(32.0 / 3.0) * u - ui3 * ui * ui * T(1.0 / 15.0);
        P = T(16.0 / 5.0) - ui * T(1.0 / 15.0) +
            u2 * (T(-32.0 / 3.0) + u * (T(16.0) + u * (T(-48.0 / 5.0) + T(32.0 / 15.0) * u)));
    }
}

// ---------------------------------------------------------------------------
// Pair loops, mixed precision
// ---------------------------------------------------------------------------

// Sums of one pair (target q): A, J1', J2', Tp (and P).  v' is the source
// velocity relative to the tile's velocity centre.
template <int KT, bool POT>
__device__ __forceinline__ void accumulate_f(float acc[KT][kNCPot], int q, float dx, float dy,
                                             float dz, float vx, float vy, float vz, float mf,
                                             float mg, float mp)
{
    acc[q][A0 + 0] = fmaf(mf, dx, acc[q][A0 + 0]);
    acc[q][A0 + 1] = fmaf(mf, dy, acc[q][A0 + 1]);
    acc[q][A0 + 2] = fmaf(mf, dz, acc[q][A0 + 2]);
    acc[q][J10 + 0] = fmaf(mf, vx, acc[q][J10 + 0]);
    acc[q][J10 + 1] = fmaf(mf, vy, acc[q][J10 + 1]);
    acc[q][J10 + 2] = fmaf(mf, vz, acc[q][J10 + 2]);
    float dv = fmaf(dx, vx, fmaf(dy, vy, dz * vz));
    float gx = mg * dx, gy = mg * dy, gz = mg * dz;
    acc[q][TXX] = fmaf(gx, dx, acc[q][TXX]);
    acc[q][TYY] = fmaf(gy, dy, acc[q][TYY]);
    acc[q][TZZ] = fmaf(gz, dz, acc[q][TZZ]);
    acc[q][TXY] = fmaf(gx, dy, acc[q][TXY]);
    acc[q][TXZ] = fmaf(gx, dz, acc[q][TXZ]);
    acc[q][TYZ] = fmaf(gy, dz, acc[q][TYZ]);
    acc[q][J20 + 0] = fmaf(gx, dv, acc[q][J20 + 0]);
    acc[q][J20 + 1] = fmaf(gy, dv, acc[q][J20 + 1]);
    acc[q][J20 + 2] = fmaf(gz, dv, acc[q][J20 + 2]);
    if (POT) acc[q][PSUM] += mp;
}

// Newtonian loop: every pair is at least h apart and none is a self pair.
template <int KT, int S, int U, bool POT>
__device__ __forceinline__ void far_loop_f(const float4 *__restrict__ sp,
                                           const float4 *__restrict__ sv, const float tx[KT][3],
                                           float acc[KT][kNCPot])
{
#pragma unroll U
    for (int j = 0; j < S; ++j) {
        const float4 p = sp[j];
        const float4 v = sv[j];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            float dx = p.x - tx[q][0], dy = p.y - tx[q][1], dz = p.z - tx[q][2];
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float ri = rsqrt_sfu(r2);
            float ri2 = ri * ri;
            float mp = p.w * ri;
            float mf = mp * ri2;
            float mg = mf * ri2;
            accumulate_f<KT, POT>(acc, q, dx, dy, dz, v.x, v.y, v.z, mf, mg, mp);
        }
    }
}

// Paired layout, Newtonian loop: two sources per packed FP32x2 instruction
// (fma/add/mul .f32x2), so one issue slot does the work of two pairs; the
// SFU rsqrt runs per source.  Lane 0 sums the even sources, lane 1 the odd.
template <int KT, int S, int U, bool POT>
__device__ __forceinline__ void far_loop_pair(const float *__restrict__ tile, const float tx[KT][3],
                                              float2 acc[KT][kNCPot])
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
        const float2 vz = V1[k];
        const float2 vx = make_float2(v0.x, v0.y), vy = make_float2(v0.z, v0.w);
        const float2 m = make_float2(p1.z, p1.w);
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
            const float2 mp = __fmul2_rn(m, ri);
            const float2 mf = __fmul2_rn(mp, ri2);
            const float2 mg = __fmul2_rn(mf, ri2);
            acc[q][A0 + 0] = __ffma2_rn(mf, dx, acc[q][A0 + 0]);
            acc[q][A0 + 1] = __ffma2_rn(mf, dy, acc[q][A0 + 1]);
            acc[q][A0 + 2] = __ffma2_rn(mf, dz, acc[q][A0 + 2]);
            acc[q][J10 + 0] = __ffma2_rn(mf, vx, acc[q][J10 + 0]);
            acc[q][J10 + 1] = __ffma2_rn(mf, vy, acc[q][J10 + 1]);
            acc[q][J10 + 2] = __ffma2_rn(mf, vz, acc[q][J10 + 2]);
            float2 dv = __fmul2_rn(dz, vz);
            dv = __ffma2_rn(dy, vy, dv);
            dv = __ffma2_rn(dx, vx, dv);
            const float2 gx = __fmul2_rn(mg, dx), gy = __fmul2_rn(mg, dy), gz = __fmul2_rn(mg, dz);
            acc[q][TXX] = __ffma2_rn(gx, dx, acc[q][TXX]);
            acc[q][TYY] = __ffma2_rn(gy, dy, acc[q][TYY]);
            acc[q][TZZ] = __ffma2_rn(gz, dz, acc[q][TZZ]);
            acc[q][TXY] = __ffma2_rn(gx, dy, acc[q][TXY]);
            acc[q][TXZ] = __ffma2_rn(gx, dz, acc[q][TXZ]);
            acc[q][TYZ] = __ffma2_rn(gy, dz, acc[q][TYZ]);
            acc[q][J20 + 0] = __ffma2_rn(gx, dv, acc[q][J20 + 0]);
            acc[q][J20 + 1] = __ffma2_rn(gy, dv, acc[q][J20 + 1]);
            acc[q][J20 + 2] = __ffma2_rn(gz, dv, acc[q][J20 + 2]);
            if (POT) acc[q][PSUM] = __fadd2_rn(acc[q][PSUM], mp);
        }
    }
}

// ---------------------------------------------------------------------------
// Periodic box (nearest periodic image)
// ---------------------------------------------------------------------------

// Nearest image of an FP64 separation: d - box * rint(d / box).
__device__ __forceinline__ double wrap_d(double d, double box, double box_inv)
{
    return fma(-box, rint(__dmul_rn(d, box_inv)), d);
}

// Nearest image of a pair separation with the image index decided exactly as
// a plain FP64 evaluation decides it: d = x_j - x_i, k = rint(d / box) with a
// correctly rounded division, d - box * k.  The force is discontinuous where
// a component crosses half a box, so the image index is an integer decision
// that both evaluations must take in the same precision.
__device__ __forceinline__ double nearest_image_exact(double xj, double xi, double box)
{
    const double d = __dsub_rn(xj, xi);
    return __dsub_rn(d, __dmul_rn(box, rint(__ddiv_rn(d, box))));
}

// Same decision at the cost of a multiplication: the product d * (1/box) can
// round across a half-integer only when the result lies within a few ulp of
// half a box, so only components beyond `tie` (half a box less 2^-40 box) are
// redone with the division.
__device__ __forceinline__ double nearest_image_d(double xj, double xi, double box,
                                                  double box_inv, double tie)
{
    const double w = wrap_d(xj - xi, box, box_inv);
    return fabs(w) > tie ? nearest_image_exact(xj, xi, box) : w;
}

// Tiles whose FP32 position offsets (from the tile centre, rounded to half
// an ulp) could make a separation wrong by more than about 8e-6 of itself:
// the rounding is at most 2^-24 (|t| + |e|), t the target's offset from the
// tile centre and e the box's half-diagonal, and |t| <= gap + e for a target
// at distance gap from the box, so a separation (>= gap) can lose that much
// only when gap < C (gap + 2e), C = 2^-24 / 8e-6 ~ 1/128, i.e. gap <
// C / (1 - C) times the box's diagonal.  Over a warp the gap between the
// warp's box and the tile's is a lower bound of every target's.  Compact
// tiles meet it only next to the targets; a tile that spans a jump of the
// element order (a core and a distant outskirt in one Morton range) meets it
// wherever its members are.
constexpr float kLooseC = 1.0f / 128.0f;

// Per target and tile of the periodic box: bit 0 when the tile needs the
// general loop (softened pairs, or sources that might not lie within `tie`,
// a little under half a box, of the target's image of the tile centre), bit
// 1 when the tile comes within the target's close radius (rc2, squared; see
// close_radii).  t is the target's wrapped offset from the tile centre.
// Outside the general loop every pair separation is shorter than half a box
// by more than the FP32 rounding of the offsets, so its nearest image is
// unambiguous.  Distances are rounded down (any doubt means "near").
template <int KT>
__device__ __forceinline__ int periodic_class(const float t[KT][3], const int64_t ti[KT],
                                              const TileGeom &g, float h2_up, float tie,
                                              const float rc2[KT])
{
    float e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) e[c] = __fmul_ru(0.5f, __fsub_ru(g.hi[c], g.lo[c]));
    const float e2 = fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2]));
    int cls = 0;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        if (ti[q] < 0) continue;
        float d2 = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float at = fabsf(t[q][c]);
            if (__fadd_ru(at, e[c]) >= tie) cls |= 1;
            const float gap = fmaxf(0.0f, __fsub_rd(at, e[c]));
            d2 = __fmaf_rd(gap, gap, d2);
        }
        if (d2 < h2_up) cls |= 1;
        // the close radius, or the FP32 offsets' reach (kLooseC): with
        // (|t| + |e|)^2 <= 2 (t.t + e.e)
        const float t2 = fmaf(t[q][0], t[q][0], fmaf(t[q][1], t[q][1], t[q][2] * t[q][2]));
        const float loose2 = (2.0f * kLooseC * kLooseC) * (t2 + e2);
        if (d2 < fmaxf(rc2[q], loose2)) cls |= 2;
    }
    return cls;
}

// Squared gap between two outward-rounded boxes (rounded down: any doubt
// means "nearer").
__device__ __forceinline__ float box_gap2(const float blo[3], const float bhi[3], const TileGeom &g)
{
    float d2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(g.lo[c], bhi[c]), __fsub_rd(blo[c], g.hi[c])));
        d2 = __fmaf_rd(gap, gap, d2);
    }
    return d2;
}

// Squared diagonal of a box.
__device__ __forceinline__ float box_diag2(const float lo[3], const float hi[3])
{
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float e = hi[c] - lo[c];
        s = fmaf(e, e, s);
    }
    return s;
}

// Which loop a tile takes for one warp's targets; the force kernels and the
// close-tile kernel decide alike (warp-uniform results).  near: some pair
// may lie inside the softening (in a periodic box: or reach half a box);
// close: the tile is summed by the close loops -- in a periodic box when it
// comes within a target's close radius or the FP32 offsets' reach
// (periodic_class), with open boundaries when it lies inside h of the warp's
// box or within the offsets' reach, gap < C/(1-C) diag_t (kLooseC).
template <int KT, int MODE>
__device__ __forceinline__ void classify_tile(const EvalArgs &a, const TileGeom &g,
                                              const float tx[KT][3], const int64_t ti[KT],
                                              const float blo[3], const float bhi[3],
                                              const float rc2[KT], float h2_tile, bool &near,
                                              bool &close)
{
    close = false;
    if (MODE == kModePeriodic) {
        const int cls = periodic_class<KT>(tx, ti, g, a.h2f_up, a.box_tie_f, rc2);
        close = __any_sync(0xffffffffu, (cls & 2) != 0);
        near = __any_sync(0xffffffffu, (cls & 1) != 0);
    } else if (MODE == kModeSoft) {
        near = tile_is_near(blo, bhi, g, h2_tile);
    } else {
        const float g2 = box_gap2(blo, bhi, g);
        near = !(g2 >= a.h2f_up);
        constexpr float kL = kLooseC / (1.0f - kLooseC);
        close = near || g2 < (kL * kL) * box_diag2(g.lo, g.hi);
    }
}

// The low parts of a target's position offset to a tile's centre (tx the
// high parts, formed the same way: FP64 difference, wrapped in a periodic
// box, rounded once).
__device__ __forceinline__ void target_low_parts(const EvalArgs &a, const TileGeom &g,
                                                 const double x[3], const float tx[3],
                                                 bool periodic, float tl[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d = __dsub_rn(x[c], g.c[c]);
        if (periodic) d = wrap_d(d, a.box, a.box_inv);
        tl[c] = __double2float_rn(__dsub_rn(d, (double)tx[c]));
    }
}

// ---------------------------------------------------------------------------
// Periodic box: the close field of a target.  On a lattice the tidal tensor
// and the jerk of an element are near-cancellations of the pair terms of its
// nearest neighbours (sum_j ||T_ij|| / ||T_i|| reaches 10^3 - 10^4 on the
// pancake lattices), so the FP32 rounding of those few terms, and of long FP32
// running sums of positive terms such as sum m dx^2 / r^5, is amplified that
// much.  Two radii around each target scale with the distance r_own from it
// to the nearest other source of its own tile:
//   - pairs closer than R_p = 2.4 r_own are left out of the FP32 sums, listed,
//     and evaluated in FP64 from the FP64 positions, velocities and masses once
//     the item's tiles are done (at most kCloseList per target; past that a
//     pair stays in the FP32 sums);
//   - tiles whose box comes within R_c = 4.5 r_own of a target of the warp take
//     a close loop, whose FP32 sums run over kCloseRun sources before they
//     enter the compensated carry.
// Everything else keeps the FP32 loops.  The FP64 kernels use R_c only (their
// pair terms are FP64 already; their close tiles are summed in runs too).  A
// target alone in its tile, or with a coincident source there, has no close
// field.
// ---------------------------------------------------------------------------
constexpr int kCloseRun = 32;
constexpr int kCloseList = 64;
constexpr float kCloseRp = 2.4f;
constexpr float kCloseRc = 4.5f;

// One listed pair in FP64 (target i at FP64 position xi, source j != i): the
// pair's contributions to the accumulated sums, in the slots of the mixed
// path (A, J1, J2 with the pair's own relative velocity, E = m f - m g' r^2,
// Tp, and P); in a periodic box the nearest image decided as the FP64
// kernels decide it.
template <bool POT, bool PERIODIC>
__device__ __forceinline__ void close_pair_d(const EvalArgs &a, int64_t i, int64_t j,
                                             const double xi[3], double out[kNCPot])
{
    double d[3], v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d[c] = PERIODIC ? nearest_image_d(a.pos[3 * j + c], xi[c], a.box, a.box_inv, a.box_tie)
                        : a.pos[3 * j + c] - xi[c];
        v[c] = a.vel[3 * j + c] - a.vel[3 * i + c];
    }
    const double m = a.mass[j];
    const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
    double mp, mf, mg;
    if (r2 < a.h * a.h) {
        const double hinv = 1.0 / a.h;
        double F, Gp, P;
        spline_kernel<double>(sqrt(r2) * hinv, F, Gp, P);
        mf = m * F * (hinv * hinv * hinv);
        mg = m * Gp * (hinv * hinv * hinv * hinv * hinv);
        mp = m * P * hinv;
    } else {
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri;
        mp = m * ri;
        mf = mp * ri2;
        mg = mf * ri2;
    }
    const double dv = fma(d[0], v[0], fma(d[1], v[1], d[2] * v[2]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        out[A0 + c] = mf * d[c];
        out[J10 + c] = mf * v[c];
        out[J20 + c] = mg * dv * d[c];
    }
    out[ESUM] = fma(-mg, r2, mf);
    out[TXX] = mg * d[0] * d[0];
    out[TYY] = mg * d[1] * d[1];
    out[TZZ] = mg * d[2] * d[2];
    out[TXY] = mg * d[0] * d[1];
    out[TXZ] = mg * d[0] * d[2];
    out[TYZ] = mg * d[1] * d[2];
    out[PSUM] = POT ? mp : 0.0;
}

// General loop of the periodic box: every pair taken to its nearest image
// (FP32), the cubic spline inside h, the self pair excluded by index.  Reads
// either tile layout one source at a time.  A pair with a component longer
// than `tie` (half a box less 2^-20 box, several times the FP32 rounding of
// the offsets) may be equally near two images up to that rounding; its
// separation is then formed again from the FP64 positions with the image
// decided as an FP64 evaluation decides it (nearest_image_d).  Padding
// sources have m = 0 and never take that branch.
template <int KT, int S, bool POT, bool PAIR>
__device__ __forceinline__ void periodic_loop_f(const float4 *__restrict__ stage,
                                                const float tx[KT][3], const int64_t ti[KT],
                                                int64_t jbase, float h2, float hinv,
                                                const EvalArgs &a, float acc[KT][kNCPot])
{
    const float box = a.box_f, box_inv = a.box_inv_f, tie = a.box_tie_f;
    const float hinv3 = hinv * hinv * hinv;
    const float hinv5 = hinv3 * hinv * hinv;
    const float *tile = reinterpret_cast<const float *>(stage);
#pragma unroll 2
    for (int j = 0; j < S; ++j) {
        float x, y, z, m, vx, vy, vz;
        if (PAIR) {
            const int k = j >> 1, h = j & 1;
            x = tile[4 * k + h];
            y = tile[4 * k + 2 + h];
            z = tile[2 * S + 4 * k + h];
            m = tile[2 * S + 4 * k + 2 + h];
            vx = tile[4 * S + 4 * k + h];
            vy = tile[4 * S + 4 * k + 2 + h];
            vz = tile[6 * S + 2 * k + h];
        } else {
            const float4 p = stage[j], v = stage[S + j];
            x = p.x;
            y = p.y;
            z = p.z;
            m = p.w;
            vx = v.x;
            vy = v.y;
            vz = v.z;
        }
        const int64_t jg = jbase + j;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            float dx = x - tx[q][0], dy = y - tx[q][1], dz = z - tx[q][2];
            dx = fmaf(-box, rintf(dx * box_inv), dx);
            dy = fmaf(-box, rintf(dy * box_inv), dy);
            dz = fmaf(-box, rintf(dz * box_inv), dz);
            if (fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) > tie && m != 0.0f && ti[q] >= 0) {
                const double *pi = a.pos + 3 * ti[q], *pj = a.pos + 3 * jg;
                dx = __double2float_rn(nearest_image_d(pj[0], pi[0], a.box, a.box_inv, a.box_tie));
                dy = __double2float_rn(nearest_image_d(pj[1], pi[1], a.box, a.box_inv, a.box_tie));
                dz = __double2float_rn(nearest_image_d(pj[2], pi[2], a.box, a.box_inv, a.box_tie));
            }
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float ri = rsqrt_sfu(r2);
            float ri2 = ri * ri;
            float mp = m * ri;
            float mf = mp * ri2;
            float mg = mf * ri2;
            if (r2 < h2) {
                float F, Gp, P;
                spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
                mf = m * F * hinv3;
                mg = m * Gp * hinv5;
                mp = m * P * hinv;
                if (jg == ti[q]) {
                    mf = 0.0f;
                    mg = 0.0f;
                    mp = 0.0f;
                }
                acc[q][ESUM] += fmaf(-mg, r2, mf);
            }
            accumulate_f<KT, POT>(acc, q, dx, dy, dz, vx, vy, vz, mf, mg, mp);
        }
    }
}

// Near tiles with open boundaries (inside h of the warp's box, or within the
// FP32 offsets' reach: classify_tile): the softened scalar loop (the cubic
// spline inside h, the self pair excluded) with separations from both
// offsets' low parts, d = (s - t) + (s_lo - t_lo) (lo: the tile's planes of
// low parts; tl: the targets'), good to a few units in the last place of d
// however far the tile centre lies.  Velocities enter relative to the tile's
// velocity centre (the per-tile correction applies), good to about 2^-24 of
// those, which is not enough for a close pair moving with its target (w ~ u,
// |w - u| << |w| + |u|) whose jerk term outweighs the rest of the target's
// sum.  So every pair within 2h of its target (where a single pair can
// dominate: inside the spline's support and just past it) is offered to
// record(q, j) and, when taken, left out of the FP32 sums: it is summed in
// FP64 after the item's tiles, from the FP64 positions and velocities.
template <int KT, int S, bool POT, bool PAIR, typename Record>
__device__ __forceinline__ void near_loop_rec(const float4 *__restrict__ stage,
                                              const float *__restrict__ lo, const float tx[KT][3],
                                              const float tl[KT][3], const int64_t ti[KT],
                                              int64_t jbase, float h2, float hinv,
                                              float acc[KT][kNCPot], Record &record)
{
    const float hinv3 = hinv * hinv * hinv;
    const float hinv5 = hinv3 * hinv * hinv;
    const float *tile = reinterpret_cast<const float *>(stage);
#pragma unroll 4
    for (int j = 0; j < S; ++j) {
        float x, y, z, m, wx, wy, wz;
        if (PAIR) {
            const int k = j >> 1, h = j & 1;
            x = tile[4 * k + h];
            y = tile[4 * k + 2 + h];
            z = tile[2 * S + 4 * k + h];
            m = tile[2 * S + 4 * k + 2 + h];
            wx = tile[4 * S + 4 * k + h];
            wy = tile[4 * S + 4 * k + 2 + h];
            wz = tile[6 * S + 2 * k + h];
        } else {
            const float4 p = stage[j], v = stage[S + j];
            x = p.x;
            y = p.y;
            z = p.z;
            m = p.w;
            wx = v.x;
            wy = v.y;
            wz = v.z;
        }
        const float xl = lo[j], yl = lo[S + j], zl = lo[2 * S + j];
        const int64_t jg = jbase + j;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float dx = (x - tx[q][0]) + (xl - tl[q][0]);
            const float dy = (y - tx[q][1]) + (yl - tl[q][1]);
            const float dz = (z - tx[q][2]) + (zl - tl[q][2]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            // (inactive lanes, ti < 0, may record too: their lists are never
            // evaluated; padding sources lie far away)
            if (r2 < 4.0f * h2 && jg != ti[q] && record(q, jg)) continue;
            const float ri = rsqrt_sfu(r2);
            const float ri2 = ri * ri;
            float mp = m * ri;
            float mf = mp * ri2;
            float mg = mf * ri2;
            if (r2 < h2) {
                float F, Gp, P;
                spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
                mf = m * F * hinv3;
                mg = m * Gp * hinv5;
                mp = m * P * hinv;
                if (jg == ti[q]) {
                    mf = 0.0f;
                    mg = 0.0f;
                    mp = 0.0f;
                }
                acc[q][ESUM] += fmaf(-mg, r2, mf);
            }
            accumulate_f<KT, POT>(acc, q, dx, dy, dz, wx, wy, wz, mf, mg, mp);
        }
    }
}

// 1/sqrt(x) refined by one Newton-Raphson step on f(y) = y^-2 - x from the
// SFU estimate y0: y1 = y0 + (y0 / 2) (1 - x y0^2), which roughly halves the
// relative error of y0 (the close loops only: their pair terms feed the
// cancellations described above).
__device__ __forceinline__ float rsqrt_refined(float x)
{
    const float y = rsqrt_sfu(x);
    const float e = fmaf(-(x * y), y, 1.0f);
    return fmaf(0.5f * y, e, y);
}

__device__ __forceinline__ float2 rsqrt_refined2(float2 x)
{
    const float2 y = make_float2(rsqrt_sfu(x.x), rsqrt_sfu(x.y));
    const float2 xy = __fmul2_rn(x, y);
    const float2 e = __ffma2_rn(make_float2(-xy.x, -xy.y), y, make_float2(1.0f, 1.0f));
    return __ffma2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), y), e, y);
}

// Close tiles (see close_radii and the close-tile kernel) that may hold
// softened or self pairs or, in a periodic box, need wrapping: the general
// loop's pair arithmetic (in a periodic box the nearest image in FP32 and the
// FP64 re-formation near half a box; the cubic spline inside h; the self
// pair excluded) over runs of RUN sources, each run's FP32 sums handed to
// carry(acc) (the per-tile target-velocity correction and the compensated
// carry).  Separations take the low parts of both offsets, d = (s - t) +
// (s_lo - t_lo) (lo: the tile's planes of low parts; tl: the targets'),
// good to a few units in the last place of d however far the tile centre
// lies.  A pair
// closer than R_p (squared: rp2; periodic box only) is offered to
// record(q, j), which lists it for the FP64 close field and returns true, or
// returns false when the list is full and the pair stays in the FP32 sums.
template <int KT, int S, int RUN, bool POT, bool PAIR, bool PERIODIC, typename Carry,
          typename Record>
__device__ __forceinline__ void close_loop_f(const float4 *__restrict__ stage,
                                             const float *__restrict__ lo, const float tx[KT][3],
                                             const float tl[KT][3], const int64_t ti[KT],
                                             int64_t jbase, float h2, float hinv,
                                             const float rp2[KT], const EvalArgs &a, Carry &carry,
                                             Record &record)
{
    const float box = a.box_f, box_inv = a.box_inv_f, tie = a.box_tie_f;
    const float hinv3 = hinv * hinv * hinv;
    const float hinv5 = hinv3 * hinv * hinv;
    const float *tile = reinterpret_cast<const float *>(stage);
#pragma unroll 1
    for (int j0 = 0; j0 < S; j0 += RUN) {
        float acc[KT][kNCPot];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) acc[q][c] = 0.0f;
#pragma unroll 2
        for (int j = j0; j < j0 + RUN; ++j) {
            float x, y, z, m, wx, wy, wz;
            if (PAIR) {
                const int k = j >> 1, h = j & 1;
                x = tile[4 * k + h];
                y = tile[4 * k + 2 + h];
                z = tile[2 * S + 4 * k + h];
                m = tile[2 * S + 4 * k + 2 + h];
                wx = tile[4 * S + 4 * k + h];
                wy = tile[4 * S + 4 * k + 2 + h];
                wz = tile[6 * S + 2 * k + h];
            } else {
                const float4 p = stage[j], v = stage[S + j];
                x = p.x;
                y = p.y;
                z = p.z;
                m = p.w;
                wx = v.x;
                wy = v.y;
                wz = v.z;
            }
            const int64_t jg = jbase + j;
            const float xl = lo[j], yl = lo[S + j], zl = lo[2 * S + j];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                float dx = x - tx[q][0], dy = y - tx[q][1], dz = z - tx[q][2];
                float lx = xl - tl[q][0], ly = yl - tl[q][1], lz = zl - tl[q][2];
                if (PERIODIC) {
                    const float kx = rintf(dx * box_inv), ky = rintf(dy * box_inv),
                                kz = rintf(dz * box_inv);
                    dx = fmaf(-box, kx, dx);
                    dy = fmaf(-box, ky, dy);
                    dz = fmaf(-box, kz, dz);
                    lx = fmaf(-a.box_lo_f, kx, lx);
                    ly = fmaf(-a.box_lo_f, ky, ly);
                    lz = fmaf(-a.box_lo_f, kz, lz);
                }
                dx += lx;
                dy += ly;
                dz += lz;
                if (PERIODIC && fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) > tie && m != 0.0f &&
                    ti[q] >= 0) {
                    const double *pi = a.pos + 3 * ti[q], *pj = a.pos + 3 * jg;
                    dx = __double2float_rn(nearest_image_d(pj[0], pi[0], a.box, a.box_inv, a.box_tie));
                    dy = __double2float_rn(nearest_image_d(pj[1], pi[1], a.box, a.box_inv, a.box_tie));
                    dz = __double2float_rn(nearest_image_d(pj[2], pi[2], a.box, a.box_inv, a.box_tie));
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (PERIODIC && r2 < rp2[q] && jg != ti[q] && m != 0.0f && record(q, jg)) continue;
                const float ri = rsqrt_refined(r2);
                const float ri2 = ri * ri;
                float mp = m * ri;
                float mf = mp * ri2;
                float mg = mf * ri2;
                if (r2 < h2) {
                    float F, Gp, P;
                    spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
                    mf = m * F * hinv3;
                    mg = m * Gp * hinv5;
                    mp = m * P * hinv;
                    if (jg == ti[q]) {
                        mf = 0.0f;
                        mg = 0.0f;
                        mp = 0.0f;
                    }
                    acc[q][ESUM] += fmaf(-mg, r2, mf);
                }
                accumulate_f<KT, POT>(acc, q, dx, dy, dz, wx, wy, wz, mf, mg, mp);
            }
        }
        carry(acc);
    }
}

// Sums of one pair of sources (FP32x2 lanes) for one target: A, J1', J2',
// Tp (and P), as in far_loop_pair.
template <bool POT>
__device__ __forceinline__ void accumulate_pair(float2 acc[kNCPot], float2 dx, float2 dy, float2 dz,
                                                float2 vx, float2 vy, float2 vz, float2 mf,
                                                float2 mg, float2 mp)
{
    acc[A0 + 0] = __ffma2_rn(mf, dx, acc[A0 + 0]);
    acc[A0 + 1] = __ffma2_rn(mf, dy, acc[A0 + 1]);
    acc[A0 + 2] = __ffma2_rn(mf, dz, acc[A0 + 2]);
    acc[J10 + 0] = __ffma2_rn(mf, vx, acc[J10 + 0]);
    acc[J10 + 1] = __ffma2_rn(mf, vy, acc[J10 + 1]);
    acc[J10 + 2] = __ffma2_rn(mf, vz, acc[J10 + 2]);
    float2 dv = __fmul2_rn(dz, vz);
    dv = __ffma2_rn(dy, vy, dv);
    dv = __ffma2_rn(dx, vx, dv);
    const float2 gx = __fmul2_rn(mg, dx), gy = __fmul2_rn(mg, dy), gz = __fmul2_rn(mg, dz);
    acc[TXX] = __ffma2_rn(gx, dx, acc[TXX]);
    acc[TYY] = __ffma2_rn(gy, dy, acc[TYY]);
    acc[TZZ] = __ffma2_rn(gz, dz, acc[TZZ]);
    acc[TXY] = __ffma2_rn(gx, dy, acc[TXY]);
    acc[TXZ] = __ffma2_rn(gx, dz, acc[TXZ]);
    acc[TYZ] = __ffma2_rn(gy, dz, acc[TYZ]);
    acc[J20 + 0] = __ffma2_rn(gx, dv, acc[J20 + 0]);
    acc[J20 + 1] = __ffma2_rn(gy, dv, acc[J20 + 1]);
    acc[J20 + 2] = __ffma2_rn(gz, dv, acc[J20 + 2]);
    if (POT) acc[PSUM] = __fadd2_rn(acc[PSUM], mp);
}

// Close tiles of the periodic box that need no wrapping and hold no softened
// or self pair (no target of the warp flags the tile in bit 0 of
// periodic_class): the paired loop of far_loop_pair with separations from
// both offsets' low parts (as in close_loop_f), pairs closer than R_p offered
// to record(q, j) and left out of the sums when it takes them, and the sums
// carried every RUN sources.
template <int KT, int S, int RUN, bool POT, typename Carry, typename Record>
__device__ __forceinline__ void close_loop_pair(const float *__restrict__ tile,
                                                const float *__restrict__ lo, const float tx[KT][3],
                                                const float tl[KT][3], int64_t jbase,
                                                const float rp2[KT], Carry &carry, Record &record)
{
    const float4 *P0 = reinterpret_cast<const float4 *>(tile);
    const float4 *P1 = P0 + S / 2;
    const float4 *V0 = P1 + S / 2;
    const float2 *V1 = reinterpret_cast<const float2 *>(V0 + S / 2);
    const float2 *L2 = reinterpret_cast<const float2 *>(lo);      // 3 planes of S/2 pairs
#pragma unroll 1
    for (int k0 = 0; k0 < S / 2; k0 += RUN / 2) {
        float2 acc2[KT][kNCPot];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) acc2[q][c] = make_float2(0.0f, 0.0f);
#pragma unroll 2
        for (int k = k0; k < k0 + RUN / 2; ++k) {
            const float4 p0 = P0[k], p1 = P1[k], v0 = V0[k];
            const float2 vz = V1[k];
            const float2 vx = make_float2(v0.x, v0.y), vy = make_float2(v0.z, v0.w);
            const float2 lx = L2[k], ly = L2[S / 2 + k], lz = L2[S + k];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(p0.x, p0.y), make_float2(-tx[q][0], -tx[q][0])),
                                             __fadd2_rn(lx, make_float2(-tl[q][0], -tl[q][0])));
                const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(p0.z, p0.w), make_float2(-tx[q][1], -tx[q][1])),
                                             __fadd2_rn(ly, make_float2(-tl[q][1], -tl[q][1])));
                const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(p1.x, p1.y), make_float2(-tx[q][2], -tx[q][2])),
                                             __fadd2_rn(lz, make_float2(-tl[q][2], -tl[q][2])));
                float2 r2 = __fmul2_rn(dz, dz);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dx, dx, r2);
                float2 m = make_float2(p1.z, p1.w);
                if (r2.x < rp2[q] && m.x != 0.0f && record(q, jbase + 2 * k)) m.x = 0.0f;
                if (r2.y < rp2[q] && m.y != 0.0f && record(q, jbase + 2 * k + 1)) m.y = 0.0f;
                const float2 ri = rsqrt_refined2(r2);
                const float2 ri2 = __fmul2_rn(ri, ri);
                const float2 mp = __fmul2_rn(m, ri);
                const float2 mf = __fmul2_rn(mp, ri2);
                const float2 mg = __fmul2_rn(mf, ri2);
                accumulate_pair<POT>(acc2[q], dx, dy, dz, vx, vy, vz, mf, mg, mp);
            }
        }
        float acc[KT][kNCPot];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) acc[q][c] = acc2[q][c].x + acc2[q][c].y;
        carry(acc);
    }
}

// ---------------------------------------------------------------------------
// Adaptive softening: per-element supports (Section 3's fully adaptive
// softening) with the energy-conserving correction term of Price & Monaghan
// (2007).  A pair takes the mean of the kernels of support h_i (target) and
// h_j (source); the acceleration gains
//   -(1/2) m_j [zeta_i W_r(r, h_i) + zeta_j W_r(r, h_j)] d / r,
// W_r = dW/dr, zeta the per-element coefficient from the support solve.  The
// jerk and tidal sums use the averaged kernels at fixed supports.
// ---------------------------------------------------------------------------

// One side of a pair: force, g' and potential kernels of support 1/hinv at
// separation r (Newtonian from ri beyond the support) and W_r.
template <typename T>
__device__ __forceinline__ void soft_side(T r, T ri, T hinv, T &f, T &gp, T &p, T &wr)
{
    const T u = r * hinv;
    if (u < T(1)) {
        T F, Gp, P;
        spline_kernel<T>(u, F, Gp, P);
        const T h2 = hinv * hinv;
        const T h3 = h2 * hinv;
        f = F * h3;
        gp = Gp * h3 * h2;
        p = P * hinv;
        const T q = T(1) - u;
        const T dw = (u < T(0.5)) ? u * (T(-12) + T(18) * u) : T(-6) * q * q;
        wr = T(8.0 / 3.14159265358979323846) * (h2 * h2) * dw;
    } else {
        const T ri2 = ri * ri;
        f = ri * ri2;
        gp = f * ri2;
        p = ri;
        wr = T(0);
    }
}

// Near tiles with per-element supports (mixed path).  hz: the tile's
// (1/h_j, zeta_j) in shared memory; thinv, tzeta: the targets' 1/h_i, zeta_i.
// Reads either tile layout one source at a time.
template <int KT, int S, bool POT, bool PAIR>
__device__ __forceinline__ void soft_loop_f(const float4 *__restrict__ stage,
                                            const float2 *__restrict__ hz, const float tx[KT][3],
                                            const int64_t ti[KT], int64_t jbase,
                                            const float thinv[KT], const float tzeta[KT],
                                            float acc[KT][kNCPot])
{
    const float *tile = reinterpret_cast<const float *>(stage);
#pragma unroll 1
    for (int j = 0; j < S; ++j) {
        float x, y, z, m, vx, vy, vz;
        if (PAIR) {
            const int k = j >> 1, h = j & 1;
            x = tile[4 * k + h];
            y = tile[4 * k + 2 + h];
            z = tile[2 * S + 4 * k + h];
            m = tile[2 * S + 4 * k + 2 + h];
            vx = tile[4 * S + 4 * k + h];
            vy = tile[4 * S + 4 * k + 2 + h];
            vz = tile[6 * S + 2 * k + h];
        } else {
            const float4 p = stage[j], v = stage[S + j];
            x = p.x;
            y = p.y;
            z = p.z;
            m = p.w;
            vx = v.x;
            vy = v.y;
            vz = v.z;
        }
        const float2 sh = hz[j];
        const int64_t jg = jbase + j;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float dx = x - tx[q][0], dy = y - tx[q][1], dz = z - tx[q][2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_sfu(r2);
            const float ri2 = ri * ri;
            float mp = m * ri;
            float mf = mp * ri2;
            float mg = mf * ri2;
            if (r2 * (thinv[q] * thinv[q]) < 1.0f || r2 * (sh.x * sh.x) < 1.0f) {
                const float r = sqrtf(r2);
                float fi, gi, pi, wi, fj, gj, pj, wj;
                soft_side<float>(r, ri, thinv[q], fi, gi, pi, wi);
                soft_side<float>(r, ri, sh.x, fj, gj, pj, wj);
                const float hm = 0.5f * m;
                mf = hm * (fi + fj);
                mg = hm * (gi + gj);
                mp = hm * (pi + pj);
                float ca = r > 0.0f ? -hm * fmaf(tzeta[q], wi, sh.y * wj) / r : 0.0f;
                if (jg == ti[q]) {
                    mf = 0.0f;
                    mg = 0.0f;
                    mp = 0.0f;
                    ca = 0.0f;
                }
                acc[q][ESUM] += fmaf(-mg, r2, mf);
                acc[q][A0 + 0] = fmaf(ca, dx, acc[q][A0 + 0]);
                acc[q][A0 + 1] = fmaf(ca, dy, acc[q][A0 + 1]);
                acc[q][A0 + 2] = fmaf(ca, dz, acc[q][A0 + 2]);
            }
            accumulate_f<KT, POT>(acc, q, dx, dy, dz, vx, vy, vz, mf, mg, mp);
        }
    }
}

// ---------------------------------------------------------------------------
// Pair loops, FP64
// ---------------------------------------------------------------------------

template <bool POT>
__device__ __forceinline__ void accumulate_d(double acc[kNCPot], double dx, double dy, double dz,
                                             double ux, double uy, double uz, double mf, double mg,
                                             double mp)
{
    acc[A0 + 0] = fma(mf, dx, acc[A0 + 0]);
    acc[A0 + 1] = fma(mf, dy, acc[A0 + 1]);
    acc[A0 + 2] = fma(mf, dz, acc[A0 + 2]);
    acc[FSUM] += mf;
    double dv = fma(dx, ux, fma(dy, uy, dz * uz));
    acc[J10 + 0] = fma(mf, ux, acc[J10 + 0]);
    acc[J10 + 1] = fma(mf, uy, acc[J10 + 1]);
    acc[J10 + 2] = fma(mf, uz, acc[J10 + 2]);
    double gx = mg * dx, gy = mg * dy, gz = mg * dz;
    acc[TXX] = fma(gx, dx, acc[TXX]);
    acc[TYY] = fma(gy, dy, acc[TYY]);
    acc[TZZ] = fma(gz, dz, acc[TZZ]);
    acc[TXY] = fma(gx, dy, acc[TXY]);
    acc[TXZ] = fma(gx, dz, acc[TXZ]);
    acc[TYZ] = fma(gy, dz, acc[TYZ]);
    acc[J20 + 0] = fma(gx, dv, acc[J20 + 0]);
    acc[J20 + 1] = fma(gy, dv, acc[J20 + 1]);
    acc[J20 + 2] = fma(gz, dv, acc[J20 + 2]);
    if (POT) acc[PSUM] += mp;
}

// FP64 pair loop.  Source velocities are stored relative to the tile's
// velocity centre and the target's enters per tile (f64_item): the sums take
// the source velocity v_j' alone, J1 = sum m f v_j' and J2 = sum m g' (d.v_j') d.
template <int S, bool POT, bool NEAR, bool PERIODIC = false>
__device__ __forceinline__ void loop_d(const D4 *__restrict__ sp, const D4 *__restrict__ sv,
                                       const double xi[3], int64_t ti,
                                       int64_t jbase, double h2, double hinv,
                                       double acc[kNCPot], double box = 0.0, double box_inv = 0.0,
                                       double tie = 0.0)
{
    const double hinv3 = hinv * hinv * hinv;
    const double hinv5 = hinv3 * hinv * hinv;
#pragma unroll 4
    for (int j = 0; j < S; ++j) {
        const D4 p = sp[j];
        const D4 v = sv[j];
        double dx, dy, dz;
        if (PERIODIC) {
            dx = nearest_image_d(p.x, xi[0], box, box_inv, tie);
            dy = nearest_image_d(p.y, xi[1], box, box_inv, tie);
            dz = nearest_image_d(p.z, xi[2], box, box_inv, tie);
        } else {
            dx = p.x - xi[0];
            dy = p.y - xi[1];
            dz = p.z - xi[2];
        }
        double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        double ri = rsqrt(r2);
        double ri2 = ri * ri;
        double mp = p.w * ri;
        double mf = mp * ri2;
        double mg = mf * ri2;
        if (NEAR && r2 < h2) {
            double F, Gp, P;
            spline_kernel<double>(sqrt(r2) * hinv, F, Gp, P);
            mf = p.w * F * hinv3;
            mg = p.w * Gp * hinv5;
            mp = p.w * P * hinv;
            if (jbase + j == ti) {
                mf = 0.0;
                mg = 0.0;
                mp = 0.0;
            }
        }
        accumulate_d<POT>(acc, dx, dy, dz, v.x, v.y, v.z, mf, mg, mp);
    }
}

// The target's velocity in the sums of one tile (v_i' relative to the tile's
// velocity centre): J1 -= F v_i', J2 -= Tp v_i' (with v = v_j' - v_i' the
// pair sums J1 = sum m f v and J2 = sum m g' (d.v) d split exactly so).
__device__ __forceinline__ void target_velocity_d(double acc[kNCPot], const double u[3])
{
    const double f = acc[FSUM];
    const double t0 = fma(acc[TXX], u[0], fma(acc[TXY], u[1], acc[TXZ] * u[2]));
    const double t1 = fma(acc[TXY], u[0], fma(acc[TYY], u[1], acc[TYZ] * u[2]));
    const double t2 = fma(acc[TXZ], u[0], fma(acc[TYZ], u[1], acc[TZZ] * u[2]));
    acc[J10 + 0] = fma(-u[0], f, acc[J10 + 0]);
    acc[J10 + 1] = fma(-u[1], f, acc[J10 + 1]);
    acc[J10 + 2] = fma(-u[2], f, acc[J10 + 2]);
    acc[J20 + 0] -= t0;
    acc[J20 + 1] -= t1;
    acc[J20 + 2] -= t2;
}


// Near tiles with per-element supports (FP64 path): the source supports and
// coefficients are read from the caller's arrays (padding sources, j >= n_src,
// have m = 0 and take h = 1, zeta = 0).
template <int S, bool POT>
__device__ __forceinline__ void soft_loop_d(const D4 *__restrict__ sp, const D4 *__restrict__ sv,
                                            const double xi[3], const double vi[3], int64_t ti,
                                            int64_t jbase, double hinv_i, double zeta_i,
                                            const EvalArgs &a, double acc[kNCPot])
{
    const double h2i = 1.0 / (hinv_i * hinv_i);
#pragma unroll 1
    for (int j = 0; j < S; ++j) {
        const D4 p = sp[j];
        const D4 v = sv[j];
        const int64_t jg = jbase + j;
        const bool real = jg < a.n_src;
        const double hj = real ? a.h_elem[jg] : 1.0;
        const double zj = (real && a.zeta) ? a.zeta[jg] : 0.0;
        const double dx = p.x - xi[0], dy = p.y - xi[1], dz = p.z - xi[2];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri;
        double mp = p.w * ri;
        double mf = mp * ri2;
        double mg = mf * ri2;
        double ca = 0.0;
        if (r2 < h2i || r2 < hj * hj) {
            const double r = sqrt(r2);
            double fi, gi, pi, wi, fj, gj, pj, wj;
            soft_side<double>(r, ri, hinv_i, fi, gi, pi, wi);
            soft_side<double>(r, ri, 1.0 / hj, fj, gj, pj, wj);
            const double hm = 0.5 * p.w;
            mf = hm * (fi + fj);
            mg = hm * (gi + gj);
            mp = hm * (pi + pj);
            ca = r > 0.0 ? -hm * fma(zeta_i, wi, zj * wj) / r : 0.0;
            if (jg == ti) {
                mf = 0.0;
                mg = 0.0;
                mp = 0.0;
                ca = 0.0;
            }
        }
        accumulate_d<POT>(acc, dx, dy, dz, v.x - vi[0], v.y - vi[1], v.z - vi[2], mf, mg, mp);
        acc[A0 + 0] = fma(ca, dx, acc[A0 + 0]);
        acc[A0 + 1] = fma(ca, dy, acc[A0 + 1]);
        acc[A0 + 2] = fma(ca, dz, acc[A0 + 2]);
    }
}

// Largest value over the block (every thread passes one; all get the result).
template <int NT>
__device__ __forceinline__ float block_max(float v)
{
    __shared__ float wmax[NT / 32];
    __shared__ float result;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = wmax[0];
        for (int w = 1; w < NT / 32; ++w) m = fmaxf(m, wmax[w]);
        result = m;
    }
    __syncthreads();
    return result;
}


// ---------------------------------------------------------------------------
// Shared pieces of both eval kernels
// ---------------------------------------------------------------------------

// Writes one target's chunk partial (FP64) into column `slot` of the split's
// partial block: part[(sp*NC + c) * rows + slot].
template <int NC>
__device__ __forceinline__ void write_partial(const EvalArgs &a, int sp, int64_t rows, int64_t slot,
                                              const double s[kNCPot])
{
#pragma unroll
    for (int c = 0; c < NC; ++c) a.part[((int64_t)sp * NC + c) * rows + slot] = s[c];
}

// ---------------------------------------------------------------------------
// Work items.  One item is the targets idx[slot], slot in
// [slot0, min(slot0 + BT, slot_end)) (slot itself when idx is NULL), against
// the source tiles [t_begin, t_end).  Its sums go to the outputs when
// split == 1, else to column `slot` of chunk `sp`'s partial block.  Targets
// outside [elem_lo, elem_hi) are flagged and skipped.
// ---------------------------------------------------------------------------

struct ItemSpec {
    const int32_t *idx;
    int64_t slot0, slot_end;
    int64_t elem_lo, elem_hi;   // the targets' system: elements [elem_lo, elem_hi)
    int32_t t_begin, t_end;
    int32_t sp, split;
    int64_t rows;
    int32_t tile0;              // the system's first tile (holds element elem_lo)
    int32_t pad;
};

// TMA ring state of a CTA, carried from item to item.
struct Ring {
    uint32_t parity;   // bit s: parity of stage s's next completion
    uint32_t pending;  // thread 0 only: bit s while a copy is in flight into stage s
};

__device__ __forceinline__ int64_t item_target(const ItemSpec &it, int64_t slot, int32_t *flags)
{
    if (slot >= it.slot_end) return -1;
    int64_t i = it.idx ? (int64_t)it.idx[slot] : slot;
    if (i < it.elem_lo || i >= it.elem_hi) {
        flag_or(flags, GRAV_FLAG_BADINDEX);
        return -1;
    }
    return i;
}

// Squared radii R_p^2 and R_c^2 of target i (element of the item's system, at
// FP64 position xi) from r_own^2, found over the packed sources of its own
// tile: mixed tiles (FP32 offsets from the tile centre, paired or float4
// layout) in FP32, FP64 tiles in FP64; separations wrapped to the nearest
// image.  -1 (no close field) when the tile holds no other source or a
// coincident one.
template <int S, bool MIXED, bool PAIR>
__device__ __forceinline__ void close_radii(const EvalArgs &a, const ItemSpec &it, int64_t i,
                                            const double xi[3], float &rp2, float &rc2)
{
    const int64_t k = (i - it.elem_lo) / S;
    const int32_t t = it.tile0 + (int32_t)k;
    const int self = (int)(i - (it.elem_lo + k * S));
    float r2min = __int_as_float(0x7f800000);
    if (MIXED) {
        const TileGeom &g = a.geo[t];
        float to[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) to[c] = __double2float_rn(__dsub_rn(xi[c], g.c[c]));
        const float *tile = static_cast<const float *>(a.src) + (int64_t)t * 8 * S;
        const float4 *t4 = static_cast<const float4 *>(a.src) + (int64_t)t * 2 * S;
#pragma unroll 4
        for (int j = 0; j < S; ++j) {
            float x, y, z, m;
            if (PAIR) {
                const int kk = j >> 1, h = j & 1;
                x = tile[4 * kk + h];
                y = tile[4 * kk + 2 + h];
                z = tile[2 * S + 4 * kk + h];
                m = tile[2 * S + 4 * kk + 2 + h];
            } else {
                const float4 p = t4[j];
                x = p.x;
                y = p.y;
                z = p.z;
                m = p.w;
            }
            float dx = x - to[0], dy = y - to[1], dz = z - to[2];
            dx = fmaf(-a.box_f, rintf(dx * a.box_inv_f), dx);
            dy = fmaf(-a.box_f, rintf(dy * a.box_inv_f), dy);
            dz = fmaf(-a.box_f, rintf(dz * a.box_inv_f), dz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (j != self && m != 0.0f) r2min = fminf(r2min, r2);
        }
    } else {
        const D4 *tile = static_cast<const D4 *>(a.src) + (int64_t)t * 2 * S;
        double m2 = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll 4
        for (int j = 0; j < S; ++j) {
            const D4 p = tile[j];
            const double dx = wrap_d(p.x - xi[0], a.box, a.box_inv);
            const double dy = wrap_d(p.y - xi[1], a.box, a.box_inv);
            const double dz = wrap_d(p.z - xi[2], a.box, a.box_inv);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (j != self && p.w != 0.0) m2 = fmin(m2, r2);
        }
        r2min = __double2float_rn(m2);
    }
    if (!(r2min > 0.0f) || isinf(r2min)) {
        rp2 = -1.0f;
        rc2 = -1.0f;
        return;
    }
    rp2 = (kCloseRp * kCloseRp) * r2min;
    rc2 = (kCloseRc * kCloseRc) * r2min;
}

// Never leave a copy in flight into shared memory (only after a timeout).
template <int NSTAGE>
__device__ __forceinline__ void drain_ring(uint64_t *bar, const Ring &ring, int32_t *flags)
{
    if (threadIdx.x == 0 && ring.pending) {
        for (int s = 0; s < NSTAGE; ++s)
            if (ring.pending & (1u << s)) mbar_wait_bounded(&bar[s], (ring.parity >> s) & 1u, flags);
    }
}

// Batched launches: the device-side plan (see grav_eval_batched).
struct BatchHeader {
    int64_t total_items;
    int32_t total_tiles;
    int32_t pad;
    unsigned long long ticket;   // next work item (atomic counter, reset by the plan kernel)
    int64_t pad2;
};

struct BatchView {
    BatchHeader *hdr;
    const grav_system *sys;    // [n_sys] (device)
    int32_t *tile_off;         // [n_sys + 1]
    int32_t *idx_lo, *idx_hi;  // [n_sys]: each system's range of the target list
    int32_t *ntb;              // [n_sys]: target blocks
    int32_t *order;            // [n_sys]: systems, longest work item first
    int64_t *item_off;         // [n_sys + 1]: first work item of each rank
    int32_t n_sys;
    int32_t pad;
};

// A system's softening h in a copy of the launch's arguments, with the
// roundings the host applies to grav_params.h: FP32 h and 1/h to nearest,
// h^2 in FP64 then to FP32 rounded up.
__device__ __forceinline__ void softening_f(double h, float &h2f_up, float &hinvf)
{
    const double h2 = __dmul_rn(h, h);
    float h2f = __double2float_rn(h2);
    if ((double)h2f < h2) h2f = nextafterf(h2f, __int_as_float(0x7f800000));
    h2f_up = h2f;
    hinvf = __double2float_rn(__ddiv_rn(1.0, h));
}

__device__ __forceinline__ void set_softening(EvalArgs &a, double h)
{
    a.h = h;
    a.hf = __double2float_rn(h);
    softening_f(h, a.h2f_up, a.hinvf);
}

// The plan of a batched launch (grav_eval_host.cu): per-system tiles and
// target ranges (idx == NULL: every element of a system is a target), the
// longest-first order of the systems, the work-item offsets; resets the
// ticket.  Systems that are out of range, overlap, or have an h that is
// neither 0 nor finite, positive and (box > 0) under half the box are
// skipped with GRAV_FLAG_BADINDEX.
int launch_batch_plan(const BatchView &b, const int32_t *idx, const int32_t *n_idx_dev,
                      int64_t n_idx_max, int64_t n_total, int32_t S, int32_t BT, double box,
                      int32_t *flags, cudaStream_t st);

// Rank r such that item_off[r] <= ticket < item_off[r + 1].
__device__ __forceinline__ int item_rank(const BatchView &b, int64_t ticket)
{
    int lo = 0, hi = b.n_sys;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (b.item_off[mid] <= ticket)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Batched packing: tile t belongs to the system s with
// tile_off[s] <= t < tile_off[s + 1]; tiles never straddle two systems.
template <int S, bool MIXED, bool VOFF, bool PAIR>
__global__ void __launch_bounds__(S)
pack_tiles_batched_kernel(const BatchView b, const double *__restrict__ pos,
                          const double *__restrict__ vel, const double *__restrict__ mass,
                          TileGeom *__restrict__ geo, void *__restrict__ src, int32_t *flags,
                          float *__restrict__ src_lo)
{
    const int t = blockIdx.x;
    if (t >= b.hdr->total_tiles) return;
    int lo = 0, hi = b.n_sys;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (b.tile_off[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    const int64_t first = b.sys[lo].offset + (int64_t)(t - b.tile_off[lo]) * S;
    const int64_t sys_end = b.sys[lo].offset + b.sys[lo].n;
    const int64_t end = first + S < sys_end ? first + S : sys_end;
    pack_tile<S, MIXED, VOFF, PAIR>(t, first, end, pos, vel, mass, geo, src, flags, src_lo);
}

// ---------------------------------------------------------------------------
// K5: mixed-precision force kernel.  SACC: compensated accumulators and FP64
// target positions live in shared memory (fewer registers, more targets per
// thread); otherwise in registers.
// ---------------------------------------------------------------------------

// The mixed kernels' tile loops synchronise nothing across warps, so each
// warp releases a stage of the source ring on its own (no block barrier per
// tile) and a third stage lets warps drift apart by up to two tiles.
template <int NT, int KT, int S, bool POT, bool SACC, bool PAIR = false, int NST = 3>
struct MixedSmem {
    static constexpr int BT = NT * KT;
    static constexpr int NC = POT ? kNCPot : kNC;
    static constexpr int kStages = NST;
    // a stage: the packed tile (28 or 32 bytes per source), then the low
    // parts of its position offsets (12 bytes per source)
    static constexpr int kTileF4 = PAIR ? 7 * S / 4 : 2 * S;
    static constexpr int kLoF4 = kLoPlanes * S / 4;
    float4 stage[NST][kTileF4 + kLoF4];
    float acc[SACC ? NC * 2 * BT : 1];     // [c][hi, lo][BT]
    double x[SACC ? 3 * BT : 1];           // [c][BT]
    uint64_t bar[NST];
    int done[NST];                         // warps finished with the tile in each stage
    unsigned issued[NST];                  // copies issued into each stage
    float blo[3], bhi[3];
    int abort_flag;
    long long ticket;
};


template <typename Sm>
__device__ __forceinline__ void init_mixed_ring(Sm &sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < Sm::kStages; ++s) {
            mbar_init(&sm.bar[s], 1);
            sm.done[s] = 0;
            sm.issued[s] = 0;
        }
        sm.abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

template <typename Sm>
__device__ __forceinline__ void init_ring(Sm &sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) mbar_init(&sm.bar[s], 1);
        sm.abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
}

// Before a mixed kernel exits: wait (bounded) for any copy still in flight
// into its shared memory.  With per-warp release a copy is outstanding in
// stage s exactly when thread 0 has seen fewer completions there than were
// issued (at most one: a refill needs every warp, thread 0's included, to
// have consumed the previous copy).
template <typename Sm>
__device__ __forceinline__ void drain_mixed_ring(Sm &sm, const Ring &ring, int32_t *flags)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < Sm::kStages; ++s)
            if ((sm.issued[s] & 1u) != ((ring.parity >> s) & 1u))
                mbar_wait_bounded(&sm.bar[s], (ring.parity >> s) & 1u, flags);
    }
}

// One work item of the mixed kernel; false if a bounded wait gave up.
template <int NT, int KT, int S, int U, bool POT, bool SACC, bool PAIR, int MODE>
__device__ __forceinline__ bool mixed_item(
    const EvalArgs &a, MixedSmem<NT, KT, S, POT, SACC, PAIR> &sm, Ring &ring,
    const ItemSpec &it)
{
    using Sm = MixedSmem<NT, KT, S, POT, SACC, PAIR>;
    constexpr int BT = Sm::BT;
    constexpr int NSTAGE = Sm::kStages;
    constexpr int NC = Sm::NC;
    constexpr bool soft = MODE == kModeSoft;
    constexpr uint32_t kTileBytes = PAIR ? S * 28 : S * 2 * sizeof(float4);
    const float4 *src = static_cast<const float4 *>(a.src);
    const int t_begin = it.t_begin, t_end = it.t_end;

    // ---- targets of this item (KT per thread, strided by NT) ----
    double xr[SACC ? 1 : KT][3];
    float tvf[KT][3];
    int64_t ti[KT];
    float lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = __int_as_float(0x7f800000);
        hi[c] = -__int_as_float(0x7f800000);
    }
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        const int64_t i = item_target(it, it.slot0 + (int64_t)q * NT + threadIdx.x, a.flags);
        ti[q] = i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double x = 0.0;
            tvf[q][c] = 0.0f;
            if (i >= 0) {
                x = a.pos[3 * i + c];
                tvf[q][c] = __double2float_rn(a.vel[3 * i + c]);
                lo[c] = fminf(lo[c], __double2float_rd(x));
                hi[c] = fmaxf(hi[c], __double2float_ru(x));
            }
            if (SACC)
                sm.x[c * BT + q * NT + threadIdx.x] = x;
            else
                xr[SACC ? 0 : q][c] = x;
        }
    }
    block_bbox<NT>(lo, hi, sm.blo, sm.bhi);     // (its barriers also publish sm.x)
    // each warp takes the near/far test of a tile against its own targets'
    // box (lo/hi now hold it): far more tiles are culled than with the
    // block's box when the targets are sparse
    const float blo_r[3] = {lo[0], lo[1], lo[2]};
    const float bhi_r[3] = {hi[0], hi[1], hi[2]};

    // adaptive softening: the targets' 1/h_i and zeta_i, the warp's largest
    // support
    float thinv[soft ? KT : 1], tzeta[soft ? KT : 1];
    float h_block = 0.0f;
    if (soft) {
        float hb = 0.0f;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            thinv[soft ? q : 0] = 1.0f;
            tzeta[soft ? q : 0] = 0.0f;
            if (ti[q] >= 0) {
                const double h = a.h_elem[ti[q]];
                thinv[soft ? q : 0] = __double2float_rn(1.0 / h);
                tzeta[soft ? q : 0] = a.zeta ? __double2float_rn(a.zeta[ti[q]]) : 0.0f;
                hb = fmaxf(hb, __double2float_ru(h));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hb = fmaxf(hb, __shfl_xor_sync(0xffffffffu, hb, o));
        h_block = hb;
    }

    float rhi[SACC ? 1 : KT][SACC ? 1 : kNCPot], rlo[SACC ? 1 : KT][SACC ? 1 : kNCPot];
    if (SACC) {
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < 2 * NC; ++c) sm.acc[c * BT + q * NT + threadIdx.x] = 0.0f;
    } else {
#pragma unroll
        for (int q = 0; q < (SACC ? 1 : KT); ++q)
#pragma unroll
            for (int c = 0; c < (SACC ? 1 : kNCPot); ++c) {
                rhi[q][c] = 0.0f;
                rlo[q][c] = 0.0f;
            }
    }

    // a tile and, when packed, the low parts of its offsets, into stage s
    auto load_stage = [&](int s, int t) {
        if (a.src_lo)
            tma_load_1d_two(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes,
                            sm.stage[s] + Sm::kTileF4, a.src_lo + (int64_t)t * kLoPlanes * S,
                            4u * kLoPlanes * S, &sm.bar[s]);
        else
            tma_load_1d(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes, &sm.bar[s]);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            int t = t_begin + s;
            if (t < t_end) {
                load_stage(s, t);
                sm.issued[s] += 1u;
            }
        }
    }

    // periodic box: the close-field radii of each target (close_radii)
    constexpr bool periodic = MODE == kModePeriodic;
    float rp2[KT], rc2[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        rp2[q] = -1.0f;
        rc2[q] = -1.0f;
        if (periodic && ti[q] >= 0) {
            double x3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                x3[c] = SACC ? sm.x[c * BT + q * NT + threadIdx.x] : xr[SACC ? 0 : q][c];
            close_radii<S, true, PAIR>(a, it, ti[q], x3, rp2[q], rc2[q]);
        }
    }

    // the target velocity in one tile's FP32 sums: J1 -= v_i' F, J2 -= Tp v_i'
    // (v_i' relative to the tile's velocity centre; not for the close loops,
    // whose sums take each pair's own relative velocity); then the
    // compensated carry
    TileGeom g = a.geo[t_begin];
    auto carry_any = [&](float (&acc)[KT][kNCPot], bool correct) {
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (correct) {
                const float ux = tvf[q][0] - g.cv[0], uy = tvf[q][1] - g.cv[1], uz = tvf[q][2] - g.cv[2];
                const float Ft = acc[q][ESUM] + (acc[q][TXX] + acc[q][TYY] + acc[q][TZZ]);
                acc[q][J10 + 0] = fmaf(-ux, Ft, acc[q][J10 + 0]);
                acc[q][J10 + 1] = fmaf(-uy, Ft, acc[q][J10 + 1]);
                acc[q][J10 + 2] = fmaf(-uz, Ft, acc[q][J10 + 2]);
                acc[q][J20 + 0] -= fmaf(acc[q][TXX], ux, fmaf(acc[q][TXY], uy, acc[q][TXZ] * uz));
                acc[q][J20 + 1] -= fmaf(acc[q][TXY], ux, fmaf(acc[q][TYY], uy, acc[q][TYZ] * uz));
                acc[q][J20 + 2] -= fmaf(acc[q][TXZ], ux, fmaf(acc[q][TYZ], uy, acc[q][TZZ] * uz));
            }
            if (SACC) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float *ph = &sm.acc[(2 * c) * BT + q * NT + threadIdx.x];
                    float *pl = &sm.acc[(2 * c + 1) * BT + q * NT + threadIdx.x];
                    float h = *ph, l = *pl;
                    two_sum_acc(h, l, acc[q][c]);
                    *ph = h;
                    *pl = l;
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    two_sum_acc(rhi[SACC ? 0 : q][SACC ? 0 : c], rlo[SACC ? 0 : q][SACC ? 0 : c],
                                acc[q][c]);
            }
        }
    };
    auto carry_tile = [&](float (&acc)[KT][kNCPot]) { carry_any(acc, true); };
    // the pairs listed for FP64 (periodic: each target's close field; open
    // boundaries: the pairs within 2h), evaluated once the item's tiles are
    // done
    constexpr bool listed = !soft;
    int32_t nlist[KT][listed ? kCloseList : 1];
    int ncnt[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) ncnt[q] = 0;
    auto record = [&](int q, int64_t j) -> bool {
        if (ncnt[q] >= kCloseList) return false;
        nlist[q][ncnt[q]++] = (int32_t)j;
        return true;
    };
    // periodic: the FP64 close field of each target, summed in FP64 and added
    // to its final sums
    double nsum[listed ? KT : 1][listed ? kNCPot : 1];
    if constexpr (listed) {
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) nsum[q][c] = 0.0;
    }

    // offsets of the targets to a tile's centre (FP64, rounded once); in a
    // periodic box, to the image of the centre nearest to the target
    auto offsets = [&](const TileGeom &g, float out[KT][3]) {
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double x = SACC ? sm.x[c * BT + q * NT + threadIdx.x] : xr[SACC ? 0 : q][c];
                double d = __dsub_rn(x, g.c[c]);
                if (periodic) d = wrap_d(d, a.box, a.box_inv);
                out[q][c] = __double2float_rn(d);
            }
    };
    float tx[KT][3], tx_next[KT][3];
    offsets(g, tx);

    for (int t = t_begin; t < t_end; ++t) {
        const int s = (t - t_begin) % NSTAGE;
        // periodic: any target near the tile, or a tile that may reach past
        // half a box from a target's image of it, takes the general loop
        float h2_tile = a.h2f_up;
        if (soft) {
            const float hm = fmaxf(h_block, a.geo_h[t]);
            h2_tile = __fmul_ru(hm, hm);
        }
        bool near, close;
        classify_tile<KT, MODE>(a, g, tx, ti, blo_r, bhi_r, rc2, h2_tile, near, close);
        // next tile's geometry and offsets, computed ahead (FP64 latency)
        TileGeom gn = g;
        if (t + 1 < t_end) {
            gn = a.geo[t + 1];
            offsets(gn, tx_next);
        }
        const bool got = mbar_wait_bounded(&sm.bar[s], (ring.parity >> s) & 1u, a.flags);
        if (got)
            ring.parity ^= 1u << s;
        else
            atomicExch(&sm.abort_flag, 1);

        float acc[KT][kNCPot];
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) acc[q][c] = 0.0f;
        if (close && periodic) {
            // the targets' low parts for this tile; runs of the close loops
            // carry their own sums (acc stays zero)
            float tl[KT][3];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                double x[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    x[c] = SACC ? sm.x[c * BT + q * NT + threadIdx.x] : xr[SACC ? 0 : q][c];
                target_low_parts(a, g, x, tx[q], true, tl[q]);
            }
            const float *lo = reinterpret_cast<const float *>(sm.stage[s] + Sm::kTileF4);
            // (tiles that may need wrapping take the scalar loop)
            if (PAIR && !near)
                close_loop_pair<KT, S, kCloseRun, POT>(reinterpret_cast<const float *>(sm.stage[s]), lo,
                                                       tx, tl, g.first, rp2, carry_tile, record);
            else
                close_loop_f<KT, S, kCloseRun, POT, PAIR, true>(sm.stage[s], lo, tx, tl, ti, g.first,
                                                                a.h2f_up, a.hinvf, rp2, a, carry_tile,
                                                                record);
        } else if (close) {
            // open boundaries: near tiles, separations from the low parts
            // too, pairs within 2h listed for FP64
            float tl[KT][3];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                double x[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    x[c] = SACC ? sm.x[c * BT + q * NT + threadIdx.x] : xr[SACC ? 0 : q][c];
                target_low_parts(a, g, x, tx[q], false, tl[q]);
            }
            near_loop_rec<KT, S, POT, PAIR>(sm.stage[s],
                                            reinterpret_cast<const float *>(sm.stage[s] + Sm::kTileF4),
                                            tx, tl, ti, g.first, a.h2f_up, a.hinvf, acc, record);
        } else if (soft && near) {
            // the tile's (1/h_j, zeta_j) straight from global memory (every
            // lane reads the same source: one cached load per warp)
            soft_loop_f<KT, S, POT, PAIR>(sm.stage[s], a.hz + (int64_t)t * S, tx, ti, g.first, thinv,
                                          tzeta, acc);
        } else if (periodic && near) {
            periodic_loop_f<KT, S, POT, PAIR>(sm.stage[s], tx, ti, g.first, a.h2f_up, a.hinvf, a,
                                              acc);
        } else if (PAIR) {
            float2 acc2[KT][kNCPot];
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNCPot; ++c) acc2[q][c] = make_float2(0.0f, 0.0f);
            far_loop_pair<KT, S, U, POT>(reinterpret_cast<const float *>(sm.stage[s]), tx, acc2);
#pragma unroll
            for (int q = 0; q < KT; ++q)
#pragma unroll
                for (int c = 0; c < kNCPot; ++c) acc[q][c] = acc2[q][c].x + acc2[q][c].y;
        } else {
            far_loop_f<KT, S, U, POT>(sm.stage[s], sm.stage[s] + S, tx, acc);
        }

        // per-tile corrections for the target velocity, then the carry
        if (!(close && periodic)) carry_tile(acc);

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
        g = gn;
#pragma unroll
        for (int q = 0; q < KT; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) tx[q][c] = tx_next[q][c];
    }

    // the listed pairs in FP64 (each lane its own list; an inactive lane's
    // list is skipped)
    if constexpr (listed) {
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (ti[q] < 0) continue;
            double xi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                xi[c] = SACC ? sm.x[c * BT + q * NT + threadIdx.x] : xr[SACC ? 0 : q][c];
            for (int k = 0; k < ncnt[q]; ++k) {
                double v[kNCPot];
                close_pair_d<POT, periodic>(a, ti[q], nlist[q][k], xi, v);
#pragma unroll
                for (int c = 0; c < kNCPot; ++c) nsum[q][c] += v[c];
            }
        }
    }

    // warps may leave the tile loop at different tiles: meet here so that
    // every thread returns the same status
    __syncthreads();

    // ---- results ----
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        double sum[kNCPot];
#pragma unroll
        for (int c = 0; c < kNCPot; ++c) {
            if (c >= NC) {
                sum[c] = 0.0;
            } else if (SACC) {
                sum[c] = __dadd_rn((double)sm.acc[(2 * c) * BT + q * NT + threadIdx.x],
                                   (double)sm.acc[(2 * c + 1) * BT + q * NT + threadIdx.x]);
            } else {
                sum[c] = __dadd_rn((double)rhi[SACC ? 0 : q][SACC ? 0 : c],
                                   (double)rlo[SACC ? 0 : q][SACC ? 0 : c]);
            }
            if constexpr (listed) {
                if (c < NC) sum[c] = __dadd_rn(sum[c], nsum[q][c]);
            }
        }
        if (it.split == 1) {
            if (ti[q] >= 0) write_target<POT, true>(a, ti[q], sum);
        } else {
            write_partial<NC>(a, it.sp, it.rows, it.slot0 + (int64_t)q * NT + threadIdx.x, sum);
        }
    }
    return !sm.abort_flag;
}

template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
__global__ void __launch_bounds__(NT, MINB)
eval_mixed_kernel(const EvalArgs a)
{
    using Sm = MixedSmem<NT, KT, S, POT, SACC, PAIR>;
    constexpr int BT = Sm::BT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    init_mixed_ring(sm);
    Ring ring{0u, 0u};
    const int64_t n_act = active_count(a);
    const int64_t n_tb = (n_act + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    const int64_t items = n_tb * split;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        ItemSpec it;
        it.idx = a.idx;
        it.slot0 = tb * BT;
        it.slot_end = n_act;
        it.elem_lo = 0;
        it.elem_hi = a.n_src;
        it.t_begin = (int)((int64_t)sp * a.n_tiles / split);
        it.t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);
        it.sp = sp;
        it.split = split;
        it.rows = n_tb * BT;
        it.tile0 = 0;
        it.pad = 0;
        if (!mixed_item<NT, KT, S, U, POT, SACC, PAIR, MODE>(a, sm, ring, it)) break;
        __syncthreads();
    }
    drain_mixed_ring(sm, ring, a.flags);
}

// Batched: items of all systems from the plan, taken through an atomic
// ticket (no waiting on other CTAs).  Each target is summed by one CTA over
// its system's tiles in a fixed order, so results do not depend on which CTA
// takes which item.
template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
__global__ void __launch_bounds__(NT, MINB)
eval_mixed_batched_kernel(const EvalArgs a, const BatchView b)
{
    using Sm = MixedSmem<NT, KT, S, POT, SACC, PAIR>;
    constexpr int BT = Sm::BT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    __shared__ EvalArgs sa;   // the launch's arguments with the item's system's softening
    if (threadIdx.x == 0) sa = a;
    init_mixed_ring(sm);
    Ring ring{0u, 0u};
    const int64_t total = b.hdr->total_items;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long tk = (long long)atomicAdd(&b.hdr->ticket, 1ULL);
            sm.ticket = tk;
            if (tk < total) {
                const double hs = b.sys[b.order[item_rank(b, tk)]].h;
                set_softening(sa, hs > 0.0 ? hs : a.h);
            }
        }
        __syncthreads();
        const int64_t ticket = sm.ticket;
        __syncthreads();
        if (ticket >= total) break;
        const int r = item_rank(b, ticket);
        const int s = b.order[r];
        ItemSpec it;
        it.idx = a.idx;
        it.slot0 = (int64_t)b.idx_lo[s] + (ticket - b.item_off[r]) * BT;
        it.slot_end = b.idx_hi[s];
        it.elem_lo = b.sys[s].offset;
        it.elem_hi = b.sys[s].offset + b.sys[s].n;
        it.t_begin = b.tile_off[s];
        it.t_end = b.tile_off[s + 1];
        it.sp = 0;
        it.split = 1;
        it.rows = 0;
        it.tile0 = b.tile_off[s];
        it.pad = 0;
        if (!mixed_item<NT, KT, S, U, POT, SACC, PAIR, MODE>(sa, sm, ring, it)) break;
        __syncthreads();
    }
    drain_mixed_ring(sm, ring, a.flags);
}

// ---------------------------------------------------------------------------
// K4: FP64 force kernel (one target per thread)
// ---------------------------------------------------------------------------

template <int S>
struct F64Smem {
    D4 stage[2][2 * S];
    uint64_t bar[2];
    float blo[3], bhi[3];
    int abort_flag;
    long long ticket;
};

template <int NT, int S, bool POT, int MODE>
__device__ __forceinline__ bool f64_item(const EvalArgs &a, F64Smem<S> &sm, Ring &ring,
                                         const ItemSpec &it)
{
    constexpr int NSTAGE = 2;
    constexpr int NC = POT ? kNCPot : kNC;
    constexpr uint32_t kTileBytes = S * 2 * sizeof(D4);
    const D4 *src = static_cast<const D4 *>(a.src);
    const double h2 = a.h * a.h;
    const double hinv = 1.0 / a.h;
    const int t_begin = it.t_begin, t_end = it.t_end;

    const int64_t i = item_target(it, it.slot0 + threadIdx.x, a.flags);
    double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0};
    float lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = __int_as_float(0x7f800000);
        hi[c] = -__int_as_float(0x7f800000);
        if (i >= 0) {
            xi[c] = a.pos[3 * i + c];
            vi[c] = a.vel[3 * i + c];
            lo[c] = __double2float_rd(xi[c]);
            hi[c] = __double2float_ru(xi[c]);
        }
    }
    block_bbox<NT>(lo, hi, sm.blo, sm.bhi);
    // open boundaries: each warp tests tiles against its own targets' box
    // (lo/hi now hold it; the near and far loops synchronise nothing)
    constexpr bool kWarpBox = MODE == kModeOpen;
    const float blo_r[3] = {kWarpBox ? lo[0] : sm.blo[0], kWarpBox ? lo[1] : sm.blo[1],
                            kWarpBox ? lo[2] : sm.blo[2]};
    const float bhi_r[3] = {kWarpBox ? hi[0] : sm.bhi[0], kWarpBox ? hi[1] : sm.bhi[1],
                            kWarpBox ? hi[2] : sm.bhi[2]};
    // periodic box: the target's close radius (close_radii; the FP64 pair
    // terms need no FP64 close field, only the runs)
    float rc2[1] = {-1.0f};
    if (MODE == kModePeriodic && i >= 0) {
        float rp2;
        close_radii<S, false, false>(a, it, i, xi, rp2, rc2[0]);
    }
    double hinv_i = 1.0, zeta_i = 0.0;
    float h_block = 0.0f;
    if (MODE == kModeSoft) {
        float hb = 0.0f;
        if (i >= 0) {
            const double h = a.h_elem[i];
            hinv_i = 1.0 / h;
            zeta_i = a.zeta ? a.zeta[i] : 0.0;
            hb = __double2float_ru(h);
        }
        h_block = block_max<NT>(hb);
    }

    double shi[kNCPot], slo[kNCPot];
#pragma unroll
    for (int c = 0; c < kNCPot; ++c) {
        shi[c] = 0.0;
        slo[c] = 0.0;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            int t = t_begin + s;
            if (t < t_end) {
                tma_load_1d(sm.stage[s], src + (int64_t)t * 2 * S, kTileBytes, &sm.bar[s]);
                ring.pending |= 1u << s;
            }
        }
    }
    constexpr bool periodic = MODE == kModePeriodic;
    constexpr bool soft = MODE == kModeSoft;
    for (int t = t_begin; t < t_end; ++t) {
        const int s = (t - t_begin) % NSTAGE;
        const TileGeom g = a.geo[t];
        bool near, close = false;
        if (periodic) {
            float tw[1][3];
            const int64_t ti1[1] = {i};
#pragma unroll
            for (int c = 0; c < 3; ++c)
                tw[0][c] = __double2float_rn(wrap_d(__dsub_rn(xi[c], g.c[c]), a.box, a.box_inv));
            // every FP64 periodic pair is wrapped; this decides softening and
            // the close tiles (summed in runs)
            const int cls = periodic_class<1>(tw, ti1, g, a.h2f_up, a.box_tie_f, rc2);
            close = __syncthreads_or((cls & 2) != 0) != 0;
            near = close || __syncthreads_or((cls & 1) != 0) != 0;
        } else if (soft) {
            const float hm = fmaxf(h_block, a.geo_h[t]);
            near = tile_is_near(blo_r, bhi_r, g, __fmul_ru(hm, hm));
        } else {
            near = tile_is_near(blo_r, bhi_r, g, a.h2f_up);
        }
        const bool got = mbar_wait_bounded(&sm.bar[s], (ring.parity >> s) & 1u, a.flags);
        if (got)
            ring.parity ^= 1u << s;
        else
            atomicExch(&sm.abort_flag, 1);
        double acc[kNCPot];
#pragma unroll
        for (int c = 0; c < kNCPot; ++c) acc[c] = 0.0;
        // the target's velocity relative to the tile's velocity centre (the
        // tile stores its sources' velocities relative to it)
        const double vr[3] = {vi[0] - (double)g.cv[0], vi[1] - (double)g.cv[1],
                              vi[2] - (double)g.cv[2]};
        if (soft && near) {
            soft_loop_d<S, POT>(sm.stage[s], sm.stage[s] + S, xi, vr, i, g.first, hinv_i, zeta_i, a,
                                acc);
        } else if (periodic && close) {
            // close tiles: runs of kCloseRun sources, each carried on its own
            // (acc stays zero)
            for (int j0 = 0; j0 < S; j0 += kCloseRun) {
                double racc[kNCPot];
#pragma unroll
                for (int c = 0; c < kNCPot; ++c) racc[c] = 0.0;
                loop_d<kCloseRun, POT, true, true>(sm.stage[s] + j0, sm.stage[s] + S + j0, xi, i,
                                                   g.first + j0, h2, hinv, racc, a.box, a.box_inv,
                                                   a.box_tie);
                target_velocity_d(racc, vr);
#pragma unroll
                for (int c = 0; c < NC; ++c) two_sum_acc(shi[c], slo[c], racc[c]);
            }
        } else {
            if (periodic && !near)
                loop_d<S, POT, false, true>(sm.stage[s], sm.stage[s] + S, xi, i, g.first, h2, hinv,
                                            acc, a.box, a.box_inv, a.box_tie);
            else if (periodic)
                loop_d<S, POT, true, true>(sm.stage[s], sm.stage[s] + S, xi, i, g.first, h2, hinv,
                                           acc, a.box, a.box_inv, a.box_tie);
            else if (!near)
                loop_d<S, POT, false>(sm.stage[s], sm.stage[s] + S, xi, i, g.first, h2, hinv, acc);
            else
                loop_d<S, POT, true>(sm.stage[s], sm.stage[s] + S, xi, i, g.first, h2, hinv, acc);
            target_velocity_d(acc, vr);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) two_sum_acc(shi[c], slo[c], acc[c]);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (got) ring.pending &= ~(1u << s);
            if (t + NSTAGE < t_end && !sm.abort_flag) {
                tma_load_1d(sm.stage[s], src + (int64_t)(t + NSTAGE) * 2 * S, kTileBytes, &sm.bar[s]);
                ring.pending |= 1u << s;
            }
        }
        if (sm.abort_flag) break;
    }
    double sum[kNCPot];
#pragma unroll
    for (int c = 0; c < kNCPot; ++c) sum[c] = __dadd_rn(shi[c], slo[c]);
    if (it.split == 1) {
        if (i >= 0) write_target<POT, false>(a, i, sum);
    } else {
        write_partial<NC>(a, it.sp, it.rows, it.slot0 + threadIdx.x, sum);
    }
    return !sm.abort_flag;
}

template <int NT, int S, bool POT, int MODE>
__global__ void __launch_bounds__(NT, 2)
eval_f64_kernel(const EvalArgs a)
{
    __shared__ __align__(128) F64Smem<S> sm;
    init_ring(sm);
    Ring ring{0u, 0u};
    const int64_t n_act = active_count(a);
    const int64_t n_tb = (n_act + NT - 1) / NT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, NT);
    const int64_t items = n_tb * split;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t tb = item / split;
        const int sp = (int)(item - tb * split);
        ItemSpec it;
        it.idx = a.idx;
        it.slot0 = tb * NT;
        it.slot_end = n_act;
        it.elem_lo = 0;
        it.elem_hi = a.n_src;
        it.t_begin = (int)((int64_t)sp * a.n_tiles / split);
        it.t_end = (int)((int64_t)(sp + 1) * a.n_tiles / split);
        it.sp = sp;
        it.split = split;
        it.rows = n_tb * NT;
        it.tile0 = 0;
        it.pad = 0;
        if (!f64_item<NT, S, POT, MODE>(a, sm, ring, it)) break;
        __syncthreads();
    }
    drain_ring<2>(sm.bar, ring, a.flags);
}

template <int NT, int S, bool POT, int MODE>
__global__ void __launch_bounds__(NT, 2)
eval_f64_batched_kernel(const EvalArgs a, const BatchView b)
{
    __shared__ __align__(128) F64Smem<S> sm;
    __shared__ EvalArgs sa;   // the launch's arguments with the item's system's softening
    if (threadIdx.x == 0) sa = a;
    init_ring(sm);
    Ring ring{0u, 0u};
    const int64_t total = b.hdr->total_items;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long tk = (long long)atomicAdd(&b.hdr->ticket, 1ULL);
            sm.ticket = tk;
            if (tk < total) {
                const double hs = b.sys[b.order[item_rank(b, tk)]].h;
                set_softening(sa, hs > 0.0 ? hs : a.h);
            }
        }
        __syncthreads();
        const int64_t ticket = sm.ticket;
        __syncthreads();
        if (ticket >= total) break;
        const int r = item_rank(b, ticket);
        const int s = b.order[r];
        ItemSpec it;
        it.idx = a.idx;
        it.slot0 = (int64_t)b.idx_lo[s] + (ticket - b.item_off[r]) * NT;
        it.slot_end = b.idx_hi[s];
        it.elem_lo = b.sys[s].offset;
        it.elem_hi = b.sys[s].offset + b.sys[s].n;
        it.t_begin = b.tile_off[s];
        it.t_end = b.tile_off[s + 1];
        it.sp = 0;
        it.split = 1;
        it.rows = 0;
        it.tile0 = b.tile_off[s];
        it.pad = 0;
        if (!f64_item<NT, S, POT, MODE>(sa, sm, ring, it)) break;
        __syncthreads();
    }
    drain_ring<2>(sm.bar, ring, a.flags);
}

// ---------------------------------------------------------------------------
// K9: deterministic reduction of the chunk partials (fixed chunk order)
// ---------------------------------------------------------------------------

// Threads of the split reduction: one per (target, accumulated component),
// so that a small target set (the usual case of a split) still spreads its
// FP64 work -- `split` TwoSums per component, at 1/74 of the FP32 rate on
// GB300 -- over many warps instead of queueing it on a few.
constexpr int kReduceThreads = 256;
template <bool POT>
constexpr int reduce_targets_per_block() { return kReduceThreads / (POT ? kNCPot : kNC); }

template <bool POT, bool ETRACE>
__global__ void __launch_bounds__(kReduceThreads)
reduce_partials_kernel(const EvalArgs a, int32_t BT)
{
    constexpr int NC = POT ? kNCPot : kNC;
    constexpr int TPB = reduce_targets_per_block<POT>();
    __shared__ double red[NC][TPB];
    const int64_t n_act = active_count(a);
    const int64_t n_tb = (n_act + BT - 1) / BT;
    const int split = choose_split(n_tb, a.n_tiles, a.grid, a.max_split, a.part_cap_rows, BT);
    if (split <= 1) return;
    const int64_t rows = n_tb * BT;
    const int k = threadIdx.x % TPB, c = threadIdx.x / TPB;
    // a bounded grid strides over groups of TPB targets (the count is known
    // on the device only, so the host sizes the grid for the upper bound)
    for (int64_t slot0 = (int64_t)blockIdx.x * TPB; slot0 < n_act;
         slot0 += (int64_t)gridDim.x * TPB) {
        const int64_t slot = slot0 + k;
        if (c < NC && slot < n_act) {
            // the chunk partials of component c of this target, in split order
            double hi = 0.0, lo = 0.0;
            for (int sp = 0; sp < split; ++sp)
                two_sum_acc(hi, lo, a.part[((int64_t)sp * NC + c) * rows + slot]);
            red[c][k] = __dadd_rn(hi, lo);
        }
        __syncthreads();
        if (threadIdx.x < TPB && slot0 + threadIdx.x < n_act) {
            const int64_t sl = slot0 + threadIdx.x;
            const int64_t i = a.idx ? (int64_t)a.idx[sl] : sl;
            if (i >= 0 && i < a.n_src) {
                double sum[kNCPot];
#pragma unroll
                for (int q = 0; q < kNCPot; ++q) sum[q] = q < NC ? red[q][threadIdx.x] : 0.0;
                write_target<POT, ETRACE>(a, i, sum);
            }
        }
        __syncthreads();                             // red is reused by the next group
    }
}

// ---------------------------------------------------------------------------
// Launch table
// ---------------------------------------------------------------------------

typedef void (*eval_launch_fn)(const EvalArgs &, int grid, cudaStream_t);
typedef int (*occupancy_fn)(int *blocks_per_sm);
typedef void (*pack_launch_fn)(int64_t n_src, const double *, const double *, const double *,
                               TileGeom *, void *, int32_t *, float *src_lo, int n_tiles,
                               cudaStream_t);

typedef void (*batched_launch_fn)(const EvalArgs &, const BatchView &, int grid, cudaStream_t);
typedef void (*batched_pack_fn)(const BatchView &, const double *, const double *, const double *,
                                TileGeom *, void *, int32_t *, float *src_lo, int max_tiles,
                                cudaStream_t);

// Upper bound on the tile configurations of one precision (host caches).
constexpr int kMaxTileConfigs = 32;

struct EvalConfig {
    int32_t precision;
    int32_t threads, kt, s, unroll, sacc;
    eval_launch_fn launch[3][2];   // [mode][want_pot]
    occupancy_fn occupancy[3][2];
    pack_launch_fn pack;
    batched_launch_fn launch_batched[2][2];   // [mode: open, periodic][want_pot]
    occupancy_fn occupancy_batched[2][2];
    batched_pack_fn pack_batched;
    bool paired;                   // mixed source tiles in the paired (FP32x2) layout
};

template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
void launch_mixed(const EvalArgs &a, int grid, cudaStream_t st)
{
    constexpr size_t bytes = sizeof(MixedSmem<NT, KT, S, POT, SACC, PAIR>);
    eval_mixed_kernel<NT, KT, S, MINB, U, POT, SACC, PAIR, MODE><<<grid, NT, bytes, st>>>(a);
}

template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
int occupancy_mixed(int *b)
{
    constexpr size_t bytes = sizeof(MixedSmem<NT, KT, S, POT, SACC, PAIR>);
    auto k = eval_mixed_kernel<NT, KT, S, MINB, U, POT, SACC, PAIR, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k, NT, bytes);
}

template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
void launch_mixed_batched(const EvalArgs &a, const BatchView &b, int grid, cudaStream_t st)
{
    constexpr size_t bytes = sizeof(MixedSmem<NT, KT, S, POT, SACC, PAIR>);
    eval_mixed_batched_kernel<NT, KT, S, MINB, U, POT, SACC, PAIR, MODE><<<grid, NT, bytes, st>>>(a, b);
}

template <int NT, int KT, int S, int MINB, int U, bool POT, bool SACC, bool PAIR, int MODE>
int occupancy_mixed_batched(int *b)
{
    constexpr size_t bytes = sizeof(MixedSmem<NT, KT, S, POT, SACC, PAIR>);
    auto k = eval_mixed_batched_kernel<NT, KT, S, MINB, U, POT, SACC, PAIR, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k, NT, bytes);
}

template <int NT, int S, bool POT, int MODE>
void launch_f64_batched(const EvalArgs &a, const BatchView &b, int grid, cudaStream_t st)
{
    eval_f64_batched_kernel<NT, S, POT, MODE><<<grid, NT, 0, st>>>(a, b);
}

template <int NT, int S, bool POT, int MODE>
int occupancy_f64_batched(int *b)
{
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, eval_f64_batched_kernel<NT, S, POT, MODE>, NT, 0);
}

template <int S, bool MIXED, bool VOFF, bool PAIR>
void launch_pack_batched(const BatchView &b, const double *pos, const double *vel, const double *mass,
                         TileGeom *geo, void *src, int32_t *flags, float *src_lo, int max_tiles,
                         cudaStream_t st)
{
    pack_tiles_batched_kernel<S, MIXED, VOFF, PAIR><<<max_tiles, S, 0, st>>>(b, pos, vel, mass, geo, src,
                                                                            flags, src_lo);
}

template <int NT, int S, bool POT, int MODE>
void launch_f64(const EvalArgs &a, int grid, cudaStream_t st)
{
    eval_f64_kernel<NT, S, POT, MODE><<<grid, NT, 0, st>>>(a);
}

template <int NT, int S, bool POT, int MODE>
int occupancy_f64(int *b)
{
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, eval_f64_kernel<NT, S, POT, MODE>, NT, 0);
}

template <int S, bool MIXED, bool VOFF, bool PAIR>
void launch_pack(int64_t n_src, const double *pos, const double *vel, const double *mass,
                 TileGeom *geo, void *src, int32_t *flags, float *src_lo, int n_tiles, cudaStream_t st)
{
    pack_tiles_kernel<S, MIXED, VOFF, PAIR><<<n_tiles, S, 0, st>>>(n_src, pos, vel, mass, geo, src, flags,
                                                                  src_lo);
}

// Defined in the per-precision translation units.
const EvalConfig *mixed_configs(int *count);

const EvalConfig *f64_configs(int *count);
void launch_reduce(const EvalArgs &a, int32_t BT, bool pot, bool etrace, int64_t n_targets,
                   cudaStream_t st);

}  // namespace grav
