// Oct-tree solver (Section 3: the tree code with the Barnes & Hut geometric
// opening criterion, a node of side L always split when L/r > Theta, and
// optionally the relative criterion it supplements).
//
// The tree and every decision in it are defined so that an FP64 evaluation
// on any machine builds the same tree and takes the same branches:
//   - root: the cube of side ext (largest extent of the elements' bounding
//     box) at its low corner; cell coordinates q_c = floor((x_c - lo_c) / ext
//     * 2^21) clamped to [0, 2^21 - 1]; 63-bit keys interleaving x, y, z from
//     the highest bit down;
//   - order: elements sorted by (key, index) -- a stable LSD radix sort of
//     the keys over the index order (16 passes of 4 bits);
//   - nodes: a node at level l holds the run of elements that share the top
//     3l key bits and has side ext 2^-l; it is a leaf when it holds at most
//     leaf_size elements or l = 21, else its non-empty octants are its
//     children, stored contiguously in octant order;
//   - moments: mass, centre of mass and mean velocity, summed in order (a
//     leaf over its elements, a node over its children) with correctly
//     rounded operations;
//   - walk: from the root, a node is accepted when L^2 < Theta^2 r^2 (r from
//     the target to the node's centre of mass, r^2 = (dx^2 + dy^2) + dz^2)
//     and, with alpha > 0 and a_old, also G M L^2 <= (alpha |a_old| r^2) r^2;
//     an accepted node acts as a point mass at its centre of mass moving with
//     its mean velocity, a leaf that is not accepted is summed element by
//     element (j != i), any other node is opened; children in octant order.
// Building: per level, one thread per node finds its octant runs by binary
// search and appends its children with one atomic add (node numbers vary
// from run to run, the tree and the walk order do not); moments bottom-up and
// the "next" links top-down, level by level.  The walk is stackless: after a
// node is accepted or a leaf is summed the walk continues at the node's next
// link (its next sibling, else its parent's next link).  GRAV_F64: pair terms
// as in the FP64 direct kernel, sums compensated every 32 interactions;
// GRAV_MIXED: the same decisions (FP64), pair terms in FP32.
#include <cmath>

#include "grav_eval.cuh"

namespace grav {
namespace {

constexpr int kMaxLevel = 21;
constexpr int kSortNT = 256;
constexpr int kSortPer = 16;                    // items per thread
constexpr int kSortBlock = kSortNT * kSortPer;  // 4096 items per CTA
constexpr int kBins = 16;                       // 4-bit digits
constexpr int kPasses = 16;
constexpr int kBboxBlocks = 1024;
constexpr int kWalkNT = 128;
constexpr int kFlushEvery = 32;

struct TreeView {
    int64_t n;
    int64_t max_nodes;
    int32_t leaf_size;
    uint64_t *key;        // sorted keys (after the sort)
    int32_t *order;       // sorted element indices
    double *frame;        // lo[3], ext
    int32_t *counters;    // [0] nodes, [1 + l] first node of level l (l = 0..23)
    int32_t *first, *count, *child_first, *next;
    int8_t *n_child, *level;
    double *m, *com, *vcom;
    float4 *vcom32;       // mixed walk: node mean velocity in FP32
    float4 *chi, *clo;    // node centre of mass as two FP32 parts (com = chi + clo to 2^-48);
                          // chi.w = m in FP32, clo.w = L^2 (node side squared) in FP32
    float4 *soff;         // mixed walk, per tree position: (x_j - com of its leaf, m_j) in FP32
    float4 *svel;         // mixed walk, per tree position: v_j in FP32
    int32_t *flags;
};

int64_t max_nodes_for(int64_t n, int32_t leaf)
{
    return 2 * n + 22 * (n / (leaf + 1) + 1) + 64;
}

struct TreeLayout {
    int64_t key_a, key_b, val_a, val_b, hist, part, frame, counters;
    int64_t first, count, child_first, next, n_child, level, m, com, vcom, vcom32, chi, clo, soff, svel;
    int64_t total;
    int64_t n_sort_blocks, max_nodes;
};

TreeLayout tree_layout(int64_t n, int32_t leaf)
{
    TreeLayout L;
    const int64_t nb = (n + kSortBlock - 1) / kSortBlock;
    const int64_t mn = max_nodes_for(n, leaf);
    L.n_sort_blocks = nb;
    L.max_nodes = mn;
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        int64_t at = o;
        o += round_up(std::max<int64_t>(bytes, 1), 256);
        return at;
    };
    L.key_a = take(n * 8);
    L.key_b = take(n * 8);
    L.val_a = take(n * 4);
    L.val_b = take(n * 4);
    L.hist = take(nb * kBins * 4);
    L.part = take(kBboxBlocks * 6 * 8);
    L.frame = take(4 * 8);
    L.counters = take(32 * 4);
    L.first = take(mn * 4);
    L.count = take(mn * 4);
    L.child_first = take(mn * 4);
    L.next = take(mn * 4);
    L.n_child = take(mn);
    L.level = take(mn);
    L.m = take(mn * 8);
    L.com = take(mn * 24);
    L.vcom = take(mn * 24);
    L.vcom32 = take(mn * 16);
    L.chi = take(mn * 16);
    L.clo = take(mn * 16);
    L.soff = take(n * 16);
    L.svel = take(n * 16);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// Bounding cube and keys
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) bbox_partial_kernel(int64_t n, const double *__restrict__ pos,
                                                           double *__restrict__ part)
{
    __shared__ double s[6][8];
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        for (int c = 0; c < 3; ++c) {
            const double x = pos[3 * i + c];
            lo[c] = fmin(lo[c], x);
            hi[c] = fmax(hi[c], x);
        }
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) {
            s[c][threadIdx.x >> 5] = lo[c];
            s[3 + c][threadIdx.x >> 5] = hi[c];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[threadIdx.x][0];
        for (int w = 1; w < 8; ++w)
            v = threadIdx.x < 3 ? fmin(v, s[threadIdx.x][w]) : fmax(v, s[threadIdx.x][w]);
        part[(int64_t)blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void bbox_final_kernel(int nb, const double *__restrict__ part, double *__restrict__ frame)
{
    if (threadIdx.x != 0) return;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], part[6 * b + c]);
            hi[c] = fmax(hi[c], part[6 * b + 3 + c]);
        }
    double ext = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double e = __dsub_rn(hi[c], lo[c]);
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0)) ext = 1.0;
    for (int c = 0; c < 3; ++c) frame[c] = lo[c];
    frame[3] = ext;
}

__device__ __forceinline__ uint64_t spread21(uint64_t v)
{
    uint64_t out = 0;
#pragma unroll
    for (int b = 0; b < 21; ++b) out |= ((v >> b) & 1u) << (3 * b);
    return out;
}

__global__ void __launch_bounds__(256) key_kernel(int64_t n, const double *__restrict__ pos,
                                                  const double *__restrict__ frame,
                                                  uint64_t *__restrict__ key, int32_t *__restrict__ val,
                                                  int32_t *flags)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const double ext = frame[3];
    uint64_t q[3];
    for (int c = 0; c < 3; ++c) {
        const double x = pos[3 * i + c];
        if (!isfinite(x)) flag_or(flags, GRAV_FLAG_NONFINITE);
        double s = floor(__dmul_rn(__ddiv_rn(__dsub_rn(x, frame[c]), ext), 2097152.0));
        if (!(s >= 0.0)) s = 0.0;
        if (s > 2097151.0) s = 2097151.0;
        q[c] = (uint64_t)s;
    }
    key[i] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    val[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, index), 4-bit digits
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kSortNT) sort_hist_kernel(int64_t n, const uint64_t *__restrict__ key,
                                                            int shift, int32_t *__restrict__ hist,
                                                            int64_t nb)
{
    __shared__ int32_t cnt[kBins];
    if (threadIdx.x < kBins) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortBlock + (int64_t)threadIdx.x * kSortPer;
    int32_t local[kBins];
#pragma unroll
    for (int d = 0; d < kBins; ++d) local[d] = 0;
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
        const int64_t s = base + k;
        if (s < n) {
            const int d = (int)((key[s] >> shift) & 15u);
#pragma unroll
            for (int e = 0; e < kBins; ++e) local[e] += (d == e);
        }
    }
#pragma unroll
    for (int d = 0; d < kBins; ++d)
        if (local[d]) atomicAdd(&cnt[d], local[d]);
    __syncthreads();
    if (threadIdx.x < kBins) hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan, in place, of hist[0 .. total) (digit-major), one CTA of 1024.
__global__ void __launch_bounds__(1024) sort_scan_kernel(int32_t *__restrict__ hist, int64_t total)
{
    __shared__ int32_t part[1024];
    const int64_t per = (total + 1023) / 1024;
    const int64_t a = threadIdx.x * per;
    const int64_t b = a + per < total ? a + per : total;
    int32_t s = 0;
    for (int64_t k = a; k < b; ++k) s += hist[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int64_t k = a; k < b; ++k) {
        const int32_t v = hist[k];
        hist[k] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kSortNT) sort_scatter_kernel(
    int64_t n, const uint64_t *__restrict__ key_in, const int32_t *__restrict__ val_in,
    uint64_t *__restrict__ key_out, int32_t *__restrict__ val_out, int shift,
    const int32_t *__restrict__ hist, int64_t nb)
{
    __shared__ int32_t cnt[kBins][kSortNT + 1];
    const int64_t base = (int64_t)blockIdx.x * kSortBlock + (int64_t)threadIdx.x * kSortPer;
    int32_t local[kBins];
#pragma unroll
    for (int d = 0; d < kBins; ++d) local[d] = 0;
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
        const int64_t s = base + k;
        if (s < n) {
            const int d = (int)((key_in[s] >> shift) & 15u);
#pragma unroll
            for (int e = 0; e < kBins; ++e) local[e] += (d == e);
        }
    }
#pragma unroll
    for (int d = 0; d < kBins; ++d) cnt[d][threadIdx.x] = local[d];
    __syncthreads();
    if (threadIdx.x < kBins) {                 // exclusive scan over the threads, per digit
        int32_t run = hist[(int64_t)threadIdx.x * nb + blockIdx.x];
        for (int t = 0; t < kSortNT; ++t) {
            const int32_t v = cnt[threadIdx.x][t];
            cnt[threadIdx.x][t] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < kBins; ++d) local[d] = cnt[d][threadIdx.x];
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
        const int64_t s = base + k;
        if (s < n) {
            const uint64_t kk = key_in[s];
            const int d = (int)((kk >> shift) & 15u);
            int32_t at = 0;
#pragma unroll
            for (int e = 0; e < kBins; ++e)
                if (d == e) at = local[e]++;
            key_out[at] = kk;
            val_out[at] = val_in[s];
        }
    }
}

// ---------------------------------------------------------------------------
// Tree levels
// ---------------------------------------------------------------------------

__global__ void tree_init_kernel(TreeView t)
{
    if (threadIdx.x != 0) return;
    t.counters[0] = 1;
    t.counters[1] = 0;   // level 0 starts at node 0
    t.counters[2] = 1;   // level 1 starts at node 1
    t.first[0] = 0;
    t.count[0] = (int32_t)t.n;
    t.level[0] = 0;
    t.child_first[0] = -1;
    t.n_child[0] = 0;
    t.next[0] = -1;
}

// First index in [a, b) whose octant digit is >= o (digits ascend in a run).
__device__ __forceinline__ int32_t digit_bound(const uint64_t *key, int32_t a, int32_t b, int shift,
                                               uint32_t o)
{
    while (a < b) {
        const int32_t mid = a + (b - a) / 2;
        if (((key[mid] >> shift) & 7u) < o)
            a = mid + 1;
        else
            b = mid;
    }
    return a;
}

__global__ void __launch_bounds__(256) tree_split_kernel(TreeView t, int lvl)
{
    const int32_t lb = t.counters[1 + lvl], le = t.counters[2 + lvl];
    for (int32_t k = lb + (int32_t)(blockIdx.x * 256 + threadIdx.x); k < le;
         k += (int32_t)(gridDim.x * 256)) {
        t.child_first[k] = -1;
        t.n_child[k] = 0;
        const int32_t f = t.first[k], c = t.count[k];
        if (c <= t.leaf_size || lvl >= kMaxLevel) continue;
        const int shift = 3 * (20 - lvl);
        int32_t edge[9];
        edge[0] = f;
        edge[8] = f + c;
        for (uint32_t o = 1; o < 8; ++o) edge[o] = digit_bound(t.key, edge[o - 1], f + c, shift, o);
        int nc = 0;
        for (int o = 0; o < 8; ++o) nc += edge[o + 1] > edge[o];
        const int32_t base = atomicAdd(&t.counters[0], nc);
        if ((int64_t)base + nc > t.max_nodes) {
            flag_or(t.flags, GRAV_FLAG_OVERFLOW);
            continue;
        }
        int q = 0;
        for (int o = 0; o < 8; ++o) {
            if (edge[o + 1] == edge[o]) continue;
            const int32_t ch = base + q++;
            t.first[ch] = edge[o];
            t.count[ch] = edge[o + 1] - edge[o];
            t.level[ch] = (int8_t)(lvl + 1);
            t.child_first[ch] = -1;
            t.n_child[ch] = 0;
        }
        t.child_first[k] = base;
        t.n_child[k] = (int8_t)nc;
    }
}

__global__ void tree_mark_kernel(TreeView t, int lvl)
{
    if (threadIdx.x == 0) {
        int64_t n = t.counters[0];
        if (n > t.max_nodes) n = t.max_nodes;
        t.counters[3 + lvl] = (int32_t)n;   // first node of level lvl + 2
    }
}

__global__ void __launch_bounds__(256) tree_moment_kernel(TreeView t, const double *__restrict__ pos,
                                                          const double *__restrict__ vel,
                                                          const double *__restrict__ mass, int lvl)
{
    const int32_t lb = t.counters[1 + lvl], le = t.counters[2 + lvl];
    for (int32_t k = lb + (int32_t)(blockIdx.x * 256 + threadIdx.x); k < le;
         k += (int32_t)(gridDim.x * 256)) {
        double m = 0.0, mx[3] = {0.0, 0.0, 0.0}, mv[3] = {0.0, 0.0, 0.0};
        const int32_t cf = t.child_first[k];
        if (cf < 0) {
            const int32_t f = t.first[k], c = t.count[k];
            for (int32_t s = f; s < f + c; ++s) {
                const int32_t j = t.order[s];
                const double mj = mass[j];
                m = __dadd_rn(m, mj);
                for (int q = 0; q < 3; ++q) {
                    mx[q] = __dadd_rn(mx[q], __dmul_rn(mj, pos[3 * j + q]));
                    mv[q] = __dadd_rn(mv[q], __dmul_rn(mj, vel[3 * j + q]));
                }
            }
        } else {
            const int nc = t.n_child[k];
            for (int q = 0; q < nc; ++q) {
                const int32_t ch = cf + q;
                const double mc = t.m[ch];
                m = __dadd_rn(m, mc);
                for (int e = 0; e < 3; ++e) {
                    mx[e] = __dadd_rn(mx[e], __dmul_rn(mc, t.com[3 * (int64_t)ch + e]));
                    mv[e] = __dadd_rn(mv[e], __dmul_rn(mc, t.vcom[3 * (int64_t)ch + e]));
                }
            }
        }
        t.m[k] = m;
        for (int e = 0; e < 3; ++e) {
            t.com[3 * (int64_t)k + e] = m > 0.0 ? __ddiv_rn(mx[e], m) : 0.0;
            t.vcom[3 * (int64_t)k + e] = m > 0.0 ? __ddiv_rn(mv[e], m) : 0.0;
        }
    }
}

__global__ void __launch_bounds__(256) tree_next_kernel(TreeView t, int lvl)
{
    const int32_t lb = t.counters[1 + lvl], le = t.counters[2 + lvl];
    for (int32_t k = lb + (int32_t)(blockIdx.x * 256 + threadIdx.x); k < le;
         k += (int32_t)(gridDim.x * 256)) {
        const int32_t cf = t.child_first[k];
        const int nc = t.n_child[k];
        for (int q = 0; q < nc; ++q) t.next[cf + q] = (q + 1 < nc) ? cf + q + 1 : t.next[k];
    }
}

// FP32 data of the walk.  Every node: its centre of mass as two FP32 parts
// (hi = com rounded, lo = the remainder rounded), its mass and squared side
// in FP32 (the opening decisions' FP32 bounds), its mean velocity in FP32.
// Mixed walk only, per tree position: the element's offset from its leaf's
// centre of mass (formed in FP64, rounded once), mass and velocity.
__global__ void __launch_bounds__(256) tree_walk_data_kernel(TreeView t, const double *__restrict__ pos,
                                                             const double *__restrict__ vel,
                                                             const double *__restrict__ mass,
                                                             bool mixed)
{
    int64_t nn = t.counters[0];
    if (nn > t.max_nodes) nn = t.max_nodes;
    const double ext = t.frame[3];
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < nn; k += (int64_t)gridDim.x * 256) {
        const double *vc = t.vcom + 3 * k;
        t.vcom32[k] = make_float4(__double2float_rn(vc[0]), __double2float_rn(vc[1]),
                                  __double2float_rn(vc[2]), 0.0f);
        float hi[3], lo[3];
        for (int c = 0; c < 3; ++c) {
            const double x = t.com[3 * k + c];
            hi[c] = __double2float_rn(x);
            lo[c] = __double2float_rn(__dsub_rn(x, (double)hi[c]));
        }
        const double L = scalbn(ext, -(int)t.level[k]);
        t.chi[k] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(t.m[k]));
        t.clo[k] = make_float4(lo[0], lo[1], lo[2], __double2float_rn(__dmul_rn(L, L)));
        if (!mixed || t.child_first[k] >= 0) continue;
        const double *c = t.com + 3 * k;
        const int32_t f = t.first[k], cnt = t.count[k];
        for (int32_t q = f; q < f + cnt; ++q) {
            const int32_t j = t.order[q];
            t.soff[q] = make_float4(__double2float_rn(pos[3 * j] - c[0]),
                                    __double2float_rn(pos[3 * j + 1] - c[1]),
                                    __double2float_rn(pos[3 * j + 2] - c[2]), __double2float_rn(mass[j]));
            t.svel[q] = make_float4(__double2float_rn(vel[3 * j]), __double2float_rn(vel[3 * j + 1]),
                                    __double2float_rn(vel[3 * j + 2]), 0.0f);
        }
    }
}

// ---------------------------------------------------------------------------
// Walk
// ---------------------------------------------------------------------------

struct WalkArgs {
    const double *pos, *vel, *mass, *a_old;
    const int32_t *idx, *n_idx_dev;
    int64_t n_idx_max;
    double h, theta2, alpha;
    long long *stats;
};

__device__ __forceinline__ void pair_d(double acc[kNCPot], double m, double dx, double dy, double dz,
                                       double ux, double uy, double uz, double h2, double hinv,
                                       bool self)
{
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double ri = rsqrt(r2);
    const double ri2 = ri * ri;
    double mp = m * ri;
    double mf = mp * ri2;
    double mg = mf * ri2;
    if (r2 < h2) {
        double F, Gp, P;
        spline_kernel<double>(sqrt(r2) * hinv, F, Gp, P);
        const double hinv3 = hinv * hinv * hinv;
        mf = m * F * hinv3;
        mg = m * Gp * hinv3 * hinv * hinv;
        mp = m * P * hinv;
    }
    if (self) {
        mf = 0.0;
        mg = 0.0;
        mp = 0.0;
    }
    accumulate_d<true>(acc, dx, dy, dz, ux, uy, uz, mf, mg, mp);
}

// The same pair terms in FP32 (mixed walk): A, F, J1, J2, Tp, P.
__device__ __forceinline__ void pair_f(float acc[kNCPot], float m, float dx, float dy, float dz,
                                       float ux, float uy, float uz, float h2, float hinv, bool self)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ri = rsqrt_sfu(r2);
    const float ri2 = ri * ri;
    float mp = m * ri;
    float mf = mp * ri2;
    float mg = mf * ri2;
    if (r2 < h2) {
        float F, Gp, P;
        spline_kernel<float>(sqrtf(r2) * hinv, F, Gp, P);
        const float hinv3 = hinv * hinv * hinv;
        mf = m * F * hinv3;
        mg = m * Gp * hinv3 * hinv * hinv;
        mp = m * P * hinv;
    }
    if (self) {
        mf = 0.0f;
        mg = 0.0f;
        mp = 0.0f;
    }
    acc[A0 + 0] = fmaf(mf, dx, acc[A0 + 0]);
    acc[A0 + 1] = fmaf(mf, dy, acc[A0 + 1]);
    acc[A0 + 2] = fmaf(mf, dz, acc[A0 + 2]);
    acc[FSUM] += mf;
    acc[J10 + 0] = fmaf(mf, ux, acc[J10 + 0]);
    acc[J10 + 1] = fmaf(mf, uy, acc[J10 + 1]);
    acc[J10 + 2] = fmaf(mf, uz, acc[J10 + 2]);
    const float dv = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
    const float gx = mg * dx, gy = mg * dy, gz = mg * dz;
    acc[TXX] = fmaf(gx, dx, acc[TXX]);
    acc[TYY] = fmaf(gy, dy, acc[TYY]);
    acc[TZZ] = fmaf(gz, dz, acc[TZZ]);
    acc[TXY] = fmaf(gx, dy, acc[TXY]);
    acc[TXZ] = fmaf(gx, dz, acc[TXZ]);
    acc[TYZ] = fmaf(gy, dz, acc[TYZ]);
    acc[J20 + 0] = fmaf(gx, dv, acc[J20 + 0]);
    acc[J20 + 1] = fmaf(gy, dv, acc[J20 + 1]);
    acc[J20 + 2] = fmaf(gz, dv, acc[J20 + 2]);
    acc[PSUM] += mp;
}

// Offset from a target to a node's centre of mass in FP32, and the geometric
// opening criterion of Section 3 (accept iff L^2 < Theta^2 r^2) decided from
// FP32 bounds when they are conclusive.  The offset is formed from the
// two-part FP32 forms of both positions (x = hi + lo to 2^-48 relative):
// TwoSum of the hi parts plus the difference of the lo parts, so it is within
// 2^-24 |d| + 2^-46 (|com| + |x|) of the exact difference; each component is
// widened by 2^-23 |d| + 2^-44 (|com| + |x|) into an interval that holds the
// exact one, and r^2 is bracketed by the sums of squares of the interval
// ends.  The FP64 decision (L^2 and Theta^2 r^2 rounded from values within
// 2^-50 of the exact ones) then agrees with the FP32 one whenever L^2 is
// below Theta^2 r_lo^2 (1 - 2^-18) or above Theta^2 r_hi^2 (1 + 2^-18), a
// margin far beyond the few FP32 roundings of the bounds; the guards keep
// every FP32 quantity normal.  Returns 1 (accept), 0 (open) or -1 (FP32
// bounds inconclusive: the caller decides in FP64).
__device__ __forceinline__ int open_test_f32(const float4 &hi, const float4 &lo, const float xh[3],
                                             const float xl[3], float theta2f, float d[3])
{
    const float ch[3] = {hi.x, hi.y, hi.z}, cl[3] = {lo.x, lo.y, lo.z};
    float r2lo = 0.0f, r2hi = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = ch[c], b = -xh[c];
        const float sum = __fadd_rn(a, b);
        const float bb = __fsub_rn(sum, a);
        const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
        d[c] = __fadd_rn(sum, __fadd_rn(err, __fsub_rn(cl[c], xl[c])));
        const float ad = fabsf(d[c]);
        const float del = __fmaf_rn(0x1p-23f, ad, 0x1p-44f * (fabsf(a) + fabsf(b)));
        const float l = fmaxf(__fsub_rn(ad, del), 0.0f), u = __fadd_rn(ad, del);
        r2lo = __fmaf_rn(l, l, r2lo);
        r2hi = __fmaf_rn(u, u, r2hi);
    }
    const float L2 = lo.w;
    if (L2 >= 0x1p-100f && r2hi <= 0x1p100f && theta2f <= 0x1p20f) {
        if (L2 < __fmul_rn(__fmul_rn(theta2f, r2lo), 1.0f - 0x1p-18f)) return 1;
        if (L2 > __fmul_rn(__fmul_rn(theta2f, r2hi), 1.0f + 0x1p-18f)) return 0;
    }
    return -1;
}

// The walk is warp-coherent: the 32 targets of a warp (neighbours in tree
// order) share one traversal position and read each node once.  Every lane
// still takes its own decisions, in the order and with the operations of a
// walk of its own: the warp descends into a node when any active lane opens
// it, and a lane that accepted a node (or is past its subtree) stays idle
// until the traversal leaves that node's range of tree positions -- children
// partition their parent's range in order, so a pre-order walk reaches the
// next node outside it exactly at the node the lane's own walk goes to next.
// Each lane therefore visits the same nodes, in the same order, as a walk of
// its own: the oracle's interactions, summed in the oracle's order.
//
// Decisions are those of FP64 arithmetic (open_test_f32, else FP64; always
// FP64 with the relative criterion).  MIXED: every pair term in FP32 (nodes
// from the FP32 offset of open_test_f32; leaf elements from their FP32
// offsets to the leaf's centre of mass plus that offset), FP32 sums of at
// most 32 + leaf_size interactions added into FP64.  FP64 walk: offsets and
// pair terms in FP64, partial sums carried by TwoSum.
template <bool POT, bool MIXED>
__global__ void __launch_bounds__(kWalkNT) tree_walk_kernel(TreeView t, EvalArgs a, WalkArgs w)
{
    int64_t n_tgt = w.n_idx_max;
    if (w.idx && w.n_idx_dev) {
        int64_t c = *w.n_idx_dev;
        if (c < 0) c = 0;
        if (c < n_tgt) n_tgt = c;
    }
    const int64_t s = (int64_t)blockIdx.x * kWalkNT + threadIdx.x;
    bool live = s < n_tgt;
    int64_t i = 0;
    if (live) {
        i = w.idx ? (int64_t)w.idx[s] : (int64_t)t.order[s];
        if (i < 0 || i >= t.n) {
            flag_or(t.flags, GRAV_FLAG_BADINDEX);
            live = false;
            i = 0;
        }
    }
    // the whole warp walks together; a warp without live targets leaves
    if (__ballot_sync(0xffffffffu, live) == 0u) return;
    const double xi[3] = {w.pos[3 * i], w.pos[3 * i + 1], w.pos[3 * i + 2]};
    const double vi[3] = {w.vel[3 * i], w.vel[3 * i + 1], w.vel[3 * i + 2]};
    const double h2 = w.h * w.h, hinv = 1.0 / w.h;
    const double ext = t.frame[3];
    double rel = 0.0;
    if (w.alpha > 0.0 && w.a_old) {
        const double *ao = w.a_old + 3 * i;
        rel = __dmul_rn(w.alpha, __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ao[0], ao[0]),
                                                                __dmul_rn(ao[1], ao[1])),
                                                      __dmul_rn(ao[2], ao[2]))));
    }
    double acc[kNCPot], shi[kNCPot], slo[kNCPot];
    float accf[MIXED ? kNCPot : 1];
#pragma unroll
    for (int c = 0; c < kNCPot; ++c) {
        acc[c] = 0.0;
        shi[c] = 0.0;
        slo[c] = 0.0;
        if (MIXED) accf[MIXED ? c : 0] = 0.0f;
    }
    const float h2f = (float)(w.h * w.h), hinvf = (float)(1.0 / w.h);
    const float vi32[3] = {__double2float_rn(vi[0]), __double2float_rn(vi[1]), __double2float_rn(vi[2])};
    float xh[3], xl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xh[c] = __double2float_rn(xi[c]);
        xl[c] = __double2float_rn(__dsub_rn(xi[c], (double)xh[c]));
    }
    const float theta2f = __double2float_rn(w.theta2);
    int pending = 0;
    long long inter = 0;
    // tree positions below skip_until belong to nodes this lane does not
    // visit (dead lanes visit none)
    int32_t skip_until = live ? 0 : INT32_MAX;
    int32_t node = 0;                          // shared by the warp
    int64_t steps = 0;
    const int64_t n_nodes = t.counters[0];
    while (node >= 0) {
        if (++steps > n_nodes + 1) {            // a walk visits each node at most once
            if ((threadIdx.x & 31) == 0) flag_or(t.flags, GRAV_FLAG_OVERFLOW);
            break;
        }
        const int32_t nfirst = t.first[node], ncount = t.count[node];
        const int32_t child = t.child_first[node];
        bool open = false;
        if (nfirst >= skip_until) {
            const float4 chi = t.chi[node], clo = t.clo[node];
            float d[3];
            int decided = open_test_f32(chi, clo, xh, xl, theta2f, d);
            if (decided < 0 || rel > 0.0) {
                const double dx = __dsub_rn(t.com[3 * (int64_t)node], xi[0]);
                const double dy = __dsub_rn(t.com[3 * (int64_t)node + 1], xi[1]);
                const double dz = __dsub_rn(t.com[3 * (int64_t)node + 2], xi[2]);
                const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                const double L = scalbn(ext, -(int)t.level[node]);
                const double L2 = __dmul_rn(L, L);
                bool acc64 = L2 < __dmul_rn(w.theta2, r2);
                if (acc64 && rel > 0.0)
                    acc64 = __dmul_rn(__dmul_rn(a.G, t.m[node]), L2) <= __dmul_rn(__dmul_rn(rel, r2), r2);
                decided = acc64 ? 1 : 0;
            }
            const bool accept = decided == 1;
            if (accept) skip_until = nfirst + ncount;
            if (accept || child < 0) {
                // an accepted node is one interaction, a leaf its elements in
                // order; both run through one loop so that the lanes of a warp
                // that accept and those that sum the leaf share its passes
                const int32_t cnt = accept ? 1 : ncount;
                if (MIXED) {
                    const float4 vc = t.vcom32[node];
                    for (int32_t q = 0; q < cnt; ++q) {
                        float4 o = make_float4(0.0f, 0.0f, 0.0f, chi.w), v = vc;
                        bool self = false;
                        if (!accept) {
                            o = t.soff[nfirst + q];
                            v = t.svel[nfirst + q];
                            self = t.order[nfirst + q] == i;
                        }
                        pair_f(accf, o.w, o.x + d[0], o.y + d[1], o.z + d[2], v.x - vi32[0],
                               v.y - vi32[1], v.z - vi32[2], h2f, hinvf, self);
                        inter += !self;
                        ++pending;
                    }
                } else {
                    for (int32_t q = 0; q < cnt; ++q) {
                        double m, dx, dy, dz, ux, uy, uz;
                        bool self = false;
                        if (accept) {
                            m = t.m[node];
                            dx = __dsub_rn(t.com[3 * (int64_t)node], xi[0]);
                            dy = __dsub_rn(t.com[3 * (int64_t)node + 1], xi[1]);
                            dz = __dsub_rn(t.com[3 * (int64_t)node + 2], xi[2]);
                            ux = t.vcom[3 * (int64_t)node] - vi[0];
                            uy = t.vcom[3 * (int64_t)node + 1] - vi[1];
                            uz = t.vcom[3 * (int64_t)node + 2] - vi[2];
                        } else {
                            const int32_t j = t.order[nfirst + q];
                            m = w.mass[j];
                            dx = w.pos[3 * j] - xi[0];
                            dy = w.pos[3 * j + 1] - xi[1];
                            dz = w.pos[3 * j + 2] - xi[2];
                            ux = w.vel[3 * j] - vi[0];
                            uy = w.vel[3 * j + 1] - vi[1];
                            uz = w.vel[3 * j + 2] - vi[2];
                            self = j == i;
                        }
                        pair_d(acc, m, dx, dy, dz, ux, uy, uz, h2, hinv, self);
                        inter += !self;
                        ++pending;
                    }
                }
            } else {
                open = true;
            }
        }
        // carry the partial sums into the FP64 ones when any lane of the warp
        // has gathered kFlushEvery interactions: all lanes carry together, so
        // the FP64 pipe (1/74 of the FP32 rate) runs once per warp, not once
        // per lane
        if (__any_sync(0xffffffffu, pending >= kFlushEvery)) {
#pragma unroll
            for (int c = 0; c < kNCPot; ++c) {
                if (MIXED) {
                    shi[c] += (double)accf[MIXED ? c : 0];
                    accf[MIXED ? c : 0] = 0.0f;
                } else {
                    two_sum_acc(shi[c], slo[c], acc[c]);
                    acc[c] = 0.0;
                }
            }
            pending = 0;
        }
        node = __any_sync(0xffffffffu, open) ? child : t.next[node];
    }
    if (!live) return;
    double sum[kNCPot];
#pragma unroll
    for (int c = 0; c < kNCPot; ++c) {
        if (MIXED) {
            sum[c] = shi[c] + (double)accf[MIXED ? c : 0];
        } else {
            two_sum_acc(shi[c], slo[c], acc[c]);
            sum[c] = __dadd_rn(shi[c], slo[c]);
        }
    }
    write_target<POT, false>(a, i, sum);
    if (w.stats)
        atomicAdd(reinterpret_cast<unsigned long long *>(&w.stats[1]), (unsigned long long)inter);
}

__global__ void tree_stats_kernel(TreeView t, long long *stats)
{
    if (threadIdx.x == 0) stats[0] = t.counters[0];
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int64_t grav_tree_workspace_bytes(int64_t n, int32_t leaf_size)
{
    if (n < 0 || n > INT32_MAX / 4) return fail(GRAV_EINVAL, "grav_tree_workspace_bytes: n outside [0, 2^29)");
    if (leaf_size < 1 || leaf_size > 64)
        return fail(GRAV_EINVAL, "grav_tree_workspace_bytes: leaf_size outside [1, 64]");
    if (max_nodes_for(n, leaf_size) > INT32_MAX)
        return fail(GRAV_EINVAL, "grav_tree_workspace_bytes: node bound above 2^31 (raise leaf_size)");
    return tree_layout(n, leaf_size).total;
}

extern "C" int grav_eval_tree(const grav_params *p, const grav_tree_params *tp, int64_t n,
                              const double *pos, const double *vel, const double *mass,
                              const double *a_old, const int32_t *idx, const int32_t *n_idx_dev,
                              int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                              double *pot, double *dt_grav, int32_t *order_out,
                              long long *stats_dev, int32_t *flags_dev, void *workspace,
                              int64_t workspace_bytes, void *stream)
{
    static const char *who = "grav_eval_tree";
    if (!p || !tp) return fail(GRAV_EINVAL, "%s: null parameters", who);
    if (!(p->G > 0.0) || !(p->h > 0.0) || !(p->eta > 0.0) || !std::isfinite(p->G) ||
        !std::isfinite(p->h) || !std::isfinite(p->eta))
        return fail(GRAV_EINVAL, "%s: G, h and eta must be positive and finite", who);
    if (p->box != 0.0) return fail(GRAV_EINVAL, "%s: the tree supports open boundaries only", who);
    if (p->precision != GRAV_F64 && p->precision != GRAV_MIXED)
        return fail(GRAV_EINVAL, "%s: precision must be GRAV_F64 or GRAV_MIXED", who);
    if (!(tp->theta >= 0.0) || !std::isfinite(tp->theta) || !(tp->alpha >= 0.0) ||
        !std::isfinite(tp->alpha))
        return fail(GRAV_EINVAL, "%s: theta and alpha must be finite and >= 0", who);
    if (tp->leaf_size < 1 || tp->leaf_size > 64)
        return fail(GRAV_EINVAL, "%s: leaf_size outside [1, 64]", who);
    if (n < 0 || n > INT32_MAX / 4 || n_idx_max < 0 || n_idx_max > n)
        return fail(GRAV_EINVAL, "%s: sizes outside range (n < 2^29, n_idx_max <= n)", who);
    if (!idx && n_idx_max != n) return fail(GRAV_EINVAL, "%s: idx is NULL but n_idx_max != n", who);
    if (max_nodes_for(n, tp->leaf_size) > INT32_MAX)
        return fail(GRAV_EINVAL, "%s: node bound above 2^31 (raise leaf_size)", who);
    if (n == 0) return GRAV_OK;
    if (!pos || !vel || !mass || !acc || !jerk || !tidal || (p->want_pot && !pot))
        return fail(GRAV_EINVAL, "%s: null input or output array", who);
    if (!workspace || !aligned(workspace, 256))
        return fail(GRAV_EINVAL, "%s: workspace null or not 256-byte aligned", who);
    const TreeLayout L = tree_layout(n, tp->leaf_size);
    if (workspace_bytes < L.total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)L.total);
    char *ws = static_cast<char *>(workspace);
    cudaStream_t st = as_stream(stream);
    TreeView t;
    t.n = n;
    t.max_nodes = L.max_nodes;
    t.leaf_size = tp->leaf_size;
    t.frame = reinterpret_cast<double *>(ws + L.frame);
    t.counters = reinterpret_cast<int32_t *>(ws + L.counters);
    t.first = reinterpret_cast<int32_t *>(ws + L.first);
    t.count = reinterpret_cast<int32_t *>(ws + L.count);
    t.child_first = reinterpret_cast<int32_t *>(ws + L.child_first);
    t.next = reinterpret_cast<int32_t *>(ws + L.next);
    t.n_child = reinterpret_cast<int8_t *>(ws + L.n_child);
    t.level = reinterpret_cast<int8_t *>(ws + L.level);
    t.m = reinterpret_cast<double *>(ws + L.m);
    t.com = reinterpret_cast<double *>(ws + L.com);
    t.vcom = reinterpret_cast<double *>(ws + L.vcom);
    t.vcom32 = reinterpret_cast<float4 *>(ws + L.vcom32);
    t.chi = reinterpret_cast<float4 *>(ws + L.chi);
    t.clo = reinterpret_cast<float4 *>(ws + L.clo);
    t.soff = reinterpret_cast<float4 *>(ws + L.soff);
    t.svel = reinterpret_cast<float4 *>(ws + L.svel);
    t.flags = flags_dev;

    // bounding cube and keys
    const int nbb = (int)std::min<int64_t>(kBboxBlocks, (n + 255) / 256);
    double *part = reinterpret_cast<double *>(ws + L.part);
    bbox_partial_kernel<<<nbb, 256, 0, st>>>(n, pos, part);
    bbox_final_kernel<<<1, 32, 0, st>>>(nbb, part, t.frame);
    uint64_t *ka = reinterpret_cast<uint64_t *>(ws + L.key_a), *kb = reinterpret_cast<uint64_t *>(ws + L.key_b);
    int32_t *va = reinterpret_cast<int32_t *>(ws + L.val_a), *vb = reinterpret_cast<int32_t *>(ws + L.val_b);
    key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, pos, t.frame, ka, va, flags_dev);
    int rc = check_launch("grav_eval_tree/keys");
    if (rc) return rc;

    // stable radix sort (an even number of passes ends in the a buffers)
    int32_t *hist = reinterpret_cast<int32_t *>(ws + L.hist);
    const int64_t nb = L.n_sort_blocks;
    for (int pass = 0; pass < kPasses; ++pass) {
        const int shift = 4 * pass;
        sort_hist_kernel<<<(unsigned)nb, kSortNT, 0, st>>>(n, ka, shift, hist, nb);
        sort_scan_kernel<<<1, 1024, 0, st>>>(hist, nb * kBins);
        sort_scatter_kernel<<<(unsigned)nb, kSortNT, 0, st>>>(n, ka, va, kb, vb, shift, hist, nb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    rc = check_launch("grav_eval_tree/sort");
    if (rc) return rc;
    t.key = ka;
    t.order = va;

    // levels: split top-down, moments bottom-up, next links top-down
    const unsigned g = (unsigned)std::min<int64_t>(4096, (L.max_nodes + 255) / 256);
    tree_init_kernel<<<1, 32, 0, st>>>(t);
    for (int lvl = 0; lvl <= kMaxLevel; ++lvl) {
        tree_split_kernel<<<g, 256, 0, st>>>(t, lvl);
        tree_mark_kernel<<<1, 32, 0, st>>>(t, lvl);
    }
    for (int lvl = kMaxLevel; lvl >= 0; --lvl)
        tree_moment_kernel<<<g, 256, 0, st>>>(t, pos, vel, mass, lvl);
    for (int lvl = 0; lvl < kMaxLevel; ++lvl) tree_next_kernel<<<g, 256, 0, st>>>(t, lvl);
    const bool mixed = p->precision == GRAV_MIXED;
    tree_walk_data_kernel<<<g, 256, 0, st>>>(t, pos, vel, mass, mixed);
    rc = check_launch("grav_eval_tree/build");
    if (rc) return rc;
    if (order_out) {
        rc = check_cuda(cudaMemcpyAsync(order_out, t.order, n * sizeof(int32_t),
                                        cudaMemcpyDeviceToDevice, st),
                        "grav_eval_tree/order");
        if (rc) return rc;
    }
    if (stats_dev) {
        rc = check_cuda(cudaMemsetAsync(stats_dev, 0, 2 * sizeof(long long), st), "grav_eval_tree/stats");
        if (rc) return rc;
        tree_stats_kernel<<<1, 32, 0, st>>>(t, stats_dev);
    }
    if (n_idx_max == 0) return check_launch("grav_eval_tree/stats");

    // walk
    EvalArgs a{};
    a.n_src = n;
    a.G = p->G;
    a.h = p->h;
    a.sqrt_eta = std::sqrt(p->eta);
    a.acc = acc;
    a.jerk = jerk;
    a.tidal = tidal;
    a.pot = p->want_pot ? pot : nullptr;
    a.dt_grav = dt_grav;
    a.flags = flags_dev;
    WalkArgs w;
    w.pos = pos;
    w.vel = vel;
    w.mass = mass;
    w.a_old = a_old;
    w.idx = idx;
    w.n_idx_dev = idx ? n_idx_dev : nullptr;
    w.n_idx_max = n_idx_max;
    w.h = p->h;
    w.theta2 = tp->theta * tp->theta;
    w.alpha = tp->alpha;
    w.stats = stats_dev;
    const unsigned gw = (unsigned)((n_idx_max + kWalkNT - 1) / kWalkNT);
    if (p->want_pot && mixed)
        tree_walk_kernel<true, true><<<gw, kWalkNT, 0, st>>>(t, a, w);
    else if (mixed)
        tree_walk_kernel<false, true><<<gw, kWalkNT, 0, st>>>(t, a, w);
    else if (p->want_pot)
        tree_walk_kernel<true, false><<<gw, kWalkNT, 0, st>>>(t, a, w);
    else
        tree_walk_kernel<false, false><<<gw, kWalkNT, 0, st>>>(t, a, w);
    return check_launch("grav_eval_tree/walk");
}
