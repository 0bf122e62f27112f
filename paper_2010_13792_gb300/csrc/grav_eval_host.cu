// Host entry points of the force evaluation: argument checks, tile
// configuration, workspace layout and the launch sequence
//   pack tiles (K3) -> persistent direct sum (K4 / K5) -> split reduction (K9).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "grav_eval.cuh"

namespace grav {
namespace {

// Default tile configurations (measured on 2^20-element clouds, a 2^17
// Plummer sphere and 64^3 and 96^3 periodic lattices): 768-thread CTAs, one
// per SM, from 8192 targets; 256-thread CTAs (three per SM) for smaller sets
// and batched launches, where more CTAs per SM keep the SMs busier through the
// last round of work items.
constexpr int kDefaultMixed = 11;
constexpr int kDefaultMixedLarge = 17;
constexpr int64_t kLargeTargetSet = 1 << 13;
constexpr int kDefaultF64 = 0;
constexpr int64_t kSplitRowsPerSM = 16;   // partial capacity, in target blocks per SM

const EvalConfig *config_table(int32_t precision, int *count)
{
    if (precision == GRAV_MIXED) return mixed_configs(count);
    if (precision == GRAV_F64) return f64_configs(count);
    *count = 0;
    return nullptr;
}

int check_params(const grav_params *p, const char *who)
{
    if (!p) return fail(GRAV_EINVAL, "%s: null params", who);
    if (!(p->G > 0.0) || !std::isfinite(p->G)) return fail(GRAV_EINVAL, "%s: G must be finite and > 0", who);
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(GRAV_EINVAL, "%s: h must be finite and > 0", who);
    if (!(p->eta > 0.0) || !std::isfinite(p->eta)) return fail(GRAV_EINVAL, "%s: eta must be finite and > 0", who);
    if (p->precision != GRAV_F64 && p->precision != GRAV_MIXED)
        return fail(GRAV_EINVAL, "%s: precision must be GRAV_F64 or GRAV_MIXED", who);
    if (p->max_split < 0) return fail(GRAV_EINVAL, "%s: max_split < 0", who);
    if (!(p->box >= 0.0) || !std::isfinite(p->box)) return fail(GRAV_EINVAL, "%s: box must be finite and >= 0", who);
    if (p->box > 0.0 && !(2.0 * p->h < p->box))
        return fail(GRAV_EINVAL, "%s: a periodic box must be wider than twice the softening", who);
    int n = 0;
    config_table(p->precision, &n);
    if (p->tile_config < -1 || p->tile_config >= n)
        return fail(GRAV_EINVAL, "%s: tile_config %d outside [-1, %d)", who, p->tile_config, n);
    return GRAV_OK;
}

int default_index(int32_t precision, int mode, int64_t n_targets)
{
    if (precision != GRAV_MIXED) return kDefaultF64;
    (void)mode;   // the same choice in every mode
    return n_targets >= kLargeTargetSet ? kDefaultMixedLarge : kDefaultMixed;
}

// The configuration of an evaluation: p->tile_config, or the default for its
// mode and (upper bound on the) number of targets.
const EvalConfig *resolve(const grav_params *p, int mode, int64_t n_targets, int *index)
{
    int n = 0;
    const EvalConfig *t = config_table(p->precision, &n);
    int i = p->tile_config >= 0 ? p->tile_config : default_index(p->precision, mode, n_targets);
    *index = i;
    return &t[i];
}

// Per source tile for adaptive softening: (1/h_j, zeta_j) in FP32 in tile
// order, padding (1, 0), and the tile's largest support rounded up.  One CTA
// of 256 threads per tile of S sources; flags non-positive or non-finite h.
__global__ void __launch_bounds__(256)
pack_soft_kernel(int64_t n_src, int S, const double *__restrict__ h_elem,
                 const double *__restrict__ zeta, float2 *__restrict__ hz, float *__restrict__ geo_h,
                 int32_t *flags)
{
    const int64_t t = blockIdx.x;
    float hmax = 0.0f;
    for (int k = threadIdx.x; k < S; k += 256) {
        const int64_t j = t * S + k;
        float2 v = make_float2(1.0f, 0.0f);
        if (j < n_src) {
            const double h = h_elem[j];
            const double z = zeta ? zeta[j] : 0.0;
            if (!(h > 0.0) || !isfinite(h) || !isfinite(z)) {
                flag_or(flags, GRAV_FLAG_NONFINITE);
            } else {
                v = make_float2(__double2float_rn(1.0 / h), __double2float_rn(z));
                hmax = fmaxf(hmax, __double2float_ru(h));
            }
        }
        hz[t * S + k] = v;
    }
    hmax = block_max<256>(hmax);
    if (threadIdx.x == 0) geo_h[t] = hmax;
}

// Periodic-box fields of the kernel arguments.  Beyond the tie lengths a
// pair separation component is formed again in FP64 with the image decided
// by an exact division: half a box less 2^-20 box on the mixed path (an FP32
// separation there is good to about 4 * 2^-24 box), less 2^-40 box on the
// FP64 path (1/box rounds once).
void set_box(EvalArgs &a, double box)
{
    a.box = box;
    a.box_inv = box > 0.0 ? 1.0 / box : 0.0;
    a.box_tie = box > 0.0 ? box * (0.5 - 0x1p-40) : 0.0;
    a.box_f = (float)box;
    a.box_inv_f = (float)a.box_inv;
    float tie = (float)(box * (0.5 - 0x1p-20));
    if ((double)tie > box * (0.5 - 0x1p-20)) tie = std::nextafter(tie, 0.0f);
    a.box_tie_f = box > 0.0 ? tie : 0.0f;
    a.box_lo_f = box > 0.0 ? (float)(box - (double)a.box_f) : 0.0f;
}

int grid_for(const EvalConfig *c, int index, int mode, bool pot, int *grid)
{
    static std::mutex mu;
    static int cache[64][2][kMaxTileConfigs][3][2];   // [device][precision][config][mode][pot]
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    int sms = 0;
    rc = device_sm_count(&sms);
    if (rc) return rc;
    if (dev >= 64 || index >= kMaxTileConfigs) return fail(GRAV_ECUDA, "device or config index out of range");
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][c->precision][index][mode][pot ? 1 : 0];
    if (slot == 0) {
        int b = 0;
        rc = check_cuda((cudaError_t)c->occupancy[mode][pot ? 1 : 0](&b), "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (rc) return rc;
        if (b < 1) return fail(GRAV_ECUDA, "force kernel cannot be resident on an SM");
        slot = b * sms;
    }
    *grid = slot;
    return GRAV_OK;
}

struct Layout {
    int64_t n_tiles;
    int64_t geo_off, src_off, lo_off, part_off, total;
    int64_t part_cap_rows;
    int64_t hz_off, geo_h_off;     // adaptive softening only (else 0)
    int32_t max_split;
};

int make_layout(const grav_params *p, const EvalConfig *c, int64_t n_src, int64_t n_idx_max,
                Layout *L, bool soft = false)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    const int64_t S = c->s;
    const int64_t BT = (int64_t)c->threads * c->kt;
    const int64_t elem = (c->precision == GRAV_MIXED) ? 16 : 32;
    const int NC = p->want_pot ? kNCPot : kNC;
    L->max_split = p->max_split > 0 ? p->max_split : kDefaultMaxSplit;
    L->n_tiles = (n_src + S - 1) / S;
    L->geo_off = 0;
    L->src_off = round_up(L->n_tiles * (int64_t)sizeof(TileGeom), 256);
    L->lo_off = L->src_off + round_up(L->n_tiles * 2 * S * elem, 256);
    const int64_t lo_bytes = (c->precision == GRAV_MIXED) ? L->n_tiles * kLoPlanes * S * 4 : 0;
    L->part_off = L->lo_off + round_up(lo_bytes, 256);
    const int64_t n_tb_max = (n_idx_max + BT - 1) / BT;
    int64_t blocks = 0;
    if (L->max_split > 1 && L->n_tiles > 1)
        blocks = std::min<int64_t>(n_tb_max * L->max_split, kSplitRowsPerSM * sms);
    L->part_cap_rows = blocks * BT;
    L->total = L->part_off + round_up(L->part_cap_rows * NC * 8, 256);
    L->hz_off = L->geo_h_off = 0;
    if (soft) {
        L->hz_off = L->total;
        L->geo_h_off = L->hz_off + round_up(L->n_tiles * S * (int64_t)sizeof(float2), 256);
        L->total = L->geo_h_off + round_up(L->n_tiles * (int64_t)sizeof(float), 256);
    }
    if (L->total < 256) L->total = 256;
    return GRAV_OK;
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int32_t grav_tile_config_count(int32_t precision)
{
    int n = 0;
    config_table(precision, &n);
    return n;
}

extern "C" int32_t grav_default_tile_config(int32_t precision, int32_t periodic, int32_t soft,
                                            int64_t n_targets)
{
    int n = 0;
    if (!config_table(precision, &n)) return fail(GRAV_EINVAL, "grav_default_tile_config: bad precision");
    if (n_targets < 0) return fail(GRAV_EINVAL, "grav_default_tile_config: n_targets < 0");
    const int mode = soft ? kModeSoft : (periodic ? kModePeriodic : kModeOpen);
    return default_index(precision, mode, n_targets);
}

extern "C" int grav_tile_config(int32_t precision, int32_t index, grav_tile_info *out)
{
    int n = 0;
    const EvalConfig *t = config_table(precision, &n);
    if (!out) return fail(GRAV_EINVAL, "grav_tile_config: null out");
    if (!t) return fail(GRAV_EINVAL, "grav_tile_config: bad precision");
    if (index == -1) index = default_index(precision, kModeOpen, 0);
    if (index < 0 || index >= n) return fail(GRAV_EINVAL, "grav_tile_config: index out of range");
    out->threads = t[index].threads;
    out->targets_per_thread = t[index].kt;
    out->sources_per_tile = t[index].s;
    out->targets_per_block = t[index].threads * t[index].kt;
    out->unroll = t[index].unroll;
    out->shared_accumulators = t[index].sacc;
    return GRAV_OK;
}

namespace grav {
namespace {

int64_t workspace_bytes_for(const grav_params *p, int64_t n_src, int64_t n_idx_max, bool soft,
                            const char *who)
{
    int rc = check_params(p, who);
    if (rc) return rc;
    if (soft && p->box != 0.0)
        return fail(GRAV_EINVAL, "%s: adaptive softening supports open boundaries only", who);
    if (n_src < 0 || n_idx_max < 0 || n_src > INT32_MAX || n_idx_max > INT32_MAX)
        return fail(GRAV_EINVAL, "%s: sizes outside [0, 2^31)", who);
    int index = 0;
    const int mode = soft ? kModeSoft : (p->box > 0.0 ? kModePeriodic : kModeOpen);
    const EvalConfig *c = resolve(p, mode, n_idx_max, &index);
    Layout L;
    rc = make_layout(p, c, n_src, n_idx_max, &L, soft);
    if (rc) return rc;
    return L.total;
}

// One system: open boundaries, periodic box (p->box > 0) or per-element
// adaptive softening (h_elem not NULL).
int eval_single(const char *who, const grav_params *p, bool soft, int64_t n_src, const double *pos,
                const double *vel, const double *mass, const double *h_elem, const double *zeta,
                const int32_t *idx, const int32_t *n_idx_dev, int64_t n_idx_max, double *acc,
                double *jerk, double *tidal, double *pot, double *dt_grav, int32_t *flags_dev,
                void *workspace, int64_t workspace_bytes, void *stream)
{
    const int mode = soft ? kModeSoft : (p->box > 0.0 ? kModePeriodic : kModeOpen);
    int rc = check_params(p, who);
    if (rc) return rc;
    if (soft && p->box != 0.0)
        return fail(GRAV_EINVAL, "%s: adaptive softening supports open boundaries only", who);
    if (n_src < 0 || n_idx_max < 0 || n_src > INT32_MAX || n_idx_max > INT32_MAX)
        return fail(GRAV_EINVAL, "%s: sizes outside [0, 2^31)", who);
    if (!idx && n_idx_max != n_src)
        return fail(GRAV_EINVAL, "%s: idx is NULL but n_idx_max != n_src", who);
    if (n_src == 0 || n_idx_max == 0) return GRAV_OK;
    if (!pos || !vel || !mass || !acc || !jerk || !tidal || (soft && !h_elem))
        return fail(GRAV_EINVAL, "%s: null input or output array", who);
    if (p->want_pot && !pot) return fail(GRAV_EINVAL, "%s: want_pot set but pot is NULL", who);
    if (!workspace) return fail(GRAV_EINVAL, "%s: null workspace", who);
    if (!aligned(workspace, 256)) return fail(GRAV_EINVAL, "%s: workspace not 256-byte aligned", who);
    int index = 0;
    const EvalConfig *c = resolve(p, mode, n_idx_max, &index);
    Layout L;
    rc = make_layout(p, c, n_src, n_idx_max, &L, soft);
    if (rc) return rc;
    if (workspace_bytes < L.total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)L.total);
    const bool want_pot = p->want_pot != 0;
    int grid = 0;
    rc = grid_for(c, index, mode, want_pot, &grid);
    if (rc) return rc;

    char *ws = static_cast<char *>(workspace);
    EvalArgs a{};
    a.n_src = n_src;
    a.idx = idx;
    a.n_idx_dev = n_idx_dev;
    a.n_idx_max = n_idx_max;
    a.geo = reinterpret_cast<const TileGeom *>(ws + L.geo_off);
    a.src = ws + L.src_off;
    a.n_tiles = (int32_t)L.n_tiles;
    a.max_split = L.max_split;
    a.grid = grid;
    a.pad0 = 0;
    a.part = reinterpret_cast<double *>(ws + L.part_off);
    a.part_cap_rows = L.part_cap_rows;
    a.src_lo = c->precision == GRAV_MIXED ? reinterpret_cast<const float *>(ws + L.lo_off) : nullptr;

    a.pos = pos;
    a.vel = vel;
    a.mass = mass;
    a.G = p->G;
    a.h = p->h;
    a.sqrt_eta = std::sqrt(p->eta);
    a.hf = (float)p->h;
    double h2 = p->h * p->h;
    float h2f = (float)h2;
    if ((double)h2f < h2) h2f = std::nextafter(h2f, INFINITY);
    a.h2f_up = h2f;
    a.hinvf = (float)(1.0 / p->h);
    a.pad1 = 0.0f;
    a.acc = acc;
    a.jerk = jerk;
    a.tidal = tidal;
    a.pot = want_pot ? pot : nullptr;
    a.dt_grav = dt_grav;
    a.flags = flags_dev;
    set_box(a, p->box);
    if (soft) {
        a.h_elem = h_elem;
        a.zeta = zeta;
        a.hz = reinterpret_cast<const float2 *>(ws + L.hz_off);
        a.geo_h = reinterpret_cast<const float *>(ws + L.geo_h_off);
    }

    cudaStream_t st = as_stream(stream);
    c->pack(n_src, pos, vel, mass, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev,
            const_cast<float *>(a.src_lo), (int)L.n_tiles, st);
    rc = check_launch("grav_eval/pack");
    if (rc) return rc;
    if (soft) {
        pack_soft_kernel<<<(unsigned)L.n_tiles, 256, 0, st>>>(
            n_src, c->s, h_elem, zeta, const_cast<float2 *>(a.hz), const_cast<float *>(a.geo_h),
            flags_dev);
        rc = check_launch("grav_eval_soft/pack_soft");
        if (rc) return rc;
    }
    c->launch[mode][want_pot ? 1 : 0](a, grid, st);
    rc = check_launch("grav_eval/eval");
    if (rc) return rc;
    const int32_t BT = c->threads * c->kt;
    bool need_reduce = L.part_cap_rows > 0;
    if (need_reduce && !n_idx_dev) {
        int64_t n_tb = (n_idx_max + BT - 1) / BT;
        need_reduce = choose_split(n_tb, a.n_tiles, grid, a.max_split, a.part_cap_rows, BT) > 1;
    }
    if (need_reduce) {
        launch_reduce(a, BT, want_pot, c->precision == GRAV_MIXED, n_idx_max, st);
        rc = check_launch("grav_eval/reduce");
        if (rc) return rc;
    }

    return GRAV_OK;
}

}  // namespace
}  // namespace grav

extern "C" int64_t grav_eval_workspace_bytes(const grav_params *p, int64_t n_src, int64_t n_idx_max)
{
    return workspace_bytes_for(p, n_src, n_idx_max, false, "grav_eval_workspace_bytes");
}

extern "C" int grav_eval_active(const grav_params *p, int64_t n_src, const double *pos,
                                const double *vel, const double *mass, const int32_t *idx,
                                const int32_t *n_idx_dev, int64_t n_idx_max, double *acc,
                                double *jerk, double *tidal, double *pot, double *dt_grav,
                                int32_t *flags_dev, void *workspace, int64_t workspace_bytes,
                                void *stream)
{
    return eval_single("grav_eval_active", p, false, n_src, pos, vel, mass, nullptr, nullptr, idx,
                       n_idx_dev, n_idx_max, acc, jerk, tidal, pot, dt_grav, flags_dev, workspace,
                       workspace_bytes, stream);
}

extern "C" int64_t grav_eval_soft_workspace_bytes(const grav_params *p, int64_t n_src,
                                                  int64_t n_idx_max)
{
    return workspace_bytes_for(p, n_src, n_idx_max, true, "grav_eval_soft_workspace_bytes");
}

extern "C" int grav_eval_soft(const grav_params *p, int64_t n_src, const double *pos,
                              const double *vel, const double *mass, const double *h_elem,
                              const double *zeta, const int32_t *idx, const int32_t *n_idx_dev,
                              int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                              double *pot, double *dt_grav, int32_t *flags_dev, void *workspace,
                              int64_t workspace_bytes, void *stream)
{
    return eval_single("grav_eval_soft", p, true, n_src, pos, vel, mass, h_elem, zeta, idx,
                       n_idx_dev, n_idx_max, acc, jerk, tidal, pot, dt_grav, flags_dev, workspace,
                       workspace_bytes, stream);
}

// ---------------------------------------------------------------------------
// Batched launches
// ---------------------------------------------------------------------------

namespace grav {
namespace {

constexpr int kPlanThreads = 1024;

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Exclusive scan of vals[0..n) by one CTA; out[0..n] receives the prefix
// sums and the total.  vals and out may alias.
template <typename TIn, typename TOut>
__device__ void cta_exclusive_scan(const TIn *vals, TOut *out, int n)
{
    __shared__ long long warp_tot[kPlanThreads / 32];
    __shared__ long long carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += kPlanThreads) {
        const int b = b0 + threadIdx.x;
        const long long v = (b < n) ? (long long)vals[b] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const long long excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
        __syncthreads();
        if (b < n) out[b] = (TOut)excl;
        if (threadIdx.x == 0) carry += warp_tot[kPlanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = (TOut)carry;
    __syncthreads();
}

// The plan of a batched launch (one CTA): per-system tiles and target
// ranges, the longest-first order of the systems and the work-item offsets;
// resets the ticket counter.
__global__ void __launch_bounds__(kPlanThreads)
batch_plan_kernel(BatchView b, const int32_t *__restrict__ idx, const int32_t *n_idx_dev,
                  int64_t n_idx_max, int64_t n_total, int32_t S, int32_t BT, double box,
                  int32_t *flags)
{
    const int n = b.n_sys;
    int64_t count = n_idx_max;
    if (n_idx_dev) {
        int64_t c = *n_idx_dev;
        count = c < 0 ? 0 : (c < n_idx_max ? c : n_idx_max);
    }
    for (int s = threadIdx.x; s < n; s += kPlanThreads) {
        const int64_t off = b.sys[s].offset, len = b.sys[s].n;
        const double h = b.sys[s].h;   // 0: the call's h
        bool ok = off >= 0 && len >= 0 && off + len <= n_total;
        if (ok && s > 0) ok = off >= b.sys[s - 1].offset + b.sys[s - 1].n;
        if (ok && h != 0.0) ok = h > 0.0 && isfinite(h) && (box == 0.0 || 2.0 * h < box);
        if (!ok) flag_or(flags, GRAV_FLAG_BADINDEX);
        // (no target list: every element is a target, slots are elements)
        const int64_t lo = !ok ? 0 : idx ? lower_bound_i32(idx, count, off) : off;
        const int64_t hi = !ok ? 0 : idx ? lower_bound_i32(idx, count, off + len) : off + len;
        b.idx_lo[s] = (int32_t)lo;
        b.idx_hi[s] = (int32_t)hi;
        b.ntb[s] = ok ? (int32_t)((hi - lo + BT - 1) / BT) : 0;
        b.tile_off[s] = ok ? (int32_t)((len + S - 1) / S) : 0;     // tile counts, scanned below
    }
    __syncthreads();
    cta_exclusive_scan<int32_t, int32_t>(b.tile_off, b.tile_off, n);
    // longest work item first: rank by system size, ties by index
    for (int s = threadIdx.x; s < n; s += kPlanThreads) {
        const int64_t key = b.sys[s].n;
        int rank = 0;
        for (int q = 0; q < n; ++q) {
            const int64_t kq = b.sys[q].n;
            rank += (kq > key) || (kq == key && q < s);
        }
        b.order[rank] = s;
    }
    __syncthreads();
    // items per rank, then their offsets (item_off doubles as the buffer)
    for (int r = threadIdx.x; r < n; r += kPlanThreads) b.item_off[r] = b.ntb[b.order[r]];
    __syncthreads();
    cta_exclusive_scan<int64_t, int64_t>(b.item_off, b.item_off, n);
    if (threadIdx.x == 0) {
        b.hdr->total_items = b.item_off[n];
        b.hdr->total_tiles = b.tile_off[n];
        b.hdr->ticket = 0ULL;
    }
}

struct BatchLayout {
    int64_t hdr, tile_off, idx_lo, idx_hi, ntb, order, item_off, geo, src, lo, total;
    int64_t max_tiles;
};

BatchLayout batch_layout(const EvalConfig *c, int32_t n_sys, int64_t n_total)
{
    BatchLayout L;
    const int64_t S = c->s;
    const int64_t elem = (c->precision == GRAV_MIXED) ? 16 : 32;
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
    o += round_up((c->precision == GRAV_MIXED) ? L.max_tiles * kLoPlanes * S * 4 : 0, 256);
    L.total = o;
    return L;
}

int batch_grid_for(const EvalConfig *c, int index, bool periodic, bool pot, int *grid)
{
    static std::mutex mu;
    static int cache[64][2][kMaxTileConfigs][2][2];
    int dev = 0, sms = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    rc = device_sm_count(&sms);
    if (rc) return rc;
    if (dev >= 64 || index >= kMaxTileConfigs) return fail(GRAV_ECUDA, "device or config index out of range");
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][c->precision][index][periodic ? 1 : 0][pot ? 1 : 0];
    if (slot == 0) {
        int b = 0;
        rc = check_cuda((cudaError_t)c->occupancy_batched[periodic ? 1 : 0][pot ? 1 : 0](&b),
                        "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (rc) return rc;
        if (b < 1) return fail(GRAV_ECUDA, "batched force kernel cannot be resident on an SM");
        slot = b * sms;
    }
    *grid = slot;
    return GRAV_OK;
}

}  // namespace

int launch_batch_plan(const BatchView &b, const int32_t *idx, const int32_t *n_idx_dev,
                      int64_t n_idx_max, int64_t n_total, int32_t S, int32_t BT, double box,
                      int32_t *flags, cudaStream_t st)
{
    batch_plan_kernel<<<1, kPlanThreads, 0, st>>>(b, idx, n_idx_dev, n_idx_max, n_total, S, BT, box,
                                                   flags);
    return check_launch("batch plan");
}

}  // namespace grav

extern "C" int64_t grav_batched_workspace_bytes(const grav_params *p, int32_t n_sys, int64_t n_total)
{
    int rc = check_params(p, "grav_batched_workspace_bytes");
    if (rc) return rc;
    if (n_sys < 0 || n_sys > GRAV_BATCH_MAX_SYSTEMS || n_total < 0 || n_total > INT32_MAX)
        return fail(GRAV_EINVAL, "grav_batched_workspace_bytes: n_sys or n_total out of range");
    int index = 0;
    const EvalConfig *c = resolve(p, kModeOpen, 0, &index);
    return batch_layout(c, n_sys, n_total).total;
}

extern "C" int grav_eval_batched(const grav_params *p, int32_t n_sys, const grav_system *systems,
                                 int64_t n_total, const double *pos, const double *vel,
                                 const double *mass, const int32_t *idx, const int32_t *n_idx_dev,
                                 int64_t n_idx_max, double *acc, double *jerk, double *tidal,
                                 double *pot, double *dt_grav, int32_t *flags_dev, void *workspace,
                                 int64_t workspace_bytes, void *stream)
{
    static const char *who = "grav_eval_batched";
    int rc = check_params(p, who);
    if (rc) return rc;
    if (n_sys < 0 || n_sys > GRAV_BATCH_MAX_SYSTEMS)
        return fail(GRAV_EINVAL, "%s: n_sys outside [0, %d]", who, GRAV_BATCH_MAX_SYSTEMS);
    if (n_total < 0 || n_total > INT32_MAX || n_idx_max < 0 || n_idx_max > n_total)
        return fail(GRAV_EINVAL, "%s: need 0 <= n_idx_max <= n_total < 2^31", who);
    if (n_sys == 0 || n_total == 0 || n_idx_max == 0) return GRAV_OK;
    if (!systems || !pos || !vel || !mass || !idx || !acc || !jerk || !tidal)
        return fail(GRAV_EINVAL, "%s: null array", who);
    if (p->want_pot && !pot) return fail(GRAV_EINVAL, "%s: want_pot set but pot is NULL", who);
    if (!workspace || !aligned(workspace, 256))
        return fail(GRAV_EINVAL, "%s: workspace missing or not 256-byte aligned", who);
    int index = 0;
    const EvalConfig *c = resolve(p, kModeOpen, 0, &index);
    const BatchLayout L = batch_layout(c, n_sys, n_total);
    if (workspace_bytes < L.total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)L.total);
    const bool want_pot = p->want_pot != 0;
    int grid = 0;
    rc = batch_grid_for(c, index, p->box > 0.0, want_pot, &grid);
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

    EvalArgs a{};
    a.n_src = n_total;
    a.idx = idx;
    a.n_idx_dev = n_idx_dev;
    a.n_idx_max = n_idx_max;
    a.geo = reinterpret_cast<const TileGeom *>(ws + L.geo);
    a.src = ws + L.src;
    a.src_lo = c->precision == GRAV_MIXED ? reinterpret_cast<const float *>(ws + L.lo) : nullptr;
    a.n_tiles = 0;
    a.max_split = 1;
    a.grid = grid;
    a.pad0 = 0;
    a.part = nullptr;
    a.part_cap_rows = 0;
    a.pos = pos;
    a.vel = vel;
    a.mass = mass;
    a.G = p->G;
    a.h = p->h;
    a.sqrt_eta = std::sqrt(p->eta);
    a.hf = (float)p->h;
    double h2 = p->h * p->h;
    float h2f = (float)h2;
    if ((double)h2f < h2) h2f = std::nextafter(h2f, INFINITY);
    a.h2f_up = h2f;
    a.hinvf = (float)(1.0 / p->h);
    a.pad1 = 0.0f;
    a.acc = acc;
    a.jerk = jerk;
    a.tidal = tidal;
    a.pot = want_pot ? pot : nullptr;
    a.dt_grav = dt_grav;
    a.flags = flags_dev;
    set_box(a, p->box);

    cudaStream_t st = as_stream(stream);
    const int32_t BT = c->threads * c->kt;
    rc = launch_batch_plan(b, idx, n_idx_dev, n_idx_max, n_total, c->s, BT, p->box, flags_dev, st);
    if (rc) return rc;
    c->pack_batched(b, pos, vel, mass, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src),
                    flags_dev, const_cast<float *>(a.src_lo), (int)L.max_tiles, st);
    rc = check_launch("grav_eval_batched/pack");
    if (rc) return rc;
    c->launch_batched[p->box > 0.0 ? 1 : 0][want_pot ? 1 : 0](a, b, grid, st);
    return check_launch("grav_eval_batched/eval");
}
