// Host entry points of the force evaluation: argument checks, tile
// configuration, workspace layout and the launch sequence
//   pack tiles (K3) -> persistent direct sum (K4 / K5) -> split reduction (K9).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "grav_eval.cuh"

namespace grav {
namespace {

constexpr int kDefaultMixed = 2;
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
    int n = 0;
    config_table(p->precision, &n);
    if (p->tile_config < -1 || p->tile_config >= n)
        return fail(GRAV_EINVAL, "%s: tile_config %d outside [-1, %d)", who, p->tile_config, n);
    return GRAV_OK;
}

const EvalConfig *resolve(const grav_params *p, int *index)
{
    int n = 0;
    const EvalConfig *t = config_table(p->precision, &n);
    int i = p->tile_config >= 0 ? p->tile_config : (p->precision == GRAV_MIXED ? kDefaultMixed : kDefaultF64);
    *index = i;
    return &t[i];
}

int grid_for(const EvalConfig *c, int index, bool pot, int *grid)
{
    static std::mutex mu;
    static int cache[64][2][16][2];   // [device][precision][config][pot]
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    int sms = 0;
    rc = device_sm_count(&sms);
    if (rc) return rc;
    if (dev >= 64 || index >= 16) return fail(GRAV_ECUDA, "device or config index out of range");
    std::lock_guard<std::mutex> lk(mu);
    int &slot = cache[dev][c->precision][index][pot ? 1 : 0];
    if (slot == 0) {
        int b = 0;
        rc = check_cuda((cudaError_t)c->occupancy[pot ? 1 : 0](&b), "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (rc) return rc;
        if (b < 1) return fail(GRAV_ECUDA, "force kernel cannot be resident on an SM");
        slot = b * sms;
    }
    *grid = slot;
    return GRAV_OK;
}

struct Layout {
    int64_t n_tiles;
    int64_t geo_off, src_off, part_off, total;
    int64_t part_cap_rows;
    int32_t max_split;
};

int make_layout(const grav_params *p, const EvalConfig *c, int64_t n_src, int64_t n_idx_max,
                Layout *L)
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
    L->part_off = L->src_off + round_up(L->n_tiles * 2 * S * elem, 256);
    const int64_t n_tb_max = (n_idx_max + BT - 1) / BT;
    int64_t blocks = 0;
    if (L->max_split > 1 && L->n_tiles > 1)
        blocks = std::min<int64_t>(n_tb_max * L->max_split, kSplitRowsPerSM * sms);
    L->part_cap_rows = blocks * BT;
    L->total = L->part_off + round_up(L->part_cap_rows * NC * 8, 256);
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

extern "C" int grav_tile_config(int32_t precision, int32_t index, grav_tile_info *out)
{
    int n = 0;
    const EvalConfig *t = config_table(precision, &n);
    if (!out) return fail(GRAV_EINVAL, "grav_tile_config: null out");
    if (!t) return fail(GRAV_EINVAL, "grav_tile_config: bad precision");
    if (index == -1) index = precision == GRAV_MIXED ? kDefaultMixed : kDefaultF64;
    if (index < 0 || index >= n) return fail(GRAV_EINVAL, "grav_tile_config: index out of range");
    out->threads = t[index].threads;
    out->targets_per_thread = t[index].kt;
    out->sources_per_tile = t[index].s;
    out->targets_per_block = t[index].threads * t[index].kt;
    return GRAV_OK;
}

extern "C" int64_t grav_eval_workspace_bytes(const grav_params *p, int64_t n_src, int64_t n_idx_max)
{
    int rc = check_params(p, "grav_eval_workspace_bytes");
    if (rc) return rc;
    if (n_src < 0 || n_idx_max < 0 || n_src > INT32_MAX || n_idx_max > INT32_MAX)
        return fail(GRAV_EINVAL, "grav_eval_workspace_bytes: sizes outside [0, 2^31)");
    int index = 0;
    const EvalConfig *c = resolve(p, &index);
    Layout L;
    rc = make_layout(p, c, n_src, n_idx_max, &L);
    if (rc) return rc;
    return L.total;
}

extern "C" int grav_eval_active(const grav_params *p, int64_t n_src, const double *pos,
                                const double *vel, const double *mass, const int32_t *idx,
                                const int32_t *n_idx_dev, int64_t n_idx_max, double *acc,
                                double *jerk, double *tidal, double *pot, double *dt_grav,
                                int32_t *flags_dev, void *workspace, int64_t workspace_bytes,
                                void *stream)
{
    static const char *who = "grav_eval_active";
    int rc = check_params(p, who);
    if (rc) return rc;
    if (n_src < 0 || n_idx_max < 0 || n_src > INT32_MAX || n_idx_max > INT32_MAX)
        return fail(GRAV_EINVAL, "%s: sizes outside [0, 2^31)", who);
    if (!idx && n_idx_max != n_src)
        return fail(GRAV_EINVAL, "%s: idx is NULL but n_idx_max != n_src", who);
    if (n_src == 0 || n_idx_max == 0) return GRAV_OK;
    if (!pos || !vel || !mass || !acc || !jerk || !tidal)
        return fail(GRAV_EINVAL, "%s: null input or output array", who);
    if (p->want_pot && !pot) return fail(GRAV_EINVAL, "%s: want_pot set but pot is NULL", who);
    if (!workspace) return fail(GRAV_EINVAL, "%s: null workspace", who);
    if (!aligned(workspace, 256)) return fail(GRAV_EINVAL, "%s: workspace not 256-byte aligned", who);
    int index = 0;
    const EvalConfig *c = resolve(p, &index);
    Layout L;
    rc = make_layout(p, c, n_src, n_idx_max, &L);
    if (rc) return rc;
    if (workspace_bytes < L.total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)L.total);
    const bool want_pot = p->want_pot != 0;
    int grid = 0;
    rc = grid_for(c, index, want_pot, &grid);
    if (rc) return rc;

    char *ws = static_cast<char *>(workspace);
    EvalArgs a;
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
    a.pos = pos;
    a.vel = vel;
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

    cudaStream_t st = as_stream(stream);
    c->pack(n_src, pos, vel, mass, const_cast<TileGeom *>(a.geo), const_cast<void *>(a.src), flags_dev,
            (int)L.n_tiles, st);
    rc = check_launch("grav_eval_active/pack");
    if (rc) return rc;
    c->launch[want_pot ? 1 : 0](a, grid, st);
    rc = check_launch("grav_eval_active/eval");
    if (rc) return rc;
    const int32_t BT = c->threads * c->kt;
    bool need_reduce = L.part_cap_rows > 0;
    if (need_reduce && !n_idx_dev) {
        int64_t n_tb = (n_idx_max + BT - 1) / BT;
        need_reduce = choose_split(n_tb, a.n_tiles, grid, a.max_split, a.part_cap_rows, BT) > 1;
    }
    if (need_reduce) {
        int blocks = (int)((n_idx_max + 255) / 256);
        launch_reduce(a, BT, want_pot, c->precision == GRAV_MIXED, blocks, st);
        rc = check_launch("grav_eval_active/reduce");
        if (rc) return rc;
    }
    return GRAV_OK;
}
