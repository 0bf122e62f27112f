// Per-element supports for adaptive softening (Section 3: fully adaptive
// gravitational softening with the energy-conserving correction terms of
// Price & Monaghan 2007).
//
// Each element's support h_i solves (4 pi / 3) h_i^3 rho_i(h_i) = n_ngb m_i
// with rho_i = sum_j m_j W(r_ij, h_i), the self term included.  F(h) =
// (4 pi / 3) h^3 rho(h) - n_ngb m_i is non-decreasing in h, so each element
// runs Newton iterations kept inside a bracket [lo, hi]: a step that leaves
// the bracket doubles h (no upper end yet) or bisects.  The iteration stops
// when |F| <= tol * n_ngb * m_i; the sums of that last pass give
//   Omega_i = 1 + h_i rho_h,i / (3 rho_i),   rho_h = sum_j m_j dW/dh,
//   zeta_i  = -h_i psi_h,i / (3 rho_i Omega_i),  psi_h = sum_{j != i} m_j dpsi/dh,
// the coefficient of the correction term the force kernels add.
//
// One thread per element, 128 per CTA.  Sources are packed once into tiles
// of 128: FP64 position and mass, FP32 offsets from the tile's centre, and an
// outward-rounded FP32 bounding box.  In every pass a CTA tests all tile boxes
// against its own box grown by the largest support still iterating (one tile
// per thread, compacted by ballot); for each such tile a thread skips it when
// its own element is farther than h from the box, and otherwise pre-filters
// every source with an FP32 distance test that carries an explicit bound on
// its rounding, so the FP64 sums (the distance test that decides, W, dW/dh,
// dpsi/dh) run only for candidate neighbours.  Newton steps are limited to a
// factor of 2 in h.  Every loop is bounded by max_iter passes.
#include <cmath>

#include "grav_common.cuh"

namespace grav {
namespace {

constexpr int kSoftNT = 128;   // threads (elements) per CTA
constexpr int kSoftS = 128;    // sources per tile
static_assert(kSoftNT == kSoftS, "each thread stages one source of a tile");

struct SoftBox {
    float lo[3], hi[3];
    double c[3];      // centre of the FP64 box; the FP32 offsets are taken from it
    float ext;        // largest |x - c| component over the tile, rounded up
    float pad;
};

struct SoftArgs {
    int64_t n;
    const double *pos;
    const double *mass;
    const SoftBox *box;
    const double4 *src;        // [tile][S] (x, y, z, m)
    const float4 *src32;       // [tile][S] FP32 (x - c, y - c, z - c, 0)
    int64_t n_tiles;
    double n_ngb, tol;
    int32_t max_iter;
    double *h;
    double *zeta, *omega;      // nullable
    int32_t *iters;            // nullable
    int32_t *flags;
};

__global__ void __launch_bounds__(kSoftS) soft_pack_kernel(SoftArgs a)
{
    __shared__ float slo[3][kSoftS / 32], shi[3][kSoftS / 32];
    __shared__ double dlo[3][kSoftS / 32], dhi[3][kSoftS / 32];
    __shared__ double cen[3];
    __shared__ float sext[kSoftS / 32];
    const int64_t t = blockIdx.x;
    const int64_t j = t * kSoftS + threadIdx.x;
    double4 v = make_double4(0.0, 0.0, 0.0, 0.0);
    float lo[3], hi[3];
    const float inf = __int_as_float(0x7f800000);
    if (j < a.n) {
        v = make_double4(a.pos[3 * j], a.pos[3 * j + 1], a.pos[3 * j + 2], a.mass[j]);
        if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w))
            flag_or(a.flags, GRAV_FLAG_NONFINITE);
        lo[0] = __double2float_rd(v.x);
        lo[1] = __double2float_rd(v.y);
        lo[2] = __double2float_rd(v.z);
        hi[0] = __double2float_ru(v.x);
        hi[1] = __double2float_ru(v.y);
        hi[2] = __double2float_ru(v.z);
    } else {
        for (int c = 0; c < 3; ++c) {
            lo[c] = inf;
            hi[c] = -inf;
        }
        v.x = 1.0e300;          // padding: m = 0, never within a support
    }
    const_cast<double4 *>(a.src)[j] = v;
    const bool real = j < a.n;
    const double x[3] = {v.x, v.y, v.z};
    double xl[3], xh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xl[c] = real ? x[c] : 1.0e300;
        xh[c] = real ? x[c] : -1.0e300;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
            xl[c] = fmin(xl[c], __shfl_xor_sync(0xffffffffu, xl[c], o));
            xh[c] = fmax(xh[c], __shfl_xor_sync(0xffffffffu, xh[c], o));
        }
        if ((threadIdx.x & 31) == 0) {
            slo[c][threadIdx.x >> 5] = lo[c];
            shi[c][threadIdx.x >> 5] = hi[c];
            dlo[c][threadIdx.x >> 5] = xl[c];
            dhi[c][threadIdx.x >> 5] = xh[c];
        }
    }
    __syncthreads();
    SoftBox *b = const_cast<SoftBox *>(a.box) + t;
    if (threadIdx.x < 3) {
        float l = slo[threadIdx.x][0], h = shi[threadIdx.x][0];
        double L = dlo[threadIdx.x][0], H = dhi[threadIdx.x][0];
        for (int w = 1; w < kSoftS / 32; ++w) {
            l = fminf(l, slo[threadIdx.x][w]);
            h = fmaxf(h, shi[threadIdx.x][w]);
            L = fmin(L, dlo[threadIdx.x][w]);
            H = fmax(H, dhi[threadIdx.x][w]);
        }
        b->lo[threadIdx.x] = l;
        b->hi[threadIdx.x] = h;
        const double cc = 0.5 * (L + H);
        b->c[threadIdx.x] = cc;
        cen[threadIdx.x] = cc;
    }
    __syncthreads();
    // FP32 offsets from the centre and the largest offset component
    float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float e = 0.0f;
    if (real) {
        o = make_float4(__double2float_rn(v.x - cen[0]), __double2float_rn(v.y - cen[1]),
                        __double2float_rn(v.z - cen[2]), 0.0f);
        e = fmaxf(fabsf(o.x), fmaxf(fabsf(o.y), fabsf(o.z)));
    } else {
        o.x = 3.0e38f;            // padding: beyond every support
    }
    const_cast<float4 *>(a.src32)[j] = o;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, k));
    if ((threadIdx.x & 31) == 0) sext[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = sext[0];
        for (int w = 1; w < kSoftS / 32; ++w) m = fmaxf(m, sext[w]);
        b->ext = __fmul_ru(m, 1.0f + 0x1p-20f);
        b->pad = 0.0f;
    }
}

// W(r,h) = 8/(pi h^3) w(u), u = r/h, and dW/dh, dpsi/dh of the potential
// kernel psi(r,h) = p(u)/h (dpsi/dh = -(u p)'(u) / h^2); u < 1.
__device__ __forceinline__ void density_terms(double u, double hinv, double &w, double &w_h,
                                              double &psi_h)
{
    const double c = (8.0 / 3.14159265358979323846) * hinv * hinv * hinv;
    double wu, dwu, dup;
    const double u2 = u * u;
    if (u < 0.5) {
        wu = 1.0 + u2 * (6.0 * u - 6.0);
        dwu = u * (18.0 * u - 12.0);
        dup = 2.8 + u2 * (-16.0 + u2 * (48.0 - 38.4 * u));
    } else {
        const double q = 1.0 - u;
        wu = 2.0 * q * q * q;
        dwu = -6.0 * q * q;
        dup = 3.2 + u2 * (-32.0 + u * (64.0 + u * (-48.0 + 12.8 * u)));
    }
    w = c * wu;
    w_h = -c * hinv * (3.0 * wu + u * dwu);
    psi_h = -dup * hinv * hinv;
}

// Does a box grown by H touch the tile box?  (outward-rounded: never a false no)
__device__ __forceinline__ bool box_near(const float blo[3], const float bhi[3], const SoftBox &t,
                                         float H)
{
    float d2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(t.lo[c], bhi[c]), __fsub_rd(blo[c], t.hi[c])));
        d2 = __fmaf_rd(gap, gap, d2);
    }
    return d2 < __fmul_ru(H, H);
}

__global__ void __launch_bounds__(kSoftNT) soft_solve_kernel(SoftArgs a)
{
    __shared__ double4 sx[kSoftS];
    __shared__ float4 sx32[kSoftS];
    __shared__ int32_t list[kSoftNT];
    __shared__ int32_t wcount[kSoftNT / 32];
    __shared__ float rlo[3][kSoftNT / 32], rhi[3][kSoftNT / 32], rh[kSoftNT / 32];
    __shared__ float blo[3], bhi[3], bh;

    const int64_t i = (int64_t)blockIdx.x * kSoftNT + threadIdx.x;
    const bool mine = i < a.n;
    double xi[3] = {0.0, 0.0, 0.0}, target = 0.0, h = 1.0;
    if (mine) {
        for (int c = 0; c < 3; ++c) xi[c] = a.pos[3 * i + c];
        target = a.n_ngb * a.mass[i];
        h = a.h[i];
    }
    bool done = !mine;
    if (mine && !(h > 0.0 && isfinite(h) && a.mass[i] > 0.0)) {
        flag_or(a.flags, GRAV_FLAG_NONFINITE);
        done = true;
    }
    double lo = 0.0, hi = __longlong_as_double(0x7ff0000000000000LL);
    int32_t it = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float inf = __int_as_float(0x7f800000);

    for (int pass = 0; pass < a.max_iter; ++pass) {
        // ---- the CTA's box and largest support over the elements still iterating ----
        float l[3], u[3], hm = done ? 0.0f : __double2float_ru(h);
        for (int c = 0; c < 3; ++c) {
            l[c] = done ? inf : __double2float_rd(xi[c]);
            u[c] = done ? -inf : __double2float_ru(xi[c]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
            for (int c = 0; c < 3; ++c) {
                l[c] = fminf(l[c], __shfl_xor_sync(0xffffffffu, l[c], o));
                u[c] = fmaxf(u[c], __shfl_xor_sync(0xffffffffu, u[c], o));
            }
        }
        if (lane == 0) {
            rh[wid] = hm;
            for (int c = 0; c < 3; ++c) {
                rlo[c][wid] = l[c];
                rhi[c][wid] = u[c];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float H = 0.0f;
            float L[3] = {inf, inf, inf}, U[3] = {-inf, -inf, -inf};
            for (int w = 0; w < kSoftNT / 32; ++w) {
                H = fmaxf(H, rh[w]);
                for (int c = 0; c < 3; ++c) {
                    L[c] = fminf(L[c], rlo[c][w]);
                    U[c] = fmaxf(U[c], rhi[c][w]);
                }
            }
            bh = H;
            for (int c = 0; c < 3; ++c) {
                blo[c] = L[c];
                bhi[c] = U[c];
            }
        }
        __syncthreads();
        if (!(bh > 0.0f)) break;                 // every element of the CTA is done
        const float B_lo[3] = {blo[0], blo[1], blo[2]}, B_hi[3] = {bhi[0], bhi[1], bhi[2]};
        const float H = bh;

        // ---- sums at the current supports over the tiles that can reach ----
        double rho = 0.0, rho_h = 0.0, psi_h = 0.0;
        const double hinv = 1.0 / h, h2 = h * h;
        const float hf = __double2float_ru(h);
        const float hlim2 = __fmul_ru(hf, hf);
        for (int64_t t0 = 0; t0 < a.n_tiles; t0 += kSoftNT) {
            const int64_t tt = t0 + threadIdx.x;
            const bool near = tt < a.n_tiles && box_near(B_lo, B_hi, a.box[tt], H);
            const uint32_t bal = __ballot_sync(0xffffffffu, near);
            if (lane == 0) wcount[wid] = __popc(bal);
            __syncthreads();
            int base = 0, total = 0;
            for (int w = 0; w < kSoftNT / 32; ++w) {
                if (w < wid) base += wcount[w];
                total += wcount[w];
            }
            if (near) list[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(tt - t0);
            __syncthreads();
            for (int k = 0; k < total; ++k) {
                const int64_t t = t0 + list[k];
                sx[threadIdx.x] = a.src[t * kSoftS + threadIdx.x];   // kSoftNT == kSoftS
                sx32[threadIdx.x] = a.src32[t * kSoftS + threadIdx.x];
                const SoftBox tb = a.box[t];
                __syncthreads();
                if (!done) {
                    // own offset from the tile centre (FP64, rounded once) and
                    // a lower bound of the distance to the tile's box
                    float tq[3], tmax = 0.0f, gap2 = 0.0f;
                    for (int c = 0; c < 3; ++c) {
                        tq[c] = __double2float_rn(xi[c] - tb.c[c]);
                        tmax = fmaxf(tmax, fabsf(tq[c]));
                        const float gap = fmaxf(0.0f, __fsub_rd(__fsub_rd(fabsf(tq[c]), tb.ext),
                                                                 __fmul_ru(fabsf(tq[c]), 0x1p-22f)));
                        gap2 = __fmaf_rd(gap, gap, gap2);
                    }
                    if (gap2 < hlim2) {
                        // |d32 - d| <= err per component: both offsets were
                        // rounded once and their difference once more
                        const float err = __fmul_ru(__fadd_ru(tb.ext, tmax), 0x1p-21f);
                        const float hl = __fadd_ru(hf, __fmul_ru(err, 1.8f));
                        const float lim = __fmul_ru(__fmul_ru(hl, hl), 1.0f + 0x1p-20f);
                        for (int j = 0; j < kSoftS; ++j) {
                            const float4 q = sx32[j];
                            const float ex = q.x - tq[0], ey = q.y - tq[1], ez = q.z - tq[2];
                            if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) >= lim) continue;
                            const double4 s = sx[j];
                            const double dx = s.x - xi[0], dy = s.y - xi[1], dz = s.z - xi[2];
                            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                            if (r2 < h2) {
                                double w, wh, ph;
                                density_terms(sqrt(r2) * hinv, hinv, w, wh, ph);
                                rho = fma(s.w, w, rho);
                                rho_h = fma(s.w, wh, rho_h);
                                if (t * kSoftS + j != i) psi_h = fma(s.w, ph, psi_h);
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }

        // ---- test and Newton step ----
        if (!done) {
            const double vol = (4.0 * 3.14159265358979323846 / 3.0) * h * h * h;
            const double F = vol * rho - target;
            bool finish = fabs(F) <= a.tol * target;
            if (!finish && it + 1 >= a.max_iter) {
                flag_or(a.flags, GRAV_FLAG_NOCONVERGE);
                it = -1;
                finish = true;
            }
            if (finish) {
                const double om = 1.0 + h * rho_h / (3.0 * rho);
                a.h[i] = h;
                if (a.omega) a.omega[i] = om;
                if (a.zeta) a.zeta[i] = -h * psi_h / (3.0 * rho * om);
                if (a.iters) a.iters[i] = it;
                done = true;
            } else {
                if (F < 0.0) lo = h; else hi = h;
                const double dF = 4.0 * 3.14159265358979323846 * h * h * rho + vol * rho_h;
                // Newton step limited to a factor of 2 (flat F when only the
                // self term lies inside), then kept inside the bracket
                double hn = F < 0.0 ? 2.0 * h : 0.5 * h;
                if (dF > 0.0) hn = fmin(fmax(h - F / dF, 0.5 * h), 2.0 * h);
                if (!(hn > lo && hn < hi)) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
                h = hn;
                ++it;
            }
        }
    }
    if (!done) {
        // the pass limit ran out first (only when max_iter passes all moved h)
        flag_or(a.flags, GRAV_FLAG_NOCONVERGE);
        a.h[i] = h;
        if (a.iters) a.iters[i] = -1;
    }
}

int soft_layout(int64_t n, int64_t *box_off, int64_t *src_off, int64_t *src32_off, int64_t *total)
{
    const int64_t n_tiles = (n + kSoftS - 1) / kSoftS;
    *box_off = 0;
    *src_off = round_up(n_tiles * (int64_t)sizeof(SoftBox), 256);
    *src32_off = *src_off + round_up(n_tiles * kSoftS * (int64_t)sizeof(double4), 256);
    *total = std::max<int64_t>(256, *src32_off + round_up(n_tiles * kSoftS * (int64_t)sizeof(float4), 256));
    return GRAV_OK;
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int64_t grav_soft_workspace_bytes(int64_t n)
{
    if (n < 0 || n > INT32_MAX) return fail(GRAV_EINVAL, "grav_soft_workspace_bytes: n outside [0, 2^31)");
    int64_t b, s, s32, t;
    soft_layout(n, &b, &s, &s32, &t);
    return t;
}

extern "C" int grav_soft_solve(const grav_soft_params *sp, int64_t n, const double *pos,
                               const double *mass, double *h_inout, double *zeta_out,
                               double *omega_out, int32_t *iters_out, int32_t *flags_dev,
                               void *workspace, int64_t workspace_bytes, void *stream)
{
    static const char *who = "grav_soft_solve";
    if (!sp) return fail(GRAV_EINVAL, "%s: null parameters", who);
    if (!(sp->n_ngb > 32.0 / 3.0) || !std::isfinite(sp->n_ngb))
        return fail(GRAV_EINVAL, "%s: n_ngb must be finite and above 32/3 (the self term)", who);
    if (!(sp->tol >= 1e-15 && sp->tol < 1.0))
        return fail(GRAV_EINVAL, "%s: tol outside [1e-15, 1)", who);
    if (sp->max_iter < 1 || sp->max_iter > 10000)
        return fail(GRAV_EINVAL, "%s: max_iter outside [1, 10000]", who);
    if (n < 0 || n > INT32_MAX) return fail(GRAV_EINVAL, "%s: n outside [0, 2^31)", who);
    if (n == 0) return GRAV_OK;
    if (!pos || !mass || !h_inout) return fail(GRAV_EINVAL, "%s: null pos, mass or h", who);
    if (!workspace || !aligned(workspace, 256))
        return fail(GRAV_EINVAL, "%s: workspace null or not 256-byte aligned", who);
    int64_t box_off, src_off, src32_off, total;
    soft_layout(n, &box_off, &src_off, &src32_off, &total);
    if (workspace_bytes < total)
        return fail(GRAV_ENOMEM, "%s: workspace of %lld bytes < %lld", who, (long long)workspace_bytes,
                    (long long)total);
    char *ws = static_cast<char *>(workspace);
    SoftArgs a;
    a.n = n;
    a.pos = pos;
    a.mass = mass;
    a.box = reinterpret_cast<const SoftBox *>(ws + box_off);
    a.src = reinterpret_cast<const double4 *>(ws + src_off);
    a.src32 = reinterpret_cast<const float4 *>(ws + src32_off);
    a.n_tiles = (n + kSoftS - 1) / kSoftS;
    a.n_ngb = sp->n_ngb;
    a.tol = sp->tol;
    a.max_iter = sp->max_iter;
    a.h = h_inout;
    a.zeta = zeta_out;
    a.omega = omega_out;
    a.iters = iters_out;
    a.flags = flags_dev;
    cudaStream_t st = as_stream(stream);
    soft_pack_kernel<<<(unsigned)a.n_tiles, kSoftS, 0, st>>>(a);
    int rc = check_launch("grav_soft_solve/pack");
    if (rc) return rc;
    soft_solve_kernel<<<(unsigned)((n + kSoftNT - 1) / kSoftNT), kSoftNT, 0, st>>>(a);
    return check_launch("grav_soft_solve/solve");
}
