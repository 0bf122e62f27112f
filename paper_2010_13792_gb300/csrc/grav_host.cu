// Host plumbing of libgrav: per-thread error text, CUDA status mapping,
// cached device attributes, version string.
#include <mutex>

#include "grav_common.cuh"

namespace grav {

static thread_local std::string g_error;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
}

void clear_error() { g_error.clear(); }

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GRAV_OK;
    return fail(GRAV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_launch(const char *what) { return check_cuda(cudaGetLastError(), what); }

int device_sm_count(int *out)
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return fail(GRAV_ECUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (cached[dev] == 0) {
        int v = 0;
        rc = check_cuda(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev),
                        "cudaDeviceGetAttribute");
        if (rc) return rc;
        cached[dev] = v;
    }
    *out = cached[dev];
    return GRAV_OK;
}

}  // namespace grav

extern "C" const char *grav_last_error_string(void) { return grav::g_error.c_str(); }

extern "C" const char *grav_version(void) { return "libgrav 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Failure-detection self-test: one CTA arms an mbarrier for a 16-byte
// transfer that is never issued, so the phase can never complete; its wait is
// bounded by `limit` polls, after which the kernel records GRAV_FLAG_TIMEOUT
// and returns.  No asynchronous copy is ever in flight, so returning is safe
// and the context stays usable.  This exercises the same bounded-wait path
// every TMA wait of the force kernels takes when a copy does not arrive.
// ---------------------------------------------------------------------------
namespace grav {
namespace {

__global__ void wait_timeout_selftest_kernel(int32_t *flags, uint32_t limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                     "r"(16u)
                     : "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0u, flags, limit);
}

}  // namespace
}  // namespace grav

extern "C" int grav_selftest_wait_timeout(uint32_t limit, int32_t *flags_dev, void *stream)
{
    using namespace grav;
    if (!flags_dev) return fail(GRAV_EINVAL, "grav_selftest_wait_timeout: null flags_dev");
    if (limit == 0 || limit > (1u << 20))
        return fail(GRAV_EINVAL, "grav_selftest_wait_timeout: limit outside [1, 2^20]");
    cudaStream_t st = as_stream(stream);
    wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(flags_dev, limit);
    int rc = check_launch("grav_selftest_wait_timeout");
    if (rc) return rc;
    int32_t host = 0;
    rc = check_cuda(cudaMemcpyAsync(&host, flags_dev, sizeof host, cudaMemcpyDeviceToHost, st),
                    "grav_selftest_wait_timeout: read flags");
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(st), "grav_selftest_wait_timeout: synchronize");
    if (rc) return rc;
    if (host & GRAV_FLAG_TIMEOUT) return fail(GRAV_ETIMEOUT, "bounded wait expired (self-test)");
    return GRAV_OK;
}
