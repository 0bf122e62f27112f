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
