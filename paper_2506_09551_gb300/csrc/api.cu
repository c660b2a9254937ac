// C ABI plumbing: error reporting, device checks, defaults, version.
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "msbicg_impl.cuh"

namespace msb {

thread_local int64_t g_launches = 0;
thread_local int64_t g_alloc_bytes = 0;
static thread_local std::string t_last_error;

void set_error_message(const std::string& m) { t_last_error = m; }

msb_status guard(const char* fn, const std::function<void()>& body) {
    try {
        body();
        return MSB_OK;
    } catch (const Error& e) {
        t_last_error = std::string(fn) + ": " + e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        t_last_error = std::string(fn) + ": host allocation failed";
        return MSB_ENOMEM;
    } catch (const std::exception& e) {
        t_last_error = std::string(fn) + ": " + e.what();
        return MSB_EINVAL;
    } catch (...) {
        t_last_error = std::string(fn) + ": unknown error";
        return MSB_EINVAL;
    }
}

// The library is built for sm_103a only: refuse any other device up front
// instead of failing at the first launch.
void require_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        fail(MSB_ECUDA, "no CUDA device available");
    }
    int dev = 0;
    MSB_CUDA(cudaGetDevice(&dev));
    int major = 0, minor = 0;
    MSB_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    MSB_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (major != 10 || minor != 3)
        fail(MSB_ECUDA, "this build targets sm_103a (GB300); device has compute capability " +
                            std::to_string(major) + "." + std::to_string(minor));
}

int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

}  // namespace msb

extern "C" const char* msb_last_error(void) { return msb::t_last_error.c_str(); }

extern "C" const char* msb_version(void) { return "msbicg 0.1 sm_103a"; }

extern "C" void msb_map_params_default(msb_map_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->Gamma = 0.3;
    p->eta = 0.1;
    p->gs_tol = 1e-12;
    p->gs_maxit = 300;
    p->solve_tol = 1e-10;
    p->maxit = 5000;
    p->cf_tol = 1e-10;
    p->cf_check = 50;
    p->cf_maxdepth = 4000;
    p->seed_index = -1;
    p->block = 0;
    p->precision = MSB_FP64;
}
