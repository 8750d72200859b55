// qGGMRF prior gradient with statically allocated scratch.
//
// Some callers cannot call cudaMalloc: a framework whose caching allocator
// owns the device memory budget, or a latency-critical pipeline that must not
// risk the implicit device synchronisation an allocation can cause.  This
// entry point computes the same prior gradient and value as the plan-based
// path (the qGGMRF of Sec. 3, Eqs. reg2 and reg3) but takes its per-block FP64
// partial sums from a fixed-size array in device global memory that the
// library declares at file scope.  That array exists on every GPU that loads
// the library, until the process exits.
#include <mutex>

#include "common.cuh"
#include "profile.cuh"

// Maximum number of per-block partials: one per CTA of the prior kernel (60
// columns x 16 rows of voxel columns, times its z chunks), enough for one z
// chunk at N = 4096 (69 x 256 = 17664 blocks); the launch cuts the z chunks
// to what fits.
#define TC_NOALLOC_PARTIALS 65536

static __device__ __align__(256) double g_noalloc_partials[TC_NOALLOC_PARTIALS];

int launch_prior_kernel_into(const float *x, float *g, int n, int nb, const tc_prior *pr,
                             double *partials, int max_partials, double *h_out,
                             cudaStream_t s);
int prior_configure_kernels();

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device (looked up once
// per device, with that device current).
int noalloc_scratch(double **out) {
    int dev = -1;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        TC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_partials));
        const int rc = prior_configure_kernels();   // nothing to opt into today; kept for future kernels
        if (rc) return rc;
        g_addr[dev] = static_cast<double *>(ptr);
    }
    *out = g_addr[dev];
    return TC_OK;
}

}  // namespace

extern "C" int tc_prior_grad_noalloc(const float *x, float *grad, int n, int batch,
                                     const tc_prior *prior, double *h_out, void *stream) {
    if (!x || !grad || !prior || n < 1 || n > 4096 || batch < 1 || batch > 65535) return TC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(grad) & 15u))
        return TC_ERR_INVALID_ARG;
    // grad is written at one slice while other blocks still read x around it
    const uintptr_t bytes = (uintptr_t)batch * n * n * sizeof(float);
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ga = reinterpret_cast<uintptr_t>(grad);
    if (xa < ga + bytes && ga < xa + bytes) return TC_ERR_INVALID_ARG;
    if (!(prior->dims == 2 || prior->dims == 3) || !(prior->sigma > 0) || !(prior->c > 0) ||
        !(prior->p >= 1.0 && prior->p <= 2.0) || !(prior->lambda >= 0))
        return TC_ERR_INVALID_ARG;
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    return launch_prior_kernel_into(x, grad, n, batch, prior, scratch, TC_NOALLOC_PARTIALS,
                                    h_out, (cudaStream_t)stream);
}
