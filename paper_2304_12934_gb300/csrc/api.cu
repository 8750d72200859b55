// C ABI entry points (include/nufft_radon.h): argument checks, chunking of
// batches larger than the plan's scratch, and the MBIR driver loops.  All
// compute runs in the kernels of radon_kernels.cu and mbir_kernels.cu.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"

int tc_plan_build(const tc_geom *geom, int max_batch, tc_plan **out);
void tc_plan_free(tc_plan *p);

namespace {

thread_local std::string g_detail;

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Switches to the plan's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t img_elems(const tc_plan *p) { return (size_t)p->k.N * p->k.N; }
size_t sino_elems(const tc_plan *p) { return (size_t)p->k.A * p->k.D; }

int check_ptrs(std::initializer_list<const void *> req, std::initializer_list<const void *> opt) {
    for (const void *q : req)
        if (!q || !aligned16(q)) return TC_ERR_INVALID_ARG;
    for (const void *q : opt)
        if (q && !aligned16(q)) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

// grad = A^T W (A x - b) + lambda grad H(x); scal[SC_DATA], scal[SC_PRIOR] set.
int grad_impl(tc_plan *p, const float *x, const float *b, const float *w,
              const tc_prior *prior, float *grad, int batch, cudaStream_t s,
              bool want_prior_value = true) {
    TC_CUDA(cudaMemsetAsync(p->scal + SC_DATA, 0, 2 * sizeof(double), s));
    const size_t ni = img_elems(p), ns = sino_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->max_batch) {
        const int nb = batch - c0 < p->max_batch ? batch - c0 : p->max_batch;
        int rc = launch_radon_fwd_chunk(p, x + c0 * ni, nullptr, nb, b ? b + c0 * ns : nullptr,
                                        w ? w + c0 * ns : nullptr, p->sr, p->scal + SC_DATA, s);
        if (rc) return rc;
        rc = launch_radon_adj_chunk(p, p->sr, grad + c0 * ni, nb, s);
        if (rc) return rc;
    }
    if (prior && prior->lambda != 0.0) {
        int rc = launch_prior_grad(p, x, grad, batch, prior,
                                   want_prior_value ? p->scal + SC_PRIOR : nullptr, s);
        if (rc) return rc;
    }
    return TC_OK;
}

int check_prior(const tc_prior *pr) {
    if (!pr) return TC_OK;
    if (!(pr->dims == 2 || pr->dims == 3) || !(pr->sigma > 0) || !(pr->c > 0) ||
        !(pr->p >= 1.0 && pr->p <= 2.0) || !(pr->lambda >= 0))
        return TC_ERR_INVALID_ARG;
    return TC_OK;
}

}  // namespace

int tc_cuda_fail(cudaError_t e, const char *where) {
    g_detail = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return TC_ERR_OOM;
    }
    return TC_ERR_CUDA;
}

extern "C" {

const char *tc_status_string(int status) {
    switch (status) {
        case TC_OK: return "ok";
        case TC_ERR_INVALID_ARG: return "invalid argument";
        case TC_ERR_OOM: return "out of memory";
        case TC_ERR_CUDA: return "CUDA error";
        case TC_ERR_TIMEOUT: return "device wait timed out";
        case TC_ERR_UNSUPPORTED: return "unsupported parameters";
        default: return "unknown status";
    }
}

const char *tc_last_error_detail(void) { return g_detail.c_str(); }

int tc_plan_create(const tc_geom *geom, int max_batch, tc_plan **out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!geom) return TC_ERR_INVALID_ARG;
    const int N = geom->n, A = geom->n_angles, D = geom->n_det, w = geom->kernel_width;
    if (N < 16 || N > 4096 || (N & (N - 1)) || A < 1 || D < 4 || D > 16384 || (D & 1) ||
        geom->oversample != 2 || w < 2 || w > 8 || max_batch < 1 || max_batch > 65535)
        return TC_ERR_INVALID_ARG;
    if ((long long)A * (D / 2 + 1) >= (1LL << 31) / 8) return TC_ERR_UNSUPPORTED;
    g_detail.clear();
    return tc_plan_build(geom, max_batch, out);
}

int tc_plan_destroy(tc_plan *plan) {
    if (!plan) return TC_OK;
    DeviceGuard dg(plan->device);
    cudaDeviceSynchronize();
    tc_plan_free(plan);
    return TC_OK;
}

long long tc_plan_device_bytes(const tc_plan *plan) { return plan ? plan->bytes : 0; }

int radon_fwd(tc_plan *p, const float *x, float *y, int batch, void *stream) {
    if (!p || batch < 0) return TC_ERR_INVALID_ARG;
    if (batch == 0) return TC_OK;
    if (check_ptrs({x, y}, {})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ni = img_elems(p), ns = sino_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->max_batch) {
        const int nb = batch - c0 < p->max_batch ? batch - c0 : p->max_batch;
        int rc = launch_radon_fwd_chunk(p, x + c0 * ni, y + c0 * ns, nb, nullptr, nullptr,
                                        nullptr, nullptr, s);
        if (rc) return rc;
    }
    return TC_OK;
}

int radon_adj(tc_plan *p, const float *y, float *x, int batch, void *stream) {
    if (!p || batch < 0) return TC_ERR_INVALID_ARG;
    if (batch == 0) return TC_OK;
    if (check_ptrs({x, y}, {})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ni = img_elems(p), ns = sino_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->max_batch) {
        const int nb = batch - c0 < p->max_batch ? batch - c0 : p->max_batch;
        int rc = launch_radon_adj_chunk(p, y + c0 * ns, x + c0 * ni, nb, s);
        if (rc) return rc;
    }
    return TC_OK;
}

int mbir_grad(tc_plan *p, const float *x, const float *b, const float *w,
              const tc_prior *prior, float *grad, double *obj, int batch, void *stream) {
    if (!p || batch < 0 || check_prior(prior)) return TC_ERR_INVALID_ARG;
    if (batch == 0) return TC_OK;
    if (check_ptrs({x, b, grad}, {w, obj})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = grad_impl(p, x, b, w, prior, grad, batch, s);
    if (rc) return rc;
    if (obj) TC_CUDA(cudaMemcpyAsync(obj, p->scal + SC_DATA, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return TC_OK;
}

int mbir_power_norm(tc_plan *p, const float *w, float *v, float *work, int batch,
                    int n_iter, double *lam_out, void *stream) {
    if (!p || batch < 1 || n_iter < 1 || !lam_out) return TC_ERR_INVALID_ARG;
    if (check_ptrs({v, work}, {w})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = img_elems(p) * batch;
    int rc;
    if ((rc = launch_dot(p, v, v, n, p->scal + SC_NORM, s))) return rc;
    if ((rc = launch_scale_by_inv_sqrt(v, n, p->scal + SC_NORM, s))) return rc;
    for (int it = 0; it < n_iter; ++it) {
        if ((rc = grad_impl(p, v, nullptr, w, nullptr, work, batch, s))) return rc;
        if ((rc = launch_dot(p, v, work, n, p->scal + SC_DOT_GZX, s))) return rc;
        if ((rc = launch_dot(p, work, work, n, p->scal + SC_NORM, s))) return rc;
        if ((rc = launch_copy(v, work, n, s))) return rc;
        if ((rc = launch_scale_by_inv_sqrt(v, n, p->scal + SC_NORM, s))) return rc;
    }
    double lam = 0.0;
    TC_CUDA(cudaMemcpyAsync(&lam, p->scal + SC_DOT_GZX, sizeof(double), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    *lam_out = lam;
    return TC_OK;
}

int mbir_solve(tc_plan *p, const float *b, const float *w, float *x, int batch,
               const tc_prior *prior, const tc_solve_opts *opts, tc_solve_state *st,
               void *stream) {
    if (!p || !opts || !st || batch < 1 || opts->n_iter < 0 || !(opts->step > 0) ||
        check_prior(prior))
        return TC_ERR_INVALID_ARG;
    if (check_ptrs({b, x, st->z, st->g}, {w})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = img_elems(p) * batch;
    int rc;
    if (st->k == 0) {
        if ((rc = launch_copy(st->z, x, n, s))) return rc;
        if ((rc = launch_fill_scalars_fresh(p, 1.0, 0.0, 0.0, opts->step, s))) return rc;
    } else {
        if ((rc = launch_fill_scalars_fresh(p, st->t, (double)st->k, (double)st->n_restarts,
                                            opts->step, s)))
            return rc;
    }
    for (int it = 0; it < opts->n_iter; ++it) {
        // the prior's value H is only reported for the last gradient point
        if ((rc = grad_impl(p, st->z, b, w, prior, st->g, batch, s, it == opts->n_iter - 1))) return rc;
        if ((rc = launch_dots_gzx_gg(p, st->g, st->z, x, n, s))) return rc;
        if ((rc = launch_solver_scalar(p, opts->restart, s))) return rc;
        if ((rc = launch_update(p, x, st->z, st->g, n, s))) return rc;
    }
    double sc[SC_COUNT];
    TC_CUDA(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    st->t = sc[SC_T];
    st->k = (int)sc[SC_K];
    st->n_restarts = (int)sc[SC_RESTARTS];
    if (opts->n_iter > 0) {
        st->obj[0] = sc[SC_DATA];
        st->obj[1] = (prior && prior->lambda != 0.0) ? sc[SC_PRIOR] : 0.0;
    }
    return TC_OK;
}

int mbir_solve_host(tc_plan *p, const float *b_host, const float *w_host, float *x_host,
                    float *dev_b, float *dev_w, float *dev_x, int batch,
                    const tc_prior *prior, const tc_solve_opts *opts,
                    tc_solve_state *st, void *stream) {
    if (!p || batch < 1 || !b_host || !x_host || !dev_b || !dev_x || (w_host && !dev_w))
        return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ni = img_elems(p) * batch, ns = sino_elems(p) * batch;
    TC_CUDA(cudaMemcpyAsync(dev_b, b_host, ns * sizeof(float), cudaMemcpyHostToDevice, s));
    if (w_host) TC_CUDA(cudaMemcpyAsync(dev_w, w_host, ns * sizeof(float), cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaMemcpyAsync(dev_x, x_host, ni * sizeof(float), cudaMemcpyHostToDevice, s));
    int rc = mbir_solve(p, dev_b, w_host ? dev_w : nullptr, dev_x, batch, prior, opts, st, stream);
    if (rc) return rc;
    TC_CUDA(cudaMemcpyAsync(x_host, dev_x, ni * sizeof(float), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

}  // extern "C"
