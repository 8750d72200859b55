// C ABI entry points (include/nufft_radon.h): argument checks, chunking of
// batches larger than the plan's scratch, and the MBIR driver loops.  All
// compute runs in the kernels of radon_kernels.cu and mbir_kernels.cu.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

int tc_plan_build(const tc_geom *geom, int max_batch, tc_plan **out);
void tc_plan_free(tc_plan *p);
int plan_set_col_pairs(tc_plan *p, int cp);
int plan_set_spread_chunk(tc_plan *p, int chunk);

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

// scal[SC_DATA] and scal[SC_PRIOR] before the chunks add to them: zero, or
// with the normal operator (atb given) 1/2 ||b||^2 and zero.
int data_init(tc_plan *p, const float *atb, cudaStream_t s) {
    TC_CUDA(cudaMemsetAsync(p->scal + SC_DATA, 0, 2 * sizeof(double), s));
    if (atb) return launch_reduce_finalize(p->scal + SC_BB, 1, p->scal + SC_DATA, 0, 0.5, s);
    return TC_OK;
}

// Data-term gradient of one chunk of nb slices: grad = A^T W (A x - b), its
// value added to scal[SC_DATA].  With atb (= A^T b of the chunk, W = I), A^T A
// comes from the Toeplitz-plus-Hankel embedding and the value is formed only
// when want_value.
int data_grad_chunk(tc_plan *p, const float *x, const float *b, const float *w, float *grad, int nb,
                    const float *atb, bool want_value, cudaStream_t s) {
    if (atb)
        return launch_radon_normal_chunk(p, x, grad, nb, atb, want_value ? x : nullptr, p->scal + SC_DATA, s);
    int rc = launch_radon_fwd_chunk(p, x, nullptr, nb, b, w, p->sr, p->scal + SC_DATA, s);
    if (rc) return rc;
    return launch_radon_adj_chunk(p, p->sr, grad, nb, s);
}

// grad = A^T W (A x - b) + lambda grad H(x); scal[SC_DATA], scal[SC_PRIOR] set
// (with atb, the data value and the prior value only when want_value).
// ready: optional per-chunk events the chunk's first kernel waits for (slabs
// still being copied in on another stream).
// dot_x: with a prior, the prior kernel also forms the restart-test inner
// products <grad, x - dot_x> and <grad, grad>.
// atb: A^T b of the whole batch for the normal-operator data term (W = I).
// With dot_x the prior kernel leaves the next iterate in dot_x and the
// momentum point of an iteration without restart in grad (launch_prior_grad).
// x_ready: optional per-chunk events after which dot_x's slabs are resident
// (ready then only covers b and w); the prior waits for all of them.
int grad_impl(tc_plan *p, const float *x, const float *b, const float *w,
              const tc_prior *prior, float *grad, int batch, cudaStream_t s,
              bool want_value = true, const cudaEvent_t *ready = nullptr,
              float *dot_x = nullptr, double step = 0.0, const float *atb = nullptr,
              const cudaEvent_t *x_ready = nullptr) {
    int rc = data_init(p, atb, s);
    if (rc) return rc;
    const size_t ni = img_elems(p), ns = sino_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->chunk) {
        const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
        if (ready) TC_CUDA(cudaStreamWaitEvent(s, ready[c0 / p->chunk], 0));
        rc = data_grad_chunk(p, x + c0 * ni, b ? b + c0 * ns : nullptr, w ? w + c0 * ns : nullptr,
                             grad + c0 * ni, nb, atb ? atb + c0 * ni : nullptr, want_value, s);
        if (rc) return rc;
    }
    if (prior && prior->lambda != 0.0) {
        // the copy stream is in order: its last slab's event covers every slab
        if (x_ready) TC_CUDA(cudaStreamWaitEvent(s, x_ready[(batch - 1) / p->chunk], 0));
        rc = launch_prior_grad(p, x, grad, batch, prior, want_value ? p->scal + SC_PRIOR : nullptr, s, dot_x,
                               0, -1, step);
        if (rc) return rc;
    }
    return TC_OK;
}

// *data = 1/2 sum W (A x - b)^2 (FP64), *prior_val = lambda H(x) (when a
// prior with lambda != 0 is given): the objective's value without its gradient.
int value_impl(tc_plan *p, const float *x, const float *b, const float *w, const tc_prior *prior,
               int batch, double *data, double *prior_val, cudaStream_t s,
               const cudaEvent_t *ready = nullptr) {
    TC_CUDA(cudaMemsetAsync(data, 0, sizeof(double), s));
    TC_CUDA(cudaMemsetAsync(prior_val, 0, sizeof(double), s));
    const size_t ni = img_elems(p), ns = sino_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->chunk) {
        const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
        if (ready) TC_CUDA(cudaStreamWaitEvent(s, ready[c0 / p->chunk], 0));
        int rc = launch_radon_fwd_chunk(p, x + c0 * ni, nullptr, nb, b ? b + c0 * ns : nullptr,
                                        w ? w + c0 * ns : nullptr, p->sr, data, s);
        if (rc) return rc;
    }
    if (prior && prior->lambda != 0.0) return launch_prior_value(p, x, batch, prior, prior_val, s);
    return TC_OK;
}

// The plan's device status (bounded waits) after the stream has drained;
// a recorded timeout is returned once and cleared.
int take_dev_status(tc_plan *p, cudaStream_t s) {
    int st = TC_OK;
    TC_CUDA(cudaMemcpyAsync(&st, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (st != TC_OK) TC_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
    return st;
}

// Power iteration on A^T W A from v (nonzero): v := v/||v||, then n_iter times
// u = A^T W A v, lambda = <v, u>, v := u/||u|| (FP64 norms and dots on the
// device).  The last Rayleigh quotient is left in scal[SC_DOT_GZX].
int power_impl(tc_plan *p, const float *w, float *v, float *work, int batch, int n_iter,
               cudaStream_t s) {
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
    return TC_OK;
}

// Seed of the derived step's power-iteration start vector.
constexpr unsigned long long kPowerSeed = 0x230412934ull;

// The step 1/L of the solver (reading of Sec. 3: constant step):
// L = 1.05 lambda_max(A^T W A) + lambda 8 / (sigma^2 c), lambda_max by n_iter
// power iterations over the whole batch from a seeded start held in v (work:
// the second vector).  Synchronises s (the host needs the step).
int derive_step(tc_plan *p, const float *w, const tc_prior *prior, int batch, int n_iter, float *v,
                float *work, cudaStream_t s, double *step_out) {
    const size_t n = img_elems(p) * batch;
    int rc = launch_fill_start(v, n, kPowerSeed, s);
    if (!rc) rc = power_impl(p, w, v, work, batch, n_iter, s);
    if (rc) return rc;
    double lam = 0.0;
    TC_CUDA(cudaMemcpyAsync(&lam, p->scal + SC_DOT_GZX, sizeof(double), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    double L = 1.05 * lam;
    if (prior && prior->lambda != 0.0) L += prior->lambda * 8.0 / (prior->sigma * prior->sigma * prior->c);
    if (!(L > 0.0) || !std::isfinite(L)) {
        g_detail = "derived step: A^T W A has no positive eigenvalue and there is no prior";
        return TC_ERR_INVALID_ARG;
    }
    *step_out = 1.0 / L;
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

namespace {
// copies of the host-streamed solve still allowed before an injected failure
// (negative: injection off)
std::atomic<int> g_fail_copy_after{-1};
}  // namespace

int host_copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
    int left = g_fail_copy_after.load();
    while (left >= 0 && !g_fail_copy_after.compare_exchange_weak(left, left - 1)) {
    }
    if (left == 0) {
        g_detail = "cudaMemcpyAsync: failure injected by tc_test_fail_copy_after";
        return TC_ERR_CUDA;
    }
    TC_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
    return TC_OK;
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
    if (!(std::fabs(geom->center_offset) <= 0.5 * D)) return TC_ERR_INVALID_ARG;  // also rejects NaN
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
    for (int c0 = 0; c0 < batch; c0 += p->chunk) {
        const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
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
    for (int c0 = 0; c0 < batch; c0 += p->chunk) {
        const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
        int rc = launch_radon_adj_chunk(p, y + c0 * ns, x + c0 * ni, nb, s);
        if (rc) return rc;
    }
    return TC_OK;
}

int tc_plan_prepare_normal(tc_plan *p, void *stream) {
    if (!p) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    return normal_prepare(p, (cudaStream_t)stream);
}

int radon_normal(tc_plan *p, const float *x, float *x_out, int batch, void *stream) {
    if (!p || batch < 0) return TC_ERR_INVALID_ARG;
    if (batch == 0) return TC_OK;
    if (check_ptrs({x, x_out}, {})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = normal_prepare(p, s);
    if (rc) return rc;
    const size_t ni = img_elems(p);
    for (int c0 = 0; c0 < batch; c0 += p->chunk) {
        const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
        rc = launch_radon_normal_chunk(p, x + c0 * ni, x_out + c0 * ni, nb, nullptr, nullptr, nullptr, s);
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
    int rc = power_impl(p, w, v, work, batch, n_iter, s);
    if (rc) return rc;
    double lam = 0.0;
    TC_CUDA(cudaMemcpyAsync(&lam, p->scal + SC_DOT_GZX, sizeof(double), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    *lam_out = lam;
    return take_dev_status(p, s);
}

int tc_plan_status(tc_plan *p) {
    if (!p) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    TC_CUDA(cudaDeviceSynchronize());
    return take_dev_status(p, nullptr);
}

}  // extern "C"

namespace {

// The accelerated-gradient loop.  fresh_z: z := x is still to be done;
// ready: per-chunk events gating the first iteration (host streaming).
// Destination of the last iteration's x_{k+1} in a host-streamed solve.
struct HostOut {
    float *x_host;                   // [batch][N][N], host
    cudaStream_t cs;                 // copy stream
    std::vector<cudaEvent_t> *ev;    // events created here, owned by the caller
};

// Last iteration of the gradient-restart schedule with a prior, x_{k+1}
// streamed out slab by slab: x_{k+1} = z_k - step g_k needs no global scalar,
// so a slab's x_{k+1} is final once its data gradient and its prior (which
// reads a one-slice halo) are done; its copy to the host then overlaps the
// remaining chunks.  The prior kernel writes x_{k+1} over x_k and the momentum
// point of an iteration without restart over the gradient (as every fused
// iteration does); the restart test, and the copy of x_{k+1} over z_{k+1}
// after a restart, follow at the end.  Same result as the resident iteration.
// x holds x_k, z holds z_k and gb is the gradient buffer; on return x holds
// x_{k+1} and gb holds z_{k+1}.  ready: per-chunk events of the chunk's
// inputs; x_ready (optional): of x's slabs, when ready covers b and w only.
int last_iteration_streamed(tc_plan *p, const float *b, const float *w, float *x, const float *z, float *gb,
                            int batch, const tc_prior *prior, const tc_solve_opts *opts, double step,
                            cudaStream_t s, const cudaEvent_t *ready, const HostOut &out, const float *atb,
                            const cudaEvent_t *x_ready = nullptr) {
    int rc0 = data_init(p, atb, s);
    if (rc0) return rc0;
    const size_t ni = img_elems(p), ns = sino_elems(p);
    const int nslab = (batch + p->chunk - 1) / p->chunk;
    auto finish = [&](int j) -> int {
        const int z0 = j * p->chunk, z1 = z0 + p->chunk < batch ? z0 + p->chunk : batch;
        if (x_ready) TC_CUDA(cudaStreamWaitEvent(s, x_ready[j], 0));
        int rc = launch_prior_grad(p, z, gb, batch, prior, p->scal + SC_PRIOR, s, x, z0, z1, step);
        if (rc) return rc;
        cudaEvent_t e = nullptr;
        TC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        out.ev->push_back(e);
        TC_CUDA(cudaEventRecord(e, s));
        TC_CUDA(cudaStreamWaitEvent(out.cs, e, 0));
        return host_copy_async(out.x_host + z0 * ni, x + z0 * ni, (size_t)(z1 - z0) * ni * sizeof(float),
                               cudaMemcpyDeviceToHost, out.cs);
    };
    for (int c = 0; c < nslab; ++c) {
        const int c0 = c * p->chunk, nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
        if (ready) TC_CUDA(cudaStreamWaitEvent(s, ready[c], 0));
        int rc = data_grad_chunk(p, z + c0 * ni, b + c0 * ns, w ? w + c0 * ns : nullptr, gb + c0 * ni, nb,
                                 atb ? atb + c0 * ni : nullptr, true, s);
        if (!rc && c > 0) rc = finish(c - 1);  // slab c holds the upper halo of slab c - 1
        if (rc) return rc;
    }
    int rc = finish(nslab - 1);
    if (!rc) rc = launch_solver_scalar(p, opts->restart, s);
    if (!rc && opts->restart == 1) rc = launch_restart_fixup(p, gb, x, img_elems(p) * batch, s);
    return rc;
}

// ready: per-chunk events gating the first iteration (host streaming), after
// which the chunk's b, w and x are resident; ready_bw (optional, z resident
// already): after which its b and w are, so the chunk's data gradient can
// start before its x arrives (only the prior reads x).
int solve_loop(tc_plan *p, const float *b, const float *w, float *x, int batch,
               const tc_prior *prior, const tc_solve_opts *opts, tc_solve_state *st,
               cudaStream_t s, bool fresh_z, const cudaEvent_t *ready, const HostOut *out = nullptr,
               const cudaEvent_t *ready_bw = nullptr) {
    const size_t n = img_elems(p) * batch;
    int rc;
    // the step: given, derived now (fresh solves only: z and g are free), or
    // the one a previous call derived
    double step = opts->step;
    if (!(step > 0.0)) {
        if (st->k == 0) {
            const int pit = opts->power_iter > 0 ? opts->power_iter : 30;
            if ((rc = derive_step(p, opts->normal ? nullptr : w, prior, batch, pit, st->z, st->g, s, &step)))
                return rc;
        } else {
            step = st->step;
        }
    }
    st->step = step;
    if (st->k == 0) {
        if (fresh_z && (rc = launch_copy(st->z, x, n, s))) return rc;
        if ((rc = launch_fill_scalars_fresh(p, 1.0, 0.0, 0.0, step, s))) return rc;
    } else {
        if ((rc = launch_fill_scalars_fresh(p, st->t, (double)st->k, (double)st->n_restarts,
                                            step, s)))
            return rc;
    }
    const float *atb = nullptr;
    if (opts->normal) {
        // A^T b and ||b||^2 once per call; the chunks wait for their slabs here
        if ((rc = normal_prepare(p, s))) return rc;
        const size_t ns = sino_elems(p), ni = img_elems(p);
        for (int c0 = 0; c0 < batch; c0 += p->chunk) {
            const int nb = batch - c0 < p->chunk ? batch - c0 : p->chunk;
            if (ready) TC_CUDA(cudaStreamWaitEvent(s, ready[c0 / p->chunk], 0));
            if ((rc = launch_radon_adj_chunk(p, b + c0 * ns, st->atb + c0 * ni, nb, s))) return rc;
        }
        if ((rc = launch_dot(p, b, b, ns * batch, p->scal + SC_BB, s))) return rc;
        atb = st->atb;
        ready = nullptr;
        ready_bw = nullptr;
    }
    if (opts->restart == 2) {
        // Monotone variant.  Phi(x_k) is recomputed at the start of every call
        // (deterministically), so a resumed solve matches an uninterrupted one.
        if (opts->n_iter > 0) {
            if ((rc = value_impl(p, x, b, w, prior, batch, p->scal + SC_DATA_X, p->scal + SC_PRIOR_X, s,
                                 ready)))
                return rc;
        }
        for (int it = 0; it < opts->n_iter; ++it) {
            if ((rc = grad_impl(p, st->z, b, w, prior, st->g, batch, s, false)))  // g = grad Phi(z_k)
                return rc;
            if ((rc = launch_step_to_candidate(p, st->z, st->g, n, s))) return rc;  // g := v
            if ((rc = value_impl(p, st->g, b, w, prior, batch, p->scal + SC_DATA_V, p->scal + SC_PRIOR_V, s)))
                return rc;
            if ((rc = launch_monotone_scalar(p, s))) return rc;
            if ((rc = launch_update_monotone(p, x, st->z, st->g, n, s))) return rc;
        }
    }
    if (prior && prior->lambda != 0.0 && opts->restart != 2) {
        // Gradient restart or plain momentum with a prior: the prior kernel
        // forms the restart dots, writes x_{k+1} = z_k - step g over x_k (x
        // always holds the iterate) and the momentum point of an iteration
        // without restart, x_{k+1} + beta (x_{k+1} - x_k), over the gradient.
        // z_{k+1} is thus made where the gradient was, and the buffer of z_k
        // takes the next gradient: no update pass.  After a restart (beta = 0)
        // a check-and-copy kernel sets z_{k+1} = x_{k+1}.
        float *zc = st->z, *gc = st->g;
        for (int it = 0; it < opts->n_iter; ++it) {
            const bool last = it == opts->n_iter - 1;  // the prior's value H is reported for the last point
            // the first iteration's chunks wait for their b and w (ready_bw) or
            // all their inputs (ready); with ready_bw the priors wait for x
            const cudaEvent_t *rd = it == 0 ? (ready_bw ? ready_bw : ready) : nullptr;
            const cudaEvent_t *rx = it == 0 && ready_bw ? ready : nullptr;
            if (out && last) {
                rc = last_iteration_streamed(p, b, w, x, zc, gc, batch, prior, opts, step, s, rd, *out, atb, rx);
            } else {
                rc = grad_impl(p, zc, b, w, prior, gc, batch, s, last, rd, x, step, atb, rx);
                if (!rc) rc = launch_solver_scalar(p, opts->restart, s);
                if (!rc && opts->restart == 1) rc = launch_restart_fixup(p, gc, x, n, s);
            }
            if (rc) return rc;
            float *t = zc;
            zc = gc;
            gc = t;
        }
        // z_k ends in one of the two caller buffers: the state names it
        if (zc != st->z) {
            st->g = st->z;
            st->z = zc;
        }
    } else {
        // no prior: separate restart dots and update
        for (int it = 0; it < (opts->restart == 2 ? 0 : opts->n_iter); ++it) {
            if ((rc = grad_impl(p, st->z, b, w, prior, st->g, batch, s, it == opts->n_iter - 1,
                                it == 0 ? ready : nullptr, nullptr, step, atb)))
                return rc;
            if ((rc = launch_dots_gzx_gg(p, st->g, st->z, x, n, s))) return rc;
            if ((rc = launch_solver_scalar(p, opts->restart, s))) return rc;
            if ((rc = launch_update(p, x, st->z, st->g, n, s))) return rc;
        }
    }
    double sc[SC_COUNT];
    TC_CUDA(cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    st->t = sc[SC_T];
    st->k = (int)sc[SC_K];
    st->n_restarts = (int)sc[SC_RESTARTS];
    st->dots[0] = opts->restart == 2 ? 0.0 : sc[SC_DOT_GZX];
    st->dots[1] = opts->restart == 2 ? 0.0 : sc[SC_DOT_GG];
    if (opts->n_iter > 0 && opts->restart == 2) {  // the objective at the returned x
        st->obj[0] = sc[SC_DATA_X];
        st->obj[1] = sc[SC_PRIOR_X];
    } else if (opts->n_iter > 0) {
        st->obj[0] = sc[SC_DATA];
        st->obj[1] = (prior && prior->lambda != 0.0) ? sc[SC_PRIOR] : 0.0;
    }
    if ((rc = take_dev_status(p, s))) return rc;
    return TC_OK;
}

int check_solve(tc_plan *p, int batch, const tc_prior *prior, const tc_solve_opts *opts,
                const tc_solve_state *st) {
    if (!p || !opts || !st || batch < 1 || opts->n_iter < 0 || std::isnan(opts->step) ||
        std::isinf(opts->step) || opts->power_iter < 0 ||
        (!(opts->step > 0) && st->k > 0 && !(st->step > 0)) ||
        opts->restart < 0 || opts->restart > 2 || opts->normal < 0 || opts->normal > 1 || check_prior(prior))
        return TC_ERR_INVALID_ARG;
    if (check_ptrs({st->z, st->g}, {})) return TC_ERR_INVALID_ARG;
    if (opts->normal && (opts->restart == 2 || check_ptrs({st->atb}, {}))) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

// Stream and events owned by one host-streamed solve.
#ifndef TC_HOST_OUT_STREAM
#define TC_HOST_OUT_STREAM 1
#endif
// The copy streams of a host-streamed solve: slabs go in on cs and come back
// on cs_out, so that an outbound slab does not queue behind the inbound ones
// (the two directions use separate copy engines).
struct CopyStream {
    cudaStream_t cs = nullptr, cs_out = nullptr;
    std::vector<cudaEvent_t> ev;      // inbound slabs (+ the start event); fixed during the solve
    std::vector<cudaEvent_t> ev_bw;   // inbound b and w of each slab (when x is not needed first)
    std::vector<cudaEvent_t> out_ev;  // outbound slabs, appended while the last iteration runs
    void sync() {
        if (cs) cudaStreamSynchronize(cs);
        if (cs_out && cs_out != cs) cudaStreamSynchronize(cs_out);
    }
    ~CopyStream() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : out_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_bw)
            if (e) cudaEventDestroy(e);
        if (cs_out && cs_out != cs) cudaStreamDestroy(cs_out);
        if (cs) cudaStreamDestroy(cs);
    }
};

}  // namespace

extern "C" {

int tc_plan_autotune(tc_plan *p, const float *x, float *y, int batch, int reps,
                     int *chunk_out, int *cp_out, void *stream) {
    if (!p || batch < 1 || reps < 1 || check_ptrs({x, y}, {})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    const int max_chunk = batch < p->max_batch ? batch : p->max_batch;
    float best = -1.f;
    int best_chunk = p->chunk, best_cp = p->cp_col;
    int rc = TC_OK;
    for (int cp = 1; cp <= 4 && !rc; cp <<= 1) {
        if (plan_set_col_pairs(p, cp)) continue;
        for (int ch = max_chunk; ch >= 1 && !rc; ch = (ch > 1 && ch < 4) ? 1 : ch / 2) {
            p->chunk = ch;
            rc = radon_fwd(p, x, y, batch, stream);
            if (!rc) rc = radon_adj(p, y, (float *)x, batch, stream);
            if (rc) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && !rc; ++r) {
                rc = radon_fwd(p, x, y, batch, stream);
                if (!rc) rc = radon_adj(p, y, (float *)x, batch, stream);
            }
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = tc_cuda_fail(cudaGetLastError(), "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) {
                best = ms;
                best_chunk = ch;
                best_cp = cp;
            }
            if (ch == 1) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    plan_set_col_pairs(p, best_cp);
    p->chunk = best_chunk;
    if (chunk_out) *chunk_out = best_chunk;
    if (cp_out) *cp_out = best_cp;
    return TC_OK;
}

int tc_plan_set_spread_chunk(tc_plan *p, int entries) {
    if (!p) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    return plan_set_spread_chunk(p, entries);
}

int tc_plan_get_spread_chunk(const tc_plan *p) { return p ? p->k.chunk : TC_ERR_INVALID_ARG; }

int tc_plan_autotune_spread(tc_plan *p, const float *y, float *x, int batch, int reps, int *chunk_out,
                            void *stream) {
    if (!p || batch < 1 || reps < 1 || check_ptrs({x, y}, {})) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    float best = -1.f;
    int best_chunk = p->k.chunk, rc = TC_OK;
    for (int ch : {256, 512, 1024}) {
        if ((rc = plan_set_spread_chunk(p, ch))) break;
        if ((rc = radon_adj(p, y, x, batch, stream))) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !rc; ++r) rc = radon_adj(p, y, x, batch, stream);
        cudaEventRecord(e1, s);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = tc_cuda_fail(cudaGetLastError(), "autotune (spread)");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.f || ms < best) {
            best = ms;
            best_chunk = ch;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = plan_set_spread_chunk(p, best_chunk))) return rc;
    if (chunk_out) *chunk_out = best_chunk;
    return TC_OK;
}

int tc_plan_set_launch(tc_plan *p, int chunk, int col_pairs) {
    if (!p || chunk < 1 || chunk > p->max_batch) return TC_ERR_INVALID_ARG;
    if (col_pairs && plan_set_col_pairs(p, col_pairs)) return TC_ERR_INVALID_ARG;
    p->chunk = chunk;
    return TC_OK;
}

int mbir_solve(tc_plan *p, const float *b, const float *w, float *x, int batch,
               const tc_prior *prior, const tc_solve_opts *opts, tc_solve_state *st,
               void *stream) {
    if (check_solve(p, batch, prior, opts, st)) return TC_ERR_INVALID_ARG;
    if (check_ptrs({b, x}, {w}) || (opts->normal && w)) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    return solve_loop(p, b, w, x, batch, prior, opts, st, (cudaStream_t)stream, true, nullptr);
}

int mbir_solve_host(tc_plan *p, const float *b_host, const float *w_host, float *x_host,
                    float *dev_b, float *dev_w, float *dev_x, int batch,
                    const tc_prior *prior, const tc_solve_opts *opts,
                    tc_solve_state *st, void *stream) {
    if (check_solve(p, batch, prior, opts, st)) return TC_ERR_INVALID_ARG;
    if (!b_host || !x_host || (w_host && !dev_w) || check_ptrs({dev_b, dev_x}, {dev_w}) ||
        (opts->normal && w_host))
        return TC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ni = img_elems(p), ns = sino_elems(p);
    const int nslab = (batch + p->chunk - 1) / p->chunk;
    CopyStream cp;
    TC_CUDA(cudaStreamCreateWithFlags(&cp.cs, cudaStreamNonBlocking));
    if (TC_HOST_OUT_STREAM) TC_CUDA(cudaStreamCreateWithFlags(&cp.cs_out, cudaStreamNonBlocking));
    else cp.cs_out = cp.cs;
    cp.ev.assign(nslab, nullptr);
    // a step still to be derived needs the whole batch resident (and z, g as
    // its work vectors) before the first iteration
    const bool derive = st->k == 0 && !(opts->step > 0);
    auto body = [&]() -> int {
        // the copy stream must not overtake work already queued on the caller's stream
        cudaEvent_t start = nullptr;
        TC_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
        cp.ev.push_back(start);
        TC_CUDA(cudaEventRecord(start, s));
        TC_CUDA(cudaStreamWaitEvent(cp.cs, start, 0));
        // slab c of b, w and x goes in on the copy stream; the first iteration's
        // chunk c starts once its slab is resident.  A resumed solve with a
        // prior (z resident, x read by the prior only) starts chunk c's data
        // gradient once b and w have arrived, and each prior waits for its x.
        const bool early = st->k > 0 && !derive && opts->n_iter > 0 && !opts->normal && opts->restart != 2 &&
                           prior && prior->lambda != 0.0;
        if (early) cp.ev_bw.assign(nslab, nullptr);
        int rc;
        for (int c = 0; c < nslab; ++c) {
            const size_t s0 = (size_t)c * p->chunk;
            const size_t nb = (size_t)(batch - (int)s0 < p->chunk ? batch - (int)s0 : p->chunk);
            if ((rc = host_copy_async(dev_b + s0 * ns, b_host + s0 * ns, nb * ns * sizeof(float),
                                      cudaMemcpyHostToDevice, cp.cs)))
                return rc;
            if (w_host && (rc = host_copy_async(dev_w + s0 * ns, w_host + s0 * ns, nb * ns * sizeof(float),
                                                cudaMemcpyHostToDevice, cp.cs)))
                return rc;
            if (early) {
                TC_CUDA(cudaEventCreateWithFlags(&cp.ev_bw[c], cudaEventDisableTiming));
                TC_CUDA(cudaEventRecord(cp.ev_bw[c], cp.cs));
            }
            if ((rc = host_copy_async(dev_x + s0 * ni, x_host + s0 * ni, nb * ni * sizeof(float),
                                      cudaMemcpyHostToDevice, cp.cs)))
                return rc;
            if (st->k == 0 && !derive)
                TC_CUDA(cudaMemcpyAsync(st->z + s0 * ni, dev_x + s0 * ni, nb * ni * sizeof(float),
                                        cudaMemcpyDeviceToDevice, cp.cs));
            TC_CUDA(cudaEventCreateWithFlags(&cp.ev[c], cudaEventDisableTiming));
            TC_CUDA(cudaEventRecord(cp.ev[c], cp.cs));
        }
        // the first iteration's chunk c waits for slab c only; the full-volume
        // kernels that follow the chunk loop then see every slab
        const bool overlap = opts->n_iter > 0 && !derive;
        if (!overlap)
            for (int c = 0; c < nslab; ++c) TC_CUDA(cudaStreamWaitEvent(s, cp.ev[c], 0));
        // the last gradient-restart iteration with a prior sends x back slab by
        // slab while it runs; otherwise x goes back after the solve
        const bool stream_out = opts->n_iter > 0 && opts->restart != 2 && prior && prior->lambda != 0.0;
        const HostOut out{x_host, cp.cs_out, &cp.out_ev};
        rc = solve_loop(p, dev_b, w_host ? dev_w : nullptr, dev_x, batch, prior, opts, st, s, derive,
                        overlap ? cp.ev.data() : nullptr, stream_out ? &out : nullptr,
                        early && overlap ? cp.ev_bw.data() : nullptr);
        if (rc) return rc;
        if (!stream_out &&
            (rc = host_copy_async(x_host, dev_x, (size_t)batch * ni * sizeof(float), cudaMemcpyDeviceToHost, s)))
            return rc;
        TC_CUDA(cudaStreamSynchronize(s));
        TC_CUDA(cudaStreamSynchronize(cp.cs));
        if (cp.cs_out != cp.cs) TC_CUDA(cudaStreamSynchronize(cp.cs_out));
        return TC_OK;
    };
    const int rc = body();
    if (rc) {
        // copies already issued still read or write the caller's host buffers:
        // let them finish before the caller regains those buffers
        cp.sync();
        cudaStreamSynchronize(s);
    }
    return rc;
}

int tc_test_fail_copy_after(int after) {
    g_fail_copy_after.store(after < 0 ? -1 : after);
    return TC_OK;
}

}  // extern "C"
