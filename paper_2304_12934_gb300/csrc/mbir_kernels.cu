// MBIR kernels (arXiv 2304.12934, Sec. 3): FP64 reductions for the objective
// and the restart test, and the accelerated-gradient update with restart.  The
// qGGMRF prior (Eqs. reg2, reg3) is in prior_kernels.cu.
//
// Vectors are FP32; every reduction accumulates at most a few FP32 products
// per thread before promoting to FP64, then sums per-block FP64 partials in a
// fixed order, so results are bit-reproducible run to run.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "profile.cuh"

namespace {

__global__ void k_reduce_finalize(const double *__restrict__ partials, int n,
                                  double *acc, int accumulate, double scale) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    const double tot = block_sum_f64(s, red);
    if (threadIdx.x == 0) *acc = (accumulate ? *acc : 0.0) + scale * tot;
}

__global__ void k_dots_gzx_gg(const float4 *__restrict__ g, const float4 *__restrict__ z,
                              const float4 *__restrict__ x, size_t n4,
                              double *__restrict__ p_gzx, double *__restrict__ p_gg) {
    __shared__ double red[32];
    double a1 = 0.0, a2 = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 gv = g[i], zv = z[i], xv = x[i];
        float d = gv.x * (zv.x - xv.x);
        d = fmaf(gv.y, zv.y - xv.y, d);
        d = fmaf(gv.z, zv.z - xv.z, d);
        d = fmaf(gv.w, zv.w - xv.w, d);
        float q = gv.x * gv.x;
        q = fmaf(gv.y, gv.y, q);
        q = fmaf(gv.z, gv.z, q);
        q = fmaf(gv.w, gv.w, q);
        a1 += (double)d;
        a2 += (double)q;
    }
    const double t1 = block_sum_f64(a1, red);
    const double t2 = block_sum_f64(a2, red);
    if (threadIdx.x == 0) {
        p_gzx[blockIdx.x] = t1;
        p_gg[blockIdx.x] = t2;
    }
}

// n elements; the n % 4 after the last float4 are summed by block 0
__global__ void k_dot(const float4 *__restrict__ a, const float4 *__restrict__ b, size_t n,
                      double *__restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    const size_t n4 = n / 4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 u = a[i], v = b[i];
        float d = u.x * v.x;
        d = fmaf(u.y, v.y, d);
        d = fmaf(u.z, v.z, d);
        d = fmaf(u.w, v.w, d);
        acc += (double)d;
    }
    if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) {
        const size_t i = 4 * n4 + threadIdx.x;
        acc += (double)(reinterpret_cast<const float *>(a)[i] * reinterpret_cast<const float *>(b)[i]);
    }
    const double t = block_sum_f64(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// One thread: restart test and momentum coefficient, all in FP64.
__global__ void k_solver_scalar(double *sc, int restart) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double step = sc[SC_STEP];
    // <g, x_{k+1} - x_k> with x_{k+1} = z_k - step g
    const double dot = sc[SC_DOT_GZX] - step * sc[SC_DOT_GG];
    double t = sc[SC_T];
    const bool rs = restart && dot > 0.0;
    if (rs) {
        t = 1.0;
        sc[SC_RESTARTS] += 1.0;
    }
    sc[SC_RESTARTED] = rs ? 1.0 : 0.0;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc[SC_BETA] = (t - 1.0) / tn;
    sc[SC_T] = tn;
    sc[SC_K] += 1.0;
    sc[SC_NORM] = dot;
}

__global__ void k_update(float4 *__restrict__ x, float4 *__restrict__ z,
                         const float4 *__restrict__ g, size_t n4, const double *__restrict__ sc) {
    const float step = (float)sc[SC_STEP];
    const float beta = (float)sc[SC_BETA];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 xv = x[i], zv = z[i], gv = g[i];
        float4 xn, zn;
        xn.x = fmaf(-step, gv.x, zv.x);
        xn.y = fmaf(-step, gv.y, zv.y);
        xn.z = fmaf(-step, gv.z, zv.z);
        xn.w = fmaf(-step, gv.w, zv.w);
        zn.x = fmaf(beta, xn.x - xv.x, xn.x);
        zn.y = fmaf(beta, xn.y - xv.y, xn.y);
        zn.z = fmaf(beta, xn.z - xv.z, xn.z);
        zn.w = fmaf(beta, xn.w - xv.w, xn.w);
        x[i] = xn;
        z[i] = zn;
    }
}

// z := x after a restart (beta = 0 gives z_{k+1} = x_{k+1}), when the prior
// pass has written the momentum point of an iteration without restart.
__global__ void k_restart_fixup(float4 *__restrict__ z, const float4 *__restrict__ x, size_t n4,
                                const double *__restrict__ sc) {
    if (sc[SC_RESTARTED] == 0.0) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x)
        z[i] = x[i];
}

// Monotone variant (function-value test), all decisions in FP64 on the device.
// g := z - step g (the candidate v overwrites the gradient, which this
// variant no longer needs).
__global__ void k_step_to_candidate(const float4 *__restrict__ z, float4 *__restrict__ g, size_t n4,
                                    const double *__restrict__ sc) {
    const float step = (float)sc[SC_STEP];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 zv = z[i], gv = g[i];
        g[i] = make_float4(fmaf(-step, gv.x, zv.x), fmaf(-step, gv.y, zv.y), fmaf(-step, gv.z, zv.z),
                           fmaf(-step, gv.w, zv.w));
    }
}

// Phi(x_k) is held as SC_DATA_X + SC_PRIOR_X.  Accept v if Phi(v) <= Phi(x_k);
// on rejection keep x_k and restart the momentum (t := 1, beta = 0).
__global__ void k_monotone_scalar(double *sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double phi_v = sc[SC_DATA_V] + sc[SC_PRIOR_V];
    const double phi_x = sc[SC_DATA_X] + sc[SC_PRIOR_X];
    const bool accept = phi_v <= phi_x;
    double t = sc[SC_T];
    if (accept) {
        sc[SC_DATA_X] = sc[SC_DATA_V];
        sc[SC_PRIOR_X] = sc[SC_PRIOR_V];
    } else {
        t = 1.0;
        sc[SC_RESTARTS] += 1.0;
    }
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc[SC_BETA] = accept ? (t - 1.0) / tn : 0.0;
    sc[SC_T] = tn;
    sc[SC_K] += 1.0;
    sc[SC_ACCEPT] = accept ? 1.0 : 0.0;
}

// accept_all: v is x_{k+1} (the gradient-restart schedule, with x_{k+1}
// formed ahead of the restart decision); with keep_x as well, x_{k+1} stays
// where v is and only z is written.
__global__ void k_update_monotone(float4 *__restrict__ x, float4 *__restrict__ z,
                                  const float4 *__restrict__ v, size_t n4, const double *__restrict__ sc,
                                  int accept_all, int keep_x) {
    const bool accept = accept_all || sc[SC_ACCEPT] != 0.0;
    const float beta = (float)sc[SC_BETA];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 xv = x[i];
        if (!accept) {  // x_{k+1} = x_k, z_{k+1} = x_k
            z[i] = xv;
            continue;
        }
        const float4 xn = v[i];
        float4 zn;
        zn.x = fmaf(beta, xn.x - xv.x, xn.x);
        zn.y = fmaf(beta, xn.y - xv.y, xn.y);
        zn.z = fmaf(beta, xn.z - xv.z, xn.z);
        zn.w = fmaf(beta, xn.w - xv.w, xn.w);
        if (!keep_x) x[i] = xn;
        z[i] = zn;
    }
}

__global__ void k_scale_inv_sqrt(float4 *__restrict__ v, size_t n4, const double *__restrict__ sq) {
    const float s = (float)(1.0 / sqrt(*sq));
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        float4 a = v[i];
        a.x *= s; a.y *= s; a.z *= s; a.w *= s;
        v[i] = a;
    }
}

__global__ void k_fill_scalars(double *sc, double t, double k, double restarts, double step) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc[SC_T] = t;
        sc[SC_K] = k;
        sc[SC_RESTARTS] = restarts;
        sc[SC_STEP] = step;
        sc[SC_BETA] = 0.0;
    }
}

// Seeded start vector of the step's power iteration: element i is uniform in
// [-1, 1), taken from the splitmix64 output (Steele, Lea and Flood 2014) for
// counter i of the given seed.
__global__ void k_fill_start(float *__restrict__ v, size_t n, unsigned long long seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = (float)(z >> 40) * (1.0f / 8388608.0f) - 1.0f;  // 24 bits: exact in float
    }
}

int grid_for(size_t n4) {
    size_t b = (n4 + TC_RED_THREADS - 1) / TC_RED_THREADS;
    return (int)(b < TC_RED_BLOCKS ? (b ? b : 1) : TC_RED_BLOCKS);
}

}  // namespace

int launch_step_to_candidate(tc_plan *p, const float *z, float *g, size_t n, cudaStream_t s) {
    const size_t n4 = n / 4;
    TC_PROFILED(TCK_UPDATE, s,
                k_step_to_candidate<<<grid_for(n4), TC_RED_THREADS, 0, s>>>(
        reinterpret_cast<const float4 *>(z), reinterpret_cast<float4 *>(g), n4, p->scal));
    TC_LAUNCHED("k_step_to_candidate");
    return TC_OK;
}

int launch_monotone_scalar(tc_plan *p, cudaStream_t s) {
    TC_PROFILED(TCK_SCALAR, s, k_monotone_scalar<<<1, 32, 0, s>>>(p->scal));
    TC_LAUNCHED("k_monotone_scalar");
    return TC_OK;
}

int launch_update_monotone(tc_plan *p, float *x, float *z, const float *v, size_t n,
                           cudaStream_t s, int accept_all, int keep_x) {
    const size_t n4 = n / 4;
    TC_PROFILED(TCK_UPDATE, s,
                k_update_monotone<<<grid_for(n4), TC_RED_THREADS, 0, s>>>(
        reinterpret_cast<float4 *>(x), reinterpret_cast<float4 *>(z),
        reinterpret_cast<const float4 *>(v), n4, p->scal, accept_all, keep_x));
    TC_LAUNCHED("k_update_monotone");
    return TC_OK;
}

int launch_reduce_finalize(const double *partials, int n, double *acc,
                           int accumulate, double scale, cudaStream_t s) {
    TC_PROFILED(TCK_REDUCE, s,
                k_reduce_finalize<<<1, 256, 0, s>>>(partials, n, acc, accumulate, scale));
    TC_LAUNCHED("k_reduce_finalize");
    return TC_OK;
}

int launch_dots_gzx_gg(tc_plan *p, const float *g, const float *z, const float *x,
                       size_t n, cudaStream_t s) {
    const size_t n4 = n / 4;
    const int blocks = grid_for(n4);
    double *p1 = p->partials + (size_t)2 * p->slot, *p2 = p->partials + (size_t)3 * p->slot;
    TC_PROFILED(TCK_DOTS, s,
                k_dots_gzx_gg<<<blocks, TC_RED_THREADS, 0, s>>>(
        reinterpret_cast<const float4 *>(g), reinterpret_cast<const float4 *>(z),
        reinterpret_cast<const float4 *>(x), n4, p1, p2));
    TC_LAUNCHED("k_dots_gzx_gg");
    int rc = launch_reduce_finalize(p1, blocks, p->scal + SC_DOT_GZX, 0, 1.0, s);
    if (rc) return rc;
    return launch_reduce_finalize(p2, blocks, p->scal + SC_DOT_GG, 0, 1.0, s);
}

int launch_dot(tc_plan *p, const float *a, const float *b, size_t n,
               double *out_acc, cudaStream_t s) {
    const size_t n4 = n / 4;
    const int blocks = grid_for(n4);
    double *part = p->partials + (size_t)2 * p->slot;
    TC_PROFILED(TCK_DOT, s,
                k_dot<<<blocks, TC_RED_THREADS, 0, s>>>(reinterpret_cast<const float4 *>(a),
                                            reinterpret_cast<const float4 *>(b), n, part));
    TC_LAUNCHED("k_dot");
    return launch_reduce_finalize(part, blocks, out_acc, 0, 1.0, s);
}

int launch_solver_scalar(tc_plan *p, int restart, cudaStream_t s) {
    TC_PROFILED(TCK_SCALAR, s,
                k_solver_scalar<<<1, 32, 0, s>>>(p->scal, restart));
    TC_LAUNCHED("k_solver_scalar");
    return TC_OK;
}

int launch_update(tc_plan *p, float *x, float *z, const float *g, size_t n,
                  cudaStream_t s) {
    const size_t n4 = n / 4;
    TC_PROFILED(TCK_UPDATE, s,
                k_update<<<grid_for(n4), TC_RED_THREADS, 0, s>>>(
        reinterpret_cast<float4 *>(x), reinterpret_cast<float4 *>(z),
        reinterpret_cast<const float4 *>(g), n4, p->scal));
    TC_LAUNCHED("k_update");
    return TC_OK;
}

int launch_restart_fixup(tc_plan *p, float *z, const float *x, size_t n, cudaStream_t s) {
    const size_t n4 = n / 4;
    TC_PROFILED(TCK_FIXUP, s,
                k_restart_fixup<<<grid_for(n4), TC_RED_THREADS, 0, s>>>(
        reinterpret_cast<float4 *>(z), reinterpret_cast<const float4 *>(x), n4, p->scal));
    TC_LAUNCHED("k_restart_fixup");
    return TC_OK;
}

int launch_scale_by_inv_sqrt(float *v, size_t n, const double *sq, cudaStream_t s) {
    const size_t n4 = n / 4;
    TC_PROFILED(TCK_SCALE, s,
                k_scale_inv_sqrt<<<grid_for(n4), TC_RED_THREADS, 0, s>>>(reinterpret_cast<float4 *>(v), n4, sq));
    TC_LAUNCHED("k_scale_inv_sqrt");
    return TC_OK;
}

int launch_copy(float *dst, const float *src, size_t n, cudaStream_t s) {
    TC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return TC_OK;
}

int launch_fill_start(float *v, size_t n, unsigned long long seed, cudaStream_t s) {
    TC_PROFILED(TCK_FILL, s, k_fill_start<<<grid_for(n / 4 + 1), TC_RED_THREADS, 0, s>>>(v, n, seed));
    TC_LAUNCHED("k_fill_start");
    return TC_OK;
}

int launch_fill_scalars_fresh(tc_plan *p, double t, double k, double restarts,
                              double step, cudaStream_t s) {
    TC_PROFILED(TCK_FILL, s,
                k_fill_scalars<<<1, 32, 0, s>>>(p->scal, t, k, restarts, step));
    TC_LAUNCHED("k_fill_scalars");
    return TC_OK;
}
