// Internal definitions shared by the CUDA translation units of the NUFFT Radon
// library: the plan layout, the by-value kernel argument block and complex
// helpers.  Nothing here is part of the C ABI (include/nufft_radon.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nufft_radon.h"

#define TC_MAX_RADICES 24

// Mixed-radix factorisation of the detector length D (odd primes first).
struct RadixPlan {
    int n;
    int nrad;
    int rad[TC_MAX_RADICES];
};

// Geometry and table pointers passed by value to every Radon kernel.
struct KArgs {
    int N, log2N;      // image side (power of two)
    int G;             // oversampled grid side, 2N
    int A, D, Mh;      // angles, detector bins, radial samples m = 0..D/2
    int AM;            // A * Mh polar points per slice
    int w;             // kernel width
    int R;             // grid rows jy = jmin .. jmin + R - 1 touched by any point
    int jmin, jmax;
    int kmin, kmax;    // range of the row-entry sort key jx0
    float beta, inv_h; // ES kernel: phi(z) = exp(beta (sqrt(1 - z^2) - 1)), z = offset / (w/2)
    float beta_l2;     // beta * log2(e)
    float invD;
    const float *dea;          // [N] 1 / psi(i - N/2)  (from FP64)
    const float2 *twN;         // per-stage twiddle tables of the N-point FFT (ntwN entries)
    int ntwN;
    const float2 *twG;         // [N] exp(-2 pi i (k - N/2) / G)
    const float2 *twD;         // [D] exp(-2 pi i k / D)
    const int *row_off;        // [R + 1] first entry of each grid row
    const int4 *ent;           // [E] packed Entry records (see entry_* accessors)
    // spreading records: one per (row, entry chunk, touched cell); see plan.cu
    const int2 *rec;           // x: (signed cell - kmin) | seam << 15; y: lo | hi << 16
    const int *rec_off;        // [R][2 nch + 1] record ranges (regular, seam) per row and chunk
    int nch;                   // chunks per row (max over rows)
    int chunk;                 // entries per spreading chunk (256, 512 or 1024)
    const unsigned char *angle_flip; // [A] 1: theta was in [pi, 2 pi), data conjugated
    const float2 *shiftD;      // [Mh] exp(-2 pi i m delta / D) (axis offset), or null for delta = 0
    RadixPlan rp;              // factorisation of D
    // Bluestein (chirp-z) detector DFT, used when D has a large prime factor:
    // length-L power-of-two FFTs, L >= 2D - 1
    int blue, L, log2L;
    const float2 *chirp;       // [D] exp(-i pi (n^2 mod 2D) / D)
    const float2 *bhat;        // [L] FFT_L of the conjugate chirp (wrapped), times 1/L
    const float2 *twL;         // per-stage twiddle tables of the L-point FFT
};

#ifdef __cplusplus
#include <vector>
#endif
// Host-side copies a plan keeps to rebuild its spreading records.
struct PlanHost {
    std::vector<int> keys;     // jx0 of every entry, key-sorted within each row
    std::vector<int> row_off;  // [R + 1] first entry of each row
    size_t n_rec = 0, n_roff = 0;
};

struct tc_plan {
    PlanHost *host;       // host copies (see PlanHost)
    int device;
    int max_batch;
    int chunk;            // slices per launch (<= max_batch; set by tc_plan_autotune)
    KArgs k;
    double *dea64;        // FP64 deapodisation factors (device)
    float *dea;
    float2 *twN, *twG, *twD;
    int *row_off;
    int4 *ent;
    int2 *rec;
    int *rec_off;
    unsigned char *angle_flip;
    float2 *shiftD;
    float2 *chirp, *bhat, *twL;
    long long n_entries;
    // scratch for max_batch slices
    float2 *tu;           // [MB][R][N]   column-pass output (fwd) / row-pass output (adj)
    float2 *pv;           // [MB][w][AM]  interpolation partials (fwd) / spread weights (adj, plane 0)
    float *sr;            // [MB][A][D]   weighted residual sinogram (MBIR)
    double *partials;     // TC_N_SLOTS slots of `slot` per-block FP64 partial sums
    int slot;
    double *scal;         // device scalars of the solver
    int *dev_err;         // device status of bounded waits (TC_OK or TC_ERR_TIMEOUT)
    long long bytes;
    // launch configuration
    int cp_col;           // column pairs per CTA in the column passes
    int threads_col, threads_row, threads_det;
    size_t smem_col, smem_row_fwd, smem_row_adj, smem_det;
    size_t smem_col_tma;  // forward column pass with its image strip staged by TMA (0: not used)
    // normal operator A^T A by Toeplitz-plus-Hankel embedding (normal.cu),
    // tables built on first use
    double *cs64;         // [A][2] cos, sin of the angles as given (FP64)
    double delta;         // rotation-axis offset
    int nrm_ready;
    KArgs kn;             // column passes of the embedding: rows 0..N, unit deapodisation
    float *nrm_t;         // [N+1][2N] T^ / G^2 (rows 1..N-1 doubled), cell layout [t][j], c = 2j + t
    float2 *nrm_h;        // [N+1][2N] H^ / G^2, same layout
    float *nrm_one;       // [N] ones
    float2 *nrm_tu;       // [MB][N+1][N] grid rows when tu holds fewer than N+1 rows (else null)
    double *nrm_part;     // [MB * N/2] FP64 partials of the fused data term
};

// Extra shared memory of the TMA forward column pass: 128 bytes of alignment
// slack, the image strip (N rows x 2 cp floats) and its mbarrier.
__host__ __device__ constexpr size_t col_strip_bytes(int n, int cp) {
    return 128 + (size_t)n * 2 * cp * sizeof(float) + 16;
}

// One (polar point, tap row) entry of a grid row's bin, 16 bytes:
//   x: polar point index p = a * Mh + m
//   y: gx - jx0 (float bits)
//   z: phi_y, the point's kernel weight for this row (float bits)
//   w: jx0 (low 16 bits, signed) | tap row s << 16
__host__ __device__ __forceinline__ int entry_p(int4 e) { return e.x; }
__host__ __device__ __forceinline__ int entry_key(int4 e) { return (int)(short)(e.w & 0xffff); }
__host__ __device__ __forceinline__ int entry_s(int4 e) { return (e.w >> 16) & 0xff; }
#ifdef __CUDACC__
__device__ __forceinline__ float entry_ex(int4 e) { return __int_as_float(e.y); }
__device__ __forceinline__ float entry_wy(int4 e) { return __int_as_float(e.z); }
#endif

// ------------------------------------------------------------- complex ops --
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a += w * v for real weight w
__device__ __forceinline__ void cfma(float2 &a, float wgt, float2 v) {
    a.x = fmaf(wgt, v.x, a.x);
    a.y = fmaf(wgt, v.y, a.y);
}

// Exponential-of-semicircle spreading kernel (Barnett, Magland, af Klinteberg
// 2019), evaluated at z = offset / (w/2); zero for |z| >= 1.
__device__ __forceinline__ float es_kernel(float z, float beta) {
    const float q = 1.0f - z * z;
    return q > 0.0f ? expf(beta * (sqrtf(q) - 1.0f)) : 0.0f;
}

// The same kernel with beta_l2 = beta * log2(e), through the one-instruction
// approximate square root and exp2 (relative errors ~1e-7, well inside the
// NUFFT's own error; denormals flushed).  Zero outside |z| < 1.
__device__ __forceinline__ float es_kernel_fast(float z, float beta_l2) {
    const float q = fmaf(-z, z, 1.0f);
    float r, e;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fmaf(beta_l2, r, -beta_l2)));
    return q > 0.0f ? e : 0.0f;
}

// Entries of one grid row staged per chunk by the spreading kernel: a plan
// chooses 256, 512 or 1024 (tc_plan_set_spread_chunk); this is the default.
#define TC_SPREAD_CHUNK_DEFAULT 1024

// Block-wide FP64 sum of one float per thread; thread 0 gets the total.
__device__ __forceinline__ double block_sum_f64(double d, double *red) {
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = d;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) tot += red[i];
    }
    __syncthreads();
    return tot;
}

// Reductions write one FP64 partial per block into a slot of plan->partials and
// a single-block kernel sums the slot in a fixed order (deterministic).
#define TC_RED_BLOCKS 1216   // fixed grid of the grid-stride reductions (152 SMs x 8)
#define TC_RED_THREADS 256
#define TC_N_SLOTS 4
// Device scalar block of the solver (plan->scal).
enum {
    SC_DATA = 0,     // data term 1/2 sum W r^2 (accumulated over chunks)
    SC_PRIOR,        // lambda H
    SC_DOT_GZX,      // <g, z - x>
    SC_DOT_GG,       // <g, g>
    SC_T,            // momentum t_k
    SC_BETA,         // momentum coefficient of this iteration
    SC_RESTARTS,     // restart count (as double)
    SC_K,            // iteration count (as double)
    SC_STEP,         // step
    SC_NORM,         // scratch norm / Rayleigh quotient
    // monotone variant (function-value test)
    SC_DATA_V,       // data term at the candidate v = z - step g
    SC_PRIOR_V,      // lambda H(v)
    SC_DATA_X,       // data term at the accepted iterate x_k
    SC_PRIOR_X,      // lambda H(x_k)
    SC_ACCEPT,       // 1: this iteration's candidate was accepted
    SC_BB,           // 1/2 ||b||^2 of a normal-operator solve
    SC_RESTARTED,    // 1: this iteration's gradient test restarted the momentum
    SC_COUNT = 17
};

// Launchers (defined in radon_kernels.cu / mbir_kernels.cu).
int launch_radon_fwd_chunk(tc_plan *p, const float *x, float *y, int nb,
                           const float *b, const float *w, float *resid,
                           double *obj_acc, cudaStream_t s);
int launch_radon_adj_chunk(tc_plan *p, const float *y, float *x, int nb,
                           cudaStream_t s);
// out = A^T A x by the Toeplitz-plus-Hankel embedding (tables from
// normal_prepare).  With sub: out = A^T A x - sub; with xdot as well,
// *obj_acc += 1/2 <xdot, out - sub>.
int launch_radon_normal_chunk(tc_plan *p, const float *x, float *out, int nb, const float *sub,
                              const float *xdot, double *obj_acc, cudaStream_t s);
// Builds the embedding's tables once per plan (synchronous on s).
int normal_prepare(tc_plan *p, cudaStream_t s);
// g += lambda grad H(x); h_acc (or NULL) = lambda H(x).  With dot_x (the
// solver's x_k), also scal[SC_DOT_GZX] = <g, x - dot_x> and scal[SC_DOT_GG] =
// <g, g> of the final g, and the gradient is not stored: the next iterate
// x - step g goes to dot_x (over x_k), and g receives the momentum point
// x_{k+1} + beta (x_{k+1} - x_k) with the beta of an iteration without
// restart (from scal[SC_T]).
// x holds nb slices; only slices [z0, z1) (z1 < 0: nb) get their gradient
// (neighbours outside the range are read) and enter the sums, which a slab
// with z0 > 0 adds to those already held.
int launch_prior_grad(tc_plan *p, const float *x, float *g, int nb,
                      const tc_prior *pr, double *h_acc, cudaStream_t s,
                      float *dot_x = nullptr, int z0 = 0, int z1 = -1, double step = 0.0);
// Tiles of one prior launch on N x N slices, and the FP64 partial-sum slots
// its z-chunked grid may use.
int prior_tile_count(int n);
int prior_block_slots(int n);
// h_acc = lambda H(x) only (no gradient).
int launch_prior_value(tc_plan *p, const float *x, int nb, const tc_prior *pr,
                       double *h_acc, cudaStream_t s);
// Monotone variant: v = z - step g in place of g; the accept/restart decision
// and momentum; the update x_{k+1} = accepted ? v : x_k,
// z_{k+1} = x_{k+1} + beta (x_{k+1} - x_k).
int launch_step_to_candidate(tc_plan *p, const float *z, float *g, size_t n, cudaStream_t s);
int launch_monotone_scalar(tc_plan *p, cudaStream_t s);
int launch_update_monotone(tc_plan *p, float *x, float *z, const float *v, size_t n,
                           cudaStream_t s, int accept_all = 0, int keep_x = 0);
int launch_reduce_finalize(const double *partials, int n, double *acc,
                           int accumulate, double scale, cudaStream_t s);
int launch_dots_gzx_gg(tc_plan *p, const float *g, const float *z, const float *x,
                       size_t n, cudaStream_t s);
int launch_solver_scalar(tc_plan *p, int restart, cudaStream_t s);
int launch_update(tc_plan *p, float *x, float *z, const float *g, size_t n,
                  cudaStream_t s);
// After a prior pass with next = true: z := x where the gradient test has just
// restarted the momentum (scal[SC_RESTARTED]); otherwise the kernel returns.
int launch_restart_fixup(tc_plan *p, float *z, const float *x, size_t n, cudaStream_t s);
int launch_dot(tc_plan *p, const float *a, const float *b, size_t n,
               double *out_acc, cudaStream_t s);
int launch_scale_by_inv_sqrt(float *v, size_t n, const double *sq, cudaStream_t s);
int launch_copy(float *dst, const float *src, size_t n, cudaStream_t s);
int launch_fill_scalars_fresh(tc_plan *p, double t, double k, double restarts,
                              double step, cudaStream_t s);
// v[i] uniform in [-1, 1) from a counter-based generator (power-iteration start)
int launch_fill_start(float *v, size_t n, unsigned long long seed, cudaStream_t s);
// Host-to-device / device-to-host copy of the host-streamed solve, with the
// failure-injection hook of tc_test_fail_copy_after (api.cu).
int host_copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s);

// Error plumbing (api.cu).
int tc_cuda_fail(cudaError_t e, const char *where);
#define TC_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return tc_cuda_fail(_e, #call);     \
    } while (0)
#define TC_LAUNCHED(name)                                          \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return tc_cuda_fail(_e, name);      \
    } while (0)
