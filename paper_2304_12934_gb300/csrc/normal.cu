// Normal operator A^T A of the discrete Radon operator by Toeplitz-plus-Hankel
// embedding (the Hessian of the unweighted data term, Sec. 3 Eqs. gradient
// and transpose), for unweighted least squares without gridding.
//
// For even D, with the Nyquist pair m = +-D/2 weighted 1/2 and the rotation
// axis at detector coordinate delta, the projection of pixel p at angle a is
// the Dirichlet kernel K(t_i - s_p(a) - delta), s_p(a) = p_x cos th + p_y sin th,
// K(u) = (1/D) [sin(pi u (D-1)/D) / sin(pi u/D) + cos(pi u)].  Summing two
// such kernels over the D bins t_i = i - D/2 leaves
//     K(u - v) - cos(pi (u - v)) / 2D + cos(pi (u + v)) / 2D,
// because the only frequency pairs m + m' = 0 (mod D) are m' = -m and the
// two Nyquist self-pairs.  With s linear in p,
//     (A^T A f)(p') = sum_p f(p) [T(p' - p) + H(p' + p)],
//     T(d) = sum_a K(s_d(a)) - cos(pi s_d(a)) / 2D,
//     H(e) = sum_a cos(pi (s_e(a) + 2 delta)) / 2D.
// Both terms are cyclic convolutions on the G = 2N periodic grid (|d| < N and
// -N <= e <= N - 2 fit without wrap-around), so with F the G-point DFT of the
// image placed at its centred coordinates,
//     A^T A f = IDFT(T^(k) F(k) + H^(k) F(-k)),   F(-k) = conj F(k) (f real).
// T^ is real (T is even).  The embedding is exact: its only error is FP32
// rounding in the FFT passes, against the NUFFT's kernel error.
//
// The tables are built once per plan in FP64: T + iH on the G x G grid from
// the closed forms above (one thread per grid point, summing over the
// angles as given), a G x G FFT (radix-2, one line per CTA), and the
// split T^ = (Z(k) + conj Z(-k))/2, H^ = (Z(k) - conj Z(-k))/2i.  Only the
// half plane ky = 0..N is kept: the inverse column pass completes it by
// Hermitian symmetry and takes the real part, so rows 1..N-1 carry a factor
// 2 (rows 0 and N are their own mirror images).  The 1/G^2 of the inverse DFT
// is folded in, and each row is stored in the FFT's cell order (even cells,
// then odd cells).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

__device__ __forceinline__ double2 z64mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// tw[k] = exp(-2 pi i k / G), k < G/2
__global__ void k_nrm_tw64(double2 *tw, int G) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < G / 2) {
        double sv, cv;
        sincospi(-2.0 * k / G, &sv, &cv);
        tw[k] = make_double2(cv, sv);
    }
}

// Z[jy][jx] = T(d) + i H(d), d = (jx, jy) read as signed coordinates mod G.
__global__ void k_nrm_space(double2 *Z, int N, int A, int D, const double *__restrict__ cs, double delta) {
    const int G = 2 * N;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)G * G) return;
    const int jx = (int)(idx % G), jy = (int)(idx / G);
    const double dx = jx < N ? jx : jx - G, dy = jy < N ? jy : jy - G;
    const double invD = 1.0 / D, half_invD = 0.5 / D;
    double t = 0.0, h = 0.0;
    for (int a = 0; a < A; ++a) {
        const double s = dx * cs[2 * a] + dy * cs[2 * a + 1];
        const double r = s - D * rint(s * invD);  // K is D-periodic for even D
        const double cs_pi = cospi(s);
        double kd;
        if (r == 0.0) {
            kd = 1.0;
        } else {
            kd = (sinpi(r - r * invD) / sinpi(r * invD) + cs_pi) * invD;
        }
        t += kd - cs_pi * half_invD;
        h += (delta == 0.0 ? cs_pi : cospi(s + 2.0 * delta)) * half_invD;
    }
    Z[idx] = make_double2(t, h);
}

// In-place G-point FFT (exp(-2 pi i jk/G)) of the lines a + l * line_stride,
// elements elem_stride apart; one line per CTA, radix 2 in shared memory.
__global__ void k_nrm_fft64(double2 *a, const double2 *__restrict__ tw, int logG, long long line_stride,
                            long long elem_stride) {
    extern __shared__ double2 s64[];
    const int G = 1 << logG;
    double2 *base = a + blockIdx.x * line_stride;
    for (int i = threadIdx.x; i < G; i += blockDim.x)
        s64[__brev((unsigned)i) >> (32 - logG)] = base[i * elem_stride];
    __syncthreads();
    for (int lh = 0; lh < logG; ++lh) {  // butterflies of span 2^(lh+1)
        const int half = 1 << lh;
        for (int bf = threadIdx.x; bf < G / 2; bf += blockDim.x) {
            const int j = bf & (half - 1);
            const int i0 = ((bf >> lh) << (lh + 1)) + j, i1 = i0 + half;
            const double2 w = tw[j << (logG - 1 - lh)];
            const double2 u = s64[i0], v = z64mul(s64[i1], w);
            s64[i0] = make_double2(u.x + v.x, u.y + v.y);
            s64[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < G; i += blockDim.x) base[i * elem_stride] = s64[i];
}

__global__ void k_nrm_table(const double2 *__restrict__ Z, float *__restrict__ tt, float2 *__restrict__ th,
                            int N) {
    const int G = 2 * N;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(N + 1) * G) return;
    const int c = (int)(idx % G), r = (int)(idx / G);
    const double2 zk = Z[(size_t)r * G + c];
    const double2 zm = Z[(size_t)((G - r) & (G - 1)) * G + ((G - c) & (G - 1))];
    const double sc = ((r == 0 || r == N) ? 1.0 : 2.0) / ((double)G * G);
    const size_t o = (size_t)r * G + (size_t)(c & 1) * N + (c >> 1);
    tt[o] = (float)(0.5 * (zk.x + zm.x) * sc);
    th[o] = make_float2((float)(0.5 * (zk.y + zm.y) * sc), (float)(-0.5 * (zk.x - zm.x) * sc));
}

int dev_alloc(void **ptr, size_t bytes, tc_plan *p) {
    TC_CUDA(cudaMalloc(ptr, bytes));
    p->bytes += (long long)bytes;
    return TC_OK;
}

}  // namespace

int normal_prepare(tc_plan *p, cudaStream_t s) {
    if (p->nrm_ready) return TC_OK;
    // Building the tables allocates and synchronises, which a stream capture
    // cannot record: refuse before touching the stream, so the capture stays
    // valid and the caller learns to prepare the plan first.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TC_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return TC_ERR_UNSUPPORTED;
    const KArgs &k = p->k;
    const int N = k.N, G = 2 * N, logG = k.log2N + 1, R = N + 1;
    const size_t MB = (size_t)p->max_batch;
    int rc;
    if (!p->nrm_t && (rc = dev_alloc((void **)&p->nrm_t, (size_t)R * G * sizeof(float), p))) return rc;
    if (!p->nrm_h && (rc = dev_alloc((void **)&p->nrm_h, (size_t)R * G * sizeof(float2), p))) return rc;
    if (!p->nrm_one && (rc = dev_alloc((void **)&p->nrm_one, (size_t)N * sizeof(float), p))) return rc;
    if (!p->nrm_part && (rc = dev_alloc((void **)&p->nrm_part, MB * (N / 2) * sizeof(double), p))) return rc;
    if (k.R < R && !p->nrm_tu && (rc = dev_alloc((void **)&p->nrm_tu, MB * R * N * sizeof(float2), p)))
        return rc;
    const std::vector<float> ones(N, 1.0f);
    TC_CUDA(cudaMemcpyAsync(p->nrm_one, ones.data(), N * sizeof(float), cudaMemcpyHostToDevice, s));

    double2 *Z = nullptr, *tw = nullptr;
    TC_CUDA(cudaMalloc(&Z, (size_t)G * G * sizeof(double2)));
    if (cudaMalloc(&tw, (size_t)(G / 2) * sizeof(double2)) != cudaSuccess) {
        cudaFree(Z);
        return tc_cuda_fail(cudaErrorMemoryAllocation, "normal_prepare");
    }
    rc = TC_OK;
    const size_t smem = (size_t)G * sizeof(double2);  // <= 128 KB (G <= 8192)
    // the limit is process wide per kernel: only ever raise it
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_nrm_fft64);
    if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem)
        e = cudaFuncSetAttribute(k_nrm_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        const long long GG = (long long)G * G;
        k_nrm_tw64<<<(G / 2 + 255) / 256, 256, 0, s>>>(tw, G);
        k_nrm_space<<<(unsigned)((GG + 255) / 256), 256, 0, s>>>(Z, N, k.A, k.D, p->cs64, p->delta);
        k_nrm_fft64<<<G, 512, smem, s>>>(Z, tw, logG, G, 1);   // along x
        k_nrm_fft64<<<G, 512, smem, s>>>(Z, tw, logG, 1, G);   // along y
        const long long RG = (long long)R * G;
        k_nrm_table<<<(unsigned)((RG + 255) / 256), 256, 0, s>>>(Z, p->nrm_t, p->nrm_h, N);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(Z);
    cudaFree(tw);
    if (e != cudaSuccess) return tc_cuda_fail(e, "normal_prepare");
    p->kn = k;
    p->kn.dea = p->nrm_one;
    p->kn.jmin = 0;
    p->kn.jmax = N;
    p->kn.R = R;
    p->nrm_ready = 1;
    return TC_OK;
}
