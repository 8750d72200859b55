// Shared-memory FFTs used by the NUFFT passes.
//
// fft_pow2   : in-place Stockham autosort FFT of `cnt` back-to-back power-of-two
//              transforms of length n (radix-4 stages, one radix-2 stage when
//              log2 n is odd).  Each stage loads all of its butterflies into
//              registers, synchronises, then stores, so a single buffer
//              suffices.  Requires blockDim.x >= cnt * n / 16.
// fft_mixed  : out-of-place Stockham FFT of one length-n transform for an
//              arbitrary factorisation (the detector length D, e.g. 2896 =
//              181 * 4 * 4), one output per thread and stage, ping-pong buffers.
//
// SIGN = -1 computes sum_j v_j exp(-2 pi i jk/n); SIGN = +1 the conjugate
// kernel (no 1/n).  Twiddles come from FP64-built tables, never from fast
// approximate sin/cos.
#pragma once
#include "common.cuh"

template <int SIGN>
__device__ __forceinline__ float2 tw_get(const float2 *__restrict__ tw, int idx) {
    float2 w = tw[idx];
    if (SIGN > 0) w.y = -w.y;
    return w;
}

// multiply by SIGN * i
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 v) {
    return SIGN > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

template <int SIGN>
__device__ void fft_pow2(float2 *s, int n, int log2n, int cnt,
                         const float2 *__restrict__ tw) {
    const int nt = blockDim.x, tid = threadIdx.x;
    int Ns = 1, logNs = 0;
    while (Ns < n) {
        const int rem = log2n - logNs;
        if (rem >= 2) {
            // radix 4
            const int logper = log2n - 2, per = 1 << logper;
            const int total = cnt << logper;
            const int twstride = n >> (logNs + 2);
            float2 v[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int it = tid + i * nt;
                if (it < total) {
                    const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
                    const float2 *src = s + (tr << log2n) + j;
                    v[i][0] = src[0];
#pragma unroll
                    for (int q = 1; q < 4; ++q)
                        v[i][q] = cmul(src[q * per], tw_get<SIGN>(tw, q * k * twstride));
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int it = tid + i * nt;
                if (it < total) {
                    const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
                    const float2 a0 = cadd(v[i][0], v[i][2]), a1 = csub(v[i][0], v[i][2]);
                    const float2 b0 = cadd(v[i][1], v[i][3]), b1 = mul_si<SIGN>(csub(v[i][1], v[i][3]));
                    float2 *dst = s + (tr << log2n) + ((j >> logNs) << (logNs + 2)) + k;
                    dst[0] = cadd(a0, b0);
                    dst[Ns] = cadd(a1, b1);
                    dst[2 * Ns] = csub(a0, b0);
                    dst[3 * Ns] = csub(a1, b1);
                }
            }
            __syncthreads();
            Ns <<= 2;
            logNs += 2;
        } else {
            // radix 2 (last stage when log2 n is odd)
            const int logper = log2n - 1, per = 1 << logper;
            const int total = cnt << logper;
            const int twstride = n >> (logNs + 1);
            float2 v[8][2];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int it = tid + i * nt;
                if (it < total) {
                    const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
                    const float2 *src = s + (tr << log2n) + j;
                    v[i][0] = src[0];
                    v[i][1] = cmul(src[per], tw_get<SIGN>(tw, k * twstride));
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int it = tid + i * nt;
                if (it < total) {
                    const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
                    float2 *dst = s + (tr << log2n) + ((j >> logNs) << (logNs + 1)) + k;
                    dst[0] = cadd(v[i][0], v[i][1]);
                    dst[Ns] = csub(v[i][0], v[i][1]);
                }
            }
            __syncthreads();
            Ns <<= 1;
            logNs += 1;
        }
    }
}

// Out-of-place mixed-radix Stockham; returns the buffer holding the result.
// tw: [n] exp(-2 pi i k/n); root0: [rad[0]] exp(-2 pi i k/rad[0]).
template <int SIGN>
__device__ float2 *fft_mixed(float2 *a, float2 *b, const RadixPlan &rp,
                             const float2 *tw, const float2 *root0) {
    const int n = rp.n, nt = blockDim.x, tid = threadIdx.x;
    int Ns = 1;
    for (int st = 0; st < rp.nrad; ++st) {
        const int R = rp.rad[st];
        const int per = n / R;
        if (Ns == 1) {
            for (int o = tid; o < n; o += nt) {
                const int q = o % R, jb = o / R;
                float2 acc = make_float2(0.f, 0.f);
                int e = 0;
                for (int qq = 0; qq < R; ++qq) {
                    const float2 wv = tw_get<SIGN>(root0, e);
                    const float2 v = a[jb + qq * per];
                    acc.x = fmaf(v.x, wv.x, fmaf(-v.y, wv.y, acc.x));
                    acc.y = fmaf(v.x, wv.y, fmaf(v.y, wv.x, acc.y));
                    e += q;
                    if (e >= R) e -= R;
                }
                b[o] = acc;
            }
        } else {
            const int NsR = Ns * R;
            const int tws = n / NsR;
            for (int o = tid; o < n; o += nt) {
                const int k = o % Ns, q = (o / Ns) % R, jb = o / NsR;
                const int j = jb * Ns + k;
                const int step = (k + q * Ns) * tws;  // < n
                float2 acc = make_float2(0.f, 0.f);
                int e = 0;
                for (int qq = 0; qq < R; ++qq) {
                    const float2 wv = tw_get<SIGN>(tw, e);
                    const float2 v = a[j + qq * per];
                    acc.x = fmaf(v.x, wv.x, fmaf(-v.y, wv.y, acc.x));
                    acc.y = fmaf(v.x, wv.y, fmaf(v.y, wv.x, acc.y));
                    e += step;
                    if (e >= n) e -= n;
                }
                b[o] = acc;
            }
        }
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}
