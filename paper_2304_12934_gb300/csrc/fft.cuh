// Shared-memory FFTs used by the NUFFT passes.
//
// fft_pow2   : in-place Stockham autosort FFT of `cnt` back-to-back power-of-two
//              transforms of length n: radix-16 stages with register
//              butterflies, then one radix-8/4/2 stage.  Each stage loads all
//              of its butterflies into registers, synchronises, then stores,
//              so a single (padded) buffer suffices.  Requires
//              blockDim.x >= cnt * n / 16.
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

// Shared-memory index padding: one float2 of padding after every 16, so the
// strided butterfly stores of the first stages hit distinct banks.
__host__ __device__ constexpr int spad(int i) { return i + (i >> 4); }
// float2 elements to allocate for m padded elements
__host__ __device__ constexpr int spad_size(int m) { return m + (m >> 4) + 1; }

// In-register DFTs of length 2, 4, 8, 16 (natural order in and out).
template <int SIGN>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    const float2 a0 = cadd(x0, x2), a1 = csub(x0, x2);
    const float2 b0 = cadd(x1, x3), b1 = mul_si<SIGN>(csub(x1, x3));
    x0 = cadd(a0, b0);
    x1 = cadd(a1, b1);
    x2 = csub(a0, b0);
    x3 = csub(a1, b1);
}

// exp(SIGN * 2 pi i j / 16) for the constant twiddles of the 8- and 16-point DFTs
template <int SIGN>
__device__ __forceinline__ float2 w16(int j) {
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
    float cr, ci;
    switch (j) {
        case 1: cr = c1; ci = s1; break;
        case 2: cr = r2; ci = r2; break;
        case 3: cr = s1; ci = c1; break;
        case 4: cr = 0.f; ci = 1.f; break;
        case 6: cr = -r2; ci = r2; break;
        case 9: cr = -c1; ci = -s1; break;
        default: cr = 1.f; ci = 0.f; break;
    }
    return make_float2(cr, SIGN > 0 ? ci : -ci);
}

template <int SIGN, int R>
__device__ __forceinline__ void dft_reg(float2 *v) {
    if (R == 2) {
        const float2 t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    } else if (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else if (R == 8) {
        // n = 4 n1 + n2, k = k1 + 2 k2: DFT2 over n1, twiddle W8^(n2 k1), DFT4 over n2
        float2 y[4][2];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            y[n2][0] = cadd(v[n2], v[4 + n2]);
            y[n2][1] = csub(v[n2], v[4 + n2]);
        }
        y[1][1] = cmul(y[1][1], w16<SIGN>(2));
        y[2][1] = mul_si<SIGN>(y[2][1]);
        y[3][1] = cmul(y[3][1], w16<SIGN>(6));
#pragma unroll
        for (int k1 = 0; k1 < 2; ++k1) {
            dft4<SIGN>(y[0][k1], y[1][k1], y[2][k1], y[3][k1]);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 2 * k2] = y[k2][k1];
        }
    } else if (R == 16) {
        // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            y[n2][0] = v[n2];
            y[n2][1] = v[4 + n2];
            y[n2][2] = v[8 + n2];
            y[n2][3] = v[12 + n2];
            dft4<SIGN>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
        }
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = cmul(y[n2][k1], w16<SIGN>(n2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            dft4<SIGN>(y[0][k1], y[1][k1], y[2][k1], y[3][k1]);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = y[k2][k1];
        }
    }
}

// Transform stride (in padded elements) for cnt transforms of length n kept
// back to back: the padded length rounded up to 4 (mod 16).  Element i of
// transforms 0..3 then falls 32 bytes apart in the bank space, so a
// half-warp that touches the same index of the even/odd pair of two column
// pairs (the column passes' staging and output loops) hits four disjoint
// bank groups; the FFT stages themselves never mix transforms in a warp.
__host__ __device__ constexpr int fft_tstride(int n) {
    return spad_size(n) + ((20 - (spad_size(n) & 15)) & 15);
}

// Per-stage twiddle tables of a length-n FFT (n = 2^log2n), concatenated for
// the stages after the first: stage (Ns, R) holds W_n^(q k n / (Ns R)) at
// [(q - 1) * Ns + k], q = 1..R-1, k = 0..Ns-1, so the lanes of a warp (k
// consecutive) read consecutive words (coalesced global / L1 reads).  Total
// entries: fft_twiddle_count(n).
__host__ __device__ constexpr int fft_twiddle_count(int log2n) {
    int logNs = 0, total = 0;
    while (log2n - logNs > 0) {
        const int lr = (log2n - logNs >= 4) ? 4 : (log2n - logNs);
        if (logNs > 0) total += ((1 << lr) - 1) << logNs;
        logNs += lr;
    }
    return total;
}

// One in-place Stockham stage of radix R over cnt transforms (stride ts).
// Every thread loads its IT butterflies, the block synchronises, then all
// store.
template <int SIGN, int R, int LOGR, int IT>
__device__ __forceinline__ void stockham_stage(float2 *s, int log2n, int cnt, int ts, int Ns, int logNs,
                                               const float2 *__restrict__ tws) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int logper = log2n - LOGR, per = 1 << logper;
    const int total = cnt << logper;
    float2 v[IT][R];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = tid + i * nt;
        if (it < total) {
            const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
            float2 *src = s + tr * ts;
            v[i][0] = src[spad(j)];
            if (logNs == 0) {  // first stage: every twiddle is 1
#pragma unroll
                for (int q = 1; q < R; ++q) v[i][q] = src[spad(j + q * per)];
            } else {
#pragma unroll
                for (int q = 1; q < R; ++q)
                    v[i][q] = cmul(src[spad(j + q * per)], tw_get<SIGN>(tws, ((q - 1) << logNs) + k));
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = tid + i * nt;
        if (it < total) {
            const int tr = it >> logper, j = it & (per - 1), k = j & (Ns - 1);
            dft_reg<SIGN, R>(v[i]);
            float2 *dst = s + tr * ts;
            const int base = ((j >> logNs) << (logNs + LOGR)) + k;
#pragma unroll
            for (int q = 0; q < R; ++q) dst[spad(base + q * Ns)] = v[i][q];
        }
    }
    __syncthreads();
}

// In-place FFT of cnt length-n transforms (n = 2^log2n) in the padded shared
// buffer s, transform t at s + t * ts: radix-16 stages, then one radix-8/4/2
// stage.  tw: the per-stage twiddle tables (fft_twiddle_count(log2n)
// entries).  Requires blockDim.x >= cnt * n / 16.
template <int SIGN>
__device__ void fft_pow2(float2 *s, int n, int log2n, int cnt, int ts, const float2 *__restrict__ tw) {
    int logNs = 0, toff = 0;
    while (log2n - logNs >= 4) {
        stockham_stage<SIGN, 16, 4, 1>(s, log2n, cnt, ts, 1 << logNs, logNs, tw + toff);
        if (logNs > 0) toff += 15 << logNs;
        logNs += 4;
    }
    const int rem = log2n - logNs;
    if (rem == 3) stockham_stage<SIGN, 8, 3, 2>(s, log2n, cnt, ts, 1 << logNs, logNs, tw + toff);
    else if (rem == 2) stockham_stage<SIGN, 4, 2, 4>(s, log2n, cnt, ts, 1 << logNs, logNs, tw + toff);
    else if (rem == 1) stockham_stage<SIGN, 2, 1, 8>(s, log2n, cnt, ts, 1 << logNs, logNs, tw + toff);
}

// ---------------------------------------------------------------------------
// The same FFT with the length fixed at compile time (n = 2^LOGN): every
// shared-memory and twiddle offset within a butterfly is a constant, so each
// access is a single instruction on a per-thread base address.  The padded
// index is linear in the butterfly leg q: spad(j + q per) = spad(j) +
// q (per + per/16) when per is a multiple of 16, and spad(b + q Ns) = spad(b) +
// q (Ns + Ns/16) for Ns a multiple of 16 (Ns = 1: spad(b) + q, b = R j).

// offset of the twiddle table of the stage starting at Ns = 2^logns
__host__ __device__ constexpr int fft_twiddle_offset(int logns) {
    return logns <= 4 ? 0 : fft_twiddle_offset(logns - 4) + (15 << (logns - 4));
}

// v[q] *= W^q, q = 1..R-1, from the table entries at q = 1, 2, 4, 8 (tk: the
// leg-1 entry of this butterfly, stride NS between legs): the other powers
// are products of at most three of them.
template <int SIGN, int R, int NS>
__device__ __forceinline__ void apply_stage_twiddles(float2 *v, const float2 *__restrict__ tk) {
    float2 w[R];
    w[1] = tw_get<SIGN>(tk, 0);
    if constexpr (R > 2) w[2] = tw_get<SIGN>(tk, NS);
    if constexpr (R > 4) w[4] = tw_get<SIGN>(tk, 3 * NS);
    if constexpr (R > 8) w[8] = tw_get<SIGN>(tk, 7 * NS);
    if constexpr (R > 2) w[3] = cmul(w[2], w[1]);
    if constexpr (R > 4) {
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
    }
    if constexpr (R > 8) {
#pragma unroll
        for (int q = 9; q < 16; ++q) w[q] = cmul(w[8], w[q - 8]);
    }
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], w[q]);
}

template <int SIGN, int LOGN, int LOGR, int LOGNS, int IT>
__device__ __forceinline__ void stockham_stage_ct(float2 *s, int cnt, const float2 *__restrict__ tw) {
    constexpr int R = 1 << LOGR, LOGPER = LOGN - LOGR, PER = 1 << LOGPER, NS = 1 << LOGNS;
    constexpr int TS = fft_tstride(1 << LOGN);
    constexpr int LSTRIDE = PER + PER / 16;
    constexpr int SSTRIDE = NS == 1 ? 1 : NS + NS / 16;
    static_assert(NS == 1 || NS % 16 == 0, "stage offsets assume Ns = 1 or a multiple of 16");
    const float2 *tws = tw + fft_twiddle_offset(LOGNS);
    const int nt = blockDim.x, tid = threadIdx.x, total = cnt << LOGPER;
    float2 v[IT][R];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = tid + i * nt;
        if (it < total) {
            const int tr = it >> LOGPER, j = it & (PER - 1);
            const float2 *src = s + tr * TS;
            if constexpr (PER % 16 == 0) {
                const float2 *sj = src + spad(j);
#pragma unroll
                for (int q = 0; q < R; ++q) v[i][q] = sj[q * LSTRIDE];
            } else {
#pragma unroll
                for (int q = 0; q < R; ++q) v[i][q] = src[spad(j + q * PER)];
            }
            if constexpr (LOGNS > 0) apply_stage_twiddles<SIGN, R, NS>(v[i], tws + (j & (NS - 1)));
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = tid + i * nt;
        if (it < total) {
            const int tr = it >> LOGPER, j = it & (PER - 1);
            dft_reg<SIGN, R>(v[i]);
            const int base = ((j >> LOGNS) << (LOGNS + LOGR)) + (j & (NS - 1));
            float2 *dst = s + tr * TS + spad(base);
#pragma unroll
            for (int q = 0; q < R; ++q) dst[q * SSTRIDE] = v[i][q];
        }
    }
    __syncthreads();
}

// In-place FFT of cnt length-2^LOGN transforms at s + t * fft_tstride(n);
// same stages, tables and requirement (blockDim.x >= cnt * n / 16) as fft_pow2.
template <int SIGN, int LOGN, int LOGNS = 0>
__device__ __forceinline__ void fft_ct(float2 *s, int cnt, const float2 *__restrict__ tw) {
    if constexpr (LOGN - LOGNS >= 4) {
        stockham_stage_ct<SIGN, LOGN, 4, LOGNS, 1>(s, cnt, tw);
        fft_ct<SIGN, LOGN, LOGNS + 4>(s, cnt, tw);
    } else if constexpr (LOGN - LOGNS == 3) {
        stockham_stage_ct<SIGN, LOGN, 3, LOGNS, 2>(s, cnt, tw);
    } else if constexpr (LOGN - LOGNS == 2) {
        stockham_stage_ct<SIGN, LOGN, 2, LOGNS, 4>(s, cnt, tw);
    } else if constexpr (LOGN - LOGNS == 1) {
        stockham_stage_ct<SIGN, LOGN, 1, LOGNS, 8>(s, cnt, tw);
    }
}

// The first (radix-16) stage of fft_ct with map(t, k, v) applied to every
// input element v = s[t][k] (k in natural order) as it is loaded, so an
// elementwise product needs no pass of its own over the buffer.  The other
// stages follow with fft_ct<SIGN, LOGN, 4> (or fft_ct_pair_emit<..., 4>).
// Requires LOGN >= 4 and blockDim.x >= cnt * n / 16.
template <int SIGN, int LOGN, class Map>
__device__ __forceinline__ void fft_ct_first_mapped(float2 *s, int cnt, Map &&map) {
    static_assert(LOGN >= 4, "the first stage is radix 16");
    constexpr int R = 16, LOGR = 4, LOGPER = LOGN - LOGR, PER = 1 << LOGPER;
    constexpr int TS = fft_tstride(1 << LOGN);
    constexpr int LSTRIDE = PER + PER / 16;
    const int it = threadIdx.x;
    const bool act = it < (cnt << LOGPER);
    const int tr = it >> LOGPER, j = it & (PER - 1);
    float2 v[R];
    if (act) {
        const float2 *src = s + tr * TS;
        if constexpr (PER % 16 == 0) {
            const float2 *sj = src + spad(j);
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = map(tr, j + q * PER, sj[q * LSTRIDE]);
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = map(tr, j + q * PER, src[spad(j + q * PER)]);
        }
    }
    __syncthreads();
    if (act) {
        dft_reg<SIGN, R>(v);
        float2 *dst = s + tr * TS + spad(j << LOGR);  // Ns = 1: outputs 16 j .. 16 j + 15
#pragma unroll
        for (int q = 0; q < R; ++q) dst[q] = v[q];
    }
    __syncthreads();
}

// exp(-2 pi i q / 32) times -1 for q >= 8, q = 0..15: the factor by which the
// G = 2n grid twiddle exp(-2 pi i (ix - n/2) / G) of input j + ((q + 8) mod 16) n/16
// differs from that of input j + n/2 (see fft_first_from_row).
__device__ __forceinline__ float2 w32_signed(int q) {
    const float c[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                        0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                        0.19509032201612826785f, 0.0f};
    // cos(q pi/16), sin(q pi/16) for q = 0..15 from the first quadrant
    const float cr = q <= 8 ? c[q] : -c[16 - q];
    const float si = q <= 8 ? c[8 - q] : c[q - 8];
    const float sg = q >= 8 ? -1.0f : 1.0f;
    return make_float2(sg * cr, -sg * si);
}

// The first (radix-16) stage of the even/odd pair of transforms that give the
// G = 2n point DFT of one row of n samples (n = 2^LOGN): transform 0 takes
// x[(k + n/2) mod n] at FFT index k, transform 1 the same times the grid
// twiddle tw[(k + n/2) mod n], tw[i] = exp(-2 pi i (i - n/2) / G).  The
// inputs come straight from global memory (row: n contiguous values) into
// registers, so the row is never staged in shared memory; thread t runs
// butterfly t mod n/16 of transform t / (n/16), writes its 16 outputs to
// the padded buffer (transform stride fft_tstride(n)) and the block
// synchronises.  The remaining stages follow with fft_ct<SIGN, LOGN, 4>.
// Requires blockDim.x >= n / 8.
template <int SIGN, int LOGN>
__device__ __forceinline__ void fft_first_from_row(float2 *s, const float2 *__restrict__ row,
                                                   const float2 *__restrict__ tw) {
    static_assert(LOGN >= 4, "the first stage is radix 16");
    constexpr int N = 1 << LOGN, PER = N / 16, TS = fft_tstride(N);
    const int t = threadIdx.x;
    if (t < 2 * PER) {
        const int tr = t / PER, j = t % PER;
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = row[j + ((q + 8) & 15) * PER];
        if (tr == 1) {
            const float2 wj = tw[j + N / 2];  // exp(-2 pi i j / G)
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], q == 0 ? wj : cmul(wj, w32_signed(q)));
        }
        dft_reg<SIGN, 16>(v);
        float2 *dst = s + tr * TS + spad(j << 4);  // Ns = 1: outputs 16 j .. 16 j + 15
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[q] = v[q];
    }
    __syncthreads();
}

// A pair of transforms (cnt = 2) of length 2^LOGN, LOGN = 3 (mod 4), run with
// blockDim.x == n / 8: the last (radix-8) stage then gives each thread one
// butterfly of each transform at the same index, and instead of storing it
// calls emit(k, X0[k], X1[k]) for its eight output indices k (natural order;
// a warp's k are consecutive).  The shared buffer keeps the second-to-last
// stage's result.
template <int SIGN, int LOGN, int LOGNS = 0, class Emit>
__device__ __forceinline__ void fft_ct_pair_emit(float2 *s, const float2 *__restrict__ tw, Emit &&emit) {
    if constexpr (LOGN - LOGNS >= 4) {
        stockham_stage_ct<SIGN, LOGN, 4, LOGNS, 1>(s, 2, tw);
        fft_ct_pair_emit<SIGN, LOGN, LOGNS + 4>(s, tw, emit);
    } else {
        static_assert(LOGN - LOGNS == 3, "the last stage is radix 8");
        constexpr int R = 8, LOGR = 3, PER = 1 << (LOGN - LOGR), NS = 1 << LOGNS;
        constexpr int TS = fft_tstride(1 << LOGN), LSTRIDE = PER + PER / 16;
        const int j = threadIdx.x;  // < PER = blockDim.x
        float2 v[2][R];
#pragma unroll
        for (int tr = 0; tr < 2; ++tr) {
            const float2 *sj = s + tr * TS + spad(j);
#pragma unroll
            for (int q = 0; q < R; ++q) v[tr][q] = sj[q * LSTRIDE];
            if constexpr (LOGNS > 0)
                apply_stage_twiddles<SIGN, R, NS>(v[tr], tw + fft_twiddle_offset(LOGNS) + (j & (NS - 1)));
            dft_reg<SIGN, R>(v[tr]);
        }
        const int base = ((j >> LOGNS) << (LOGNS + LOGR)) + (j & (NS - 1));
#pragma unroll
        for (int q = 0; q < R; ++q) emit(base + q * NS, v[0][q], v[1][q]);
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

// Bluestein's chirp-z DFT of length D through two length-L power-of-two FFTs:
// nk = (n^2 + k^2 - (k - n)^2) / 2 turns the DFT into a convolution with the
// chirp, evaluated cyclically with L >= 2D - 1.  On entry s[spad(n)], n < D,
// holds the input; on exit s[spad(k)], k < D, holds sum_n x_n exp(SIGN 2 pi i
// nk / D).  The +1 direction is conj(DFT_-(conj x)).  Requires blockDim.x >=
// L / 16; s has spad_size(L) elements.
template <int SIGN>
__device__ void bluestein(float2 *s, int D, int L, int log2L, const float2 *__restrict__ chirp,
                          const float2 *__restrict__ bhat, const float2 *__restrict__ twL) {
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        float2 a = make_float2(0.f, 0.f);
        if (n < D) {
            float2 v = s[spad(n)];
            if (SIGN > 0) v.y = -v.y;
            a = cmul(v, chirp[n]);
        }
        s[spad(n)] = a;
    }
    __syncthreads();
    fft_pow2<-1>(s, L, log2L, 1, 0, twL);
    for (int n = threadIdx.x; n < L; n += blockDim.x) s[spad(n)] = cmul(s[spad(n)], bhat[n]);
    __syncthreads();
    fft_pow2<+1>(s, L, log2L, 1, 0, twL);
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        float2 v = cmul(s[spad(k)], chirp[k]);
        if (SIGN > 0) v.y = -v.y;
        s[spad(k)] = v;
    }
    __syncthreads();
}

// The same with L = 2^LOGL fixed at compile time (fft_ct offsets).
template <int SIGN, int LOGL>
__device__ void bluestein_ct(float2 *s, int D, const float2 *__restrict__ chirp,
                             const float2 *__restrict__ bhat, const float2 *__restrict__ twL) {
    constexpr int L = 1 << LOGL;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        float2 a = make_float2(0.f, 0.f);
        if (n < D) {
            float2 v = s[spad(n)];
            if (SIGN > 0) v.y = -v.y;
            a = cmul(v, chirp[n]);
        }
        s[spad(n)] = a;
    }
    __syncthreads();
    fft_ct<-1, LOGL>(s, 1, twL);
    for (int n = threadIdx.x; n < L; n += blockDim.x) s[spad(n)] = cmul(s[spad(n)], bhat[n]);
    __syncthreads();
    fft_ct<+1, LOGL>(s, 1, twL);
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        float2 v = cmul(s[spad(k)], chirp[k]);
        if (SIGN > 0) v.y = -v.y;
        s[spad(k)] = v;
    }
    __syncthreads();
}
