// Pass bodies of the NUFFT Radon projector A and back-projector A^T
// (arXiv 2304.12934, Sec. 2.2 Eqs. nufft, nufft2, nufft3 and their reverse
// order; Sec. 3 Eq. transpose), and the per-plan kernels that run them on a
// (tile, slice) grid.  Included by radon_kernels.cu (per-plan launchers) and
// group_kernels.cu (persistent launches over several geometries); everything
// here has internal linkage, so each translation unit instantiates what it
// uses.
//
// Forward, per slice (image f, N x N, grid G = 2N, kernel width w):
//   col pass   deapodise by 1/(psi(x) psi(y)) and FFT_G along y of two real
//              columns packed as one complex column; keep grid rows
//              jy = jmin..jmax (the half plane touched by the polar points)
//   row pass   FFT_G along x of one grid row (G outputs from N non-zero
//              inputs, as two N-point FFTs), then the interpolation partial
//              phi(gy - jy) * sum_t phi(gx - jx_t) F(jx_t, jy) of every polar
//              point whose y-footprint contains the row, stored per tap row
//              (no atomics: every (point, tap row) slot has one writer)
//   det pass   sum the w partials of each point, C2R inverse DFT of length D
//              of two angles packed as one complex row, scale 1/D, epilogue
// Adjoint, per slice, the transposes in reverse order:
//   det pass   real-to-complex DFT of two sinogram rows, Hermitian weights
//   row pass   spread by gather: every grid cell of the row sums the polar
//              points whose footprint covers it, read from per-row bins
//              sorted by jx0 (atomic-free, fixed summation order), then an
//              inverse FFT_G along x evaluated at the N image columns
//   col pass   Hermitian completion, inverse FFT_G along y at the N image
//              rows for two columns at once, real part, deapodise
#pragma once
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace {

// Shared-memory slot of cell c of a G-row kept as two N-point transforms
// [even cells | odd cells], the even one being transform t0 (stride ts).
__host__ __device__ constexpr int cell_slot(int t0, int ts, int c) {
    return (t0 + (c & 1)) * ts + spad(c >> 1);
}

#ifndef TC_ADJ_ROW_REC_UNROLL
#define TC_ADJ_ROW_REC_UNROLL 1
#endif
#ifndef TC_ADJ_ROW_REC_PREFETCH
#define TC_ADJ_ROW_REC_PREFETCH 2
#endif
#ifndef TC_FWD_ROW_INTERP_UNROLL
#define TC_FWD_ROW_INTERP_UNROLL 4
#endif
// loop iterations unrolled so that their table loads are in flight together:
// the spreading pass's records, the interpolation's entries
constexpr int kAdjRowRecUnroll = TC_ADJ_ROW_REC_UNROLL;
constexpr int kRecAhead = TC_ADJ_ROW_REC_PREFETCH > 0 ? TC_ADJ_ROW_REC_PREFETCH : 1;   // records read ahead
constexpr int kFwdRowInterpUnroll = TC_FWD_ROW_INTERP_UNROLL;

// ------------------------------------------------------------ forward ------
// The pass kernels take the image side as a template parameter (N = 2^LOGN),
// so their FFTs and shared-memory layouts are fixed at compile time.
// TMA: the CTA's strip of 2CP image columns (N rows x 16 or 32 bytes, the
// partial-sector reads that bound the L1 path) is staged in shared memory by
// bulk tensor copies, outside the LSU/L1 pipeline (CP >= 2).
// The pass bodies take their tile (or grid row, or angle pair) and slice
// indices as arguments: the per-plan kernels pass blockIdx, the grouped
// kernels (group_kernels.cu) the item they took from their work list.
template <int LOGN, bool TMA>
__device__ __forceinline__ void fwd_col_body(const float *__restrict__ x, float2 *__restrict__ T, const KArgs &g,
                                             int CP, const CUtensorMap *tmx, int *__restrict__ err, int tile,
                                             int b) {
    extern __shared__ float2 sm[];  // 2CP transforms (stride ts) [, strip, barrier]
    constexpr int N = 1 << LOGN, ts = fft_tstride(N);
    const int x0base = tile * CP * 2;
    const float *src = x + (size_t)b * N * N + x0base;  // row iy of the strip at src + iy * pitch
    int pitch = N;
    if constexpr (TMA) {
        const unsigned base = smem_u32(sm + 2 * CP * ts);
        float *strip = reinterpret_cast<float *>(reinterpret_cast<char *>(sm + 2 * CP * ts) +
                                                 (((base + 127u) & ~127u) - base));
        uint64_t *bar = reinterpret_cast<uint64_t *>(strip + N * 2 * CP);
        constexpr int BR = N < 256 ? N : 256;  // rows per box (a box side is at most 256)
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (unsigned)(N * 2 * CP * sizeof(float)));
            for (int r = 0; r < N; r += BR) tma_load_3d(strip + r * 2 * CP, tmx, bar, x0base, r, b);
        }
        __syncthreads();
        const bool late = !mbar_wait(bar, 0, err);
        if (__syncthreads_or(late)) return;  // all threads leave together
        src = strip;
        pitch = 2 * CP;
    }
    // blockDim.x is a multiple of CP, so a thread keeps its column pair
    const int pp0 = threadIdx.x % CP, xc0 = x0base + 2 * pp0;
    const float dx0 = g.dea[xc0], dx1 = g.dea[xc0 + 1];
#pragma unroll 8
    for (int idx = threadIdx.x; idx < N * CP; idx += blockDim.x) {
        const int pp = pp0, iy = idx / CP;
        const float2 f = *reinterpret_cast<const float2 *>(src + (size_t)iy * pitch + 2 * pp0);
        const float dy = g.dea[iy];
        const float2 z = make_float2(f.x * dx0 * dy, f.y * dx1 * dy);
        const int q = (iy - N / 2) & (N - 1);
        sm[(pp * 2) * ts + spad(q)] = z;
        sm[(pp * 2 + 1) * ts + spad(q)] = cmul(z, g.twG[iy]);
    }
    __syncthreads();
    fft_ct<-1, LOGN>(sm, 2 * CP, g.twN);
    float2 *Tb = T + (size_t)b * g.R * N;
    constexpr int Gm = 2 * N - 1;
    // the two real columns of pair pp in grid row r, packed as in T
    auto row_out = [&](int pp, int r) {
        const int jy = g.jmin + r;
        const float2 zp = sm[cell_slot(pp * 2, ts, jy & Gm)];
        const float2 zm = cconj(sm[cell_slot(pp * 2, ts, (-jy) & Gm)]);
        const float2 d = csub(zp, zm);
        float4 o;
        o.x = 0.5f * (zp.x + zm.x);
        o.y = 0.5f * (zp.y + zm.y);
        o.z = 0.5f * d.y;   // (zp - zm) / (2i)
        o.w = -0.5f * d.x;
        return o;
    };
#pragma unroll 4
    for (int idx = threadIdx.x; idx < g.R * CP; idx += blockDim.x) {
        const int pp = idx % CP, r = idx / CP;
        *reinterpret_cast<float4 *>(Tb + (size_t)r * N + x0base + 2 * pp) = row_out(pp, r);
    }
}

template <int LOGN, bool TMA>
__global__ void __launch_bounds__(512) k_fwd_col(const float *__restrict__ x, float2 *__restrict__ T,
                          const KArgs g, int CP, const __grid_constant__ CUtensorMap tmx,
                          int *__restrict__ err) {
    fwd_col_body<LOGN, TMA>(x, T, g, CP, &tmx, err, blockIdx.x, blockIdx.y);
}

template <int LOGN>
__device__ __forceinline__ void fwd_row_body(const float2 *__restrict__ T, float2 *__restrict__ P, const KArgs &g,
                                             int r, int b) {
    extern __shared__ float2 sm[];  // 2 transforms (stride ts)
    constexpr int N = 1 << LOGN, ts = fft_tstride(N);
    const float2 *Tr = T + ((size_t)b * g.R + r) * N;
    fft_first_from_row<-1, LOGN>(sm, Tr, g.twG);
    fft_ct<-1, LOGN, 4>(sm, 2, g.twN);
    float2 *Pb = P + (size_t)b * g.w * g.AM;
    const int e1 = g.row_off[r + 1];
    constexpr int Gm = 2 * N - 1;
#pragma unroll kFwdRowInterpUnroll
    for (int e = g.row_off[r] + threadIdx.x; e < e1; e += blockDim.x) {
        const int4 en = g.ent[e];
        const int key = entry_key(en);
        const float nexh = -entry_ex(en) * g.inv_h;
        float2 acc = make_float2(0.f, 0.f);
        for (int t = 0; t < g.w; ++t) {
            // z = (t - ex) / h, formed exactly as in the spreading kernel
            const float wt = es_kernel_fast(fmaf((float)t, g.inv_h, nexh), g.beta_l2);
            cfma(acc, wt, sm[cell_slot(0, ts, (key + t) & Gm)]);
        }
        Pb[(size_t)entry_s(en) * g.AM + entry_p(en)] = cscale(acc, entry_wy(en));
    }
}

template <int LOGN>
__global__ void __launch_bounds__(LOGN == 11 ? 256 : 512, LOGN == 11 ? 5 : 1)
    k_fwd_row(const float2 *__restrict__ T, float2 *__restrict__ P, const KArgs g) {
    fwd_row_body<LOGN>(T, P, g, blockIdx.x, blockIdx.y);
}

// mode bits
#define DET_WRITE_Y 1
#define DET_RESID 2
#define DET_OBJ 4

// Detector-row transforms: the generic mixed-radix Stockham (BLUE = false) or
// Bluestein through power-of-two FFTs (BLUE = true); buffer index helper.
template <bool BLUE>
__device__ __forceinline__ int didx(int i) { return BLUE ? spad(i) : i; }

// LOGL > 0: Bluestein length 2^LOGL fixed at compile time.
template <bool BLUE, int LOGL = 0>
__device__ __forceinline__ void fwd_det_body(const float2 *__restrict__ P, float *__restrict__ y,
                                             const float *__restrict__ bsino, const float *__restrict__ wsino,
                                             float *__restrict__ resid, double *__restrict__ partials,
                                             const KArgs &g, int mode, int t, int b, int nt) {
    // mixed radix: [D] bufA, [D] bufB, [D] tw, [rad0] root; Bluestein: [spad(L)] buffer
    extern __shared__ float2 sm[];
    __shared__ double red[32];
    const int D = g.D, Mh = g.Mh, A = g.A;
    const int a0 = 2 * t;
    const bool has1 = (a0 + 1) < A;
    float2 *bufA = sm, *bufB = sm + D, *tw = sm + 2 * D, *root0 = sm + 3 * D;
    if (!BLUE) {
        const int R0 = g.rp.rad[0], per0 = D / R0;
        for (int k = threadIdx.x; k < D; k += blockDim.x) tw[k] = g.twD[k];
        for (int k = threadIdx.x; k < R0; k += blockDim.x) root0[k] = g.twD[k * per0];
    }
    const float2 *Pb = P + (size_t)b * g.w * g.AM;
    for (int m = threadIdx.x; m < Mh; m += blockDim.x) {
        // the w <= 8 tap-row partials, all loads in flight before the sums
        // (taps summed in order s = 0 .. w-1)
        float2 v0[8], v1[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            v0[s] = v1[s] = make_float2(0.f, 0.f);
            if (s < g.w) {
                const float2 *pl = Pb + (size_t)s * g.AM;
                v0[s] = pl[(size_t)a0 * Mh + m];
                if (has1) v1[s] = pl[(size_t)(a0 + 1) * Mh + m];
            }
        }
        float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            if (s < g.w) {
                c0 = cadd(c0, v0[s]);
                c1 = cadd(c1, v1[s]);
            }
        }
        if (g.angle_flip[a0]) c0 = cconj(c0);
        if (has1 && g.angle_flip[a0 + 1]) c1 = cconj(c1);
        if (g.shiftD) {  // axis offset: Fourier shift of the true-angle spectrum
            const float2 e = g.shiftD[m];
            c0 = cmul(c0, e);
            c1 = cmul(c1, e);
        }
        const float sg = (m & 1) ? -1.f : 1.f;
        float2 X0 = cscale(c0, sg), X1 = cscale(c1, sg);
        if (2 * m == D) { X0.y = 0.f; X1.y = 0.f; }
        bufA[didx<BLUE>(m)] = make_float2(X0.x - X1.y, X0.y + X1.x);
        if (m > 0 && 2 * m < D) bufA[didx<BLUE>(D - m)] = make_float2(X0.x + X1.y, X1.x - X0.y);
    }
    __syncthreads();
    const float2 *res;
    if (BLUE) {
        if constexpr (LOGL > 0) bluestein_ct<+1, LOGL>(sm, D, g.chirp, g.bhat, g.twL);
        else bluestein<+1>(sm, D, g.L, g.log2L, g.chirp, g.bhat, g.twL);
        res = sm;
    } else {
        res = fft_mixed<+1>(bufA, bufB, g.rp, tw, root0);
    }
    float objv = 0.f;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const float2 z = res[didx<BLUE>(i)];
        const float yv[2] = {z.x * g.invD, z.y * g.invD};
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !has1) break;
            const size_t o = ((size_t)b * A + a0 + h) * D + i;
            float v = yv[h];
            if (mode & DET_WRITE_Y) y[o] = v;
            if (mode & DET_RESID) {
                const float r = bsino ? v - bsino[o] : v;
                const float wt = wsino ? wsino[o] : 1.f;
                resid[o] = wt * r;
                objv = fmaf(0.5f * wt * r, r, objv);
            }
        }
    }
    if (mode & DET_OBJ) {
        const double tot = block_sum_f64(objv, red);
        if (threadIdx.x == 0) partials[(size_t)b * nt + t] = tot;
    }
}

template <bool BLUE, int LOGL = 0>
__global__ void __launch_bounds__(512) k_fwd_det(const float2 *__restrict__ P, float *__restrict__ y,
                          const float *__restrict__ bsino, const float *__restrict__ wsino,
                          float *__restrict__ resid, double *__restrict__ partials,
                          const KArgs g, int mode) {
    fwd_det_body<BLUE, LOGL>(P, y, bsino, wsino, resid, partials, g, mode, blockIdx.x, blockIdx.y, gridDim.x);
}

// ------------------------------------------------------------ adjoint ------
template <bool BLUE, int LOGL = 0>
__device__ __forceinline__ void adj_det_body(const float *__restrict__ ysino, float2 *__restrict__ V, const KArgs &g,
                                             int t, int b) {
    extern __shared__ float2 sm[];
    const int D = g.D, Mh = g.Mh, A = g.A;
    const int a0 = 2 * t;
    const bool has1 = (a0 + 1) < A;
    float2 *bufA = sm, *bufB = sm + D, *tw = sm + 2 * D, *root0 = sm + 3 * D;
    if (!BLUE) {
        const int R0 = g.rp.rad[0], per0 = D / R0;
        for (int k = threadIdx.x; k < D; k += blockDim.x) tw[k] = g.twD[k];
        for (int k = threadIdx.x; k < R0; k += blockDim.x) root0[k] = g.twD[k * per0];
    }
    const float *y0 = ysino + ((size_t)b * A + a0) * D;
#pragma unroll 4
    for (int i = threadIdx.x; i < D; i += blockDim.x)
        bufA[didx<BLUE>(i)] = make_float2(y0[i], has1 ? y0[D + i] : 0.f);
    __syncthreads();
    const float2 *Z;
    if (BLUE) {
        if constexpr (LOGL > 0) bluestein_ct<-1, LOGL>(sm, D, g.chirp, g.bhat, g.twL);
        else bluestein<-1>(sm, D, g.L, g.log2L, g.chirp, g.bhat, g.twL);
        Z = sm;
    } else {
        Z = fft_mixed<-1>(bufA, bufB, g.rp, tw, root0);
    }
    float2 *Vb = V + (size_t)b * g.w * g.AM;
    for (int m = threadIdx.x; m < Mh; m += blockDim.x) {
        const float2 zp = Z[didx<BLUE>(m)];
        const float2 zm = cconj(Z[didx<BLUE>(m == 0 ? 0 : D - m)]);
        // Y_a0 = (zp + zm)/2, Y_a1 = (zp - zm)/(2i); weight mu_m nu_m (-1)^m / D
        const float mn = (m == 0 || 2 * m == D) ? 1.f : 2.f;
        const float sc = ((m & 1) ? -mn : mn) * 0.5f * g.invD;
        float2 v0 = make_float2(sc * (zp.x + zm.x), sc * (zp.y + zm.y));
        float2 e = make_float2(1.f, 0.f);
        if (g.shiftD) e = cconj(g.shiftD[m]);  // transpose of the axis-offset shift
        v0 = cmul(v0, e);
        if (g.angle_flip[a0]) v0 = cconj(v0);
        Vb[(size_t)a0 * Mh + m] = v0;
        if (has1) {
            float2 v1 = make_float2(sc * (zp.y - zm.y), -sc * (zp.x - zm.x));
            v1 = cmul(v1, e);
            if (g.angle_flip[a0 + 1]) v1 = cconj(v1);
            Vb[(size_t)(a0 + 1) * Mh + m] = v1;
        }
    }
}

template <bool BLUE, int LOGL = 0>
__global__ void __launch_bounds__(512) k_adj_det(const float *__restrict__ ysino, float2 *__restrict__ V,
                          const KArgs g) {
    adj_det_body<BLUE, LOGL>(ysino, V, g, blockIdx.x, blockIdx.y);
}

// Sum over the staged entries lo..hi-1 covering cell cs of u phi((cs - key -
// ex) / h); cs - key is an exact small integer, so the weight is bitwise the
// one the interpolation uses for the same (entry, cell).
__device__ __forceinline__ float2 spread_record(const float4 *__restrict__ ce, int cs, int lo, int hi,
                                                const KArgs &g) {
    const float csf = (float)cs;
    float2 acc = make_float2(0.f, 0.f);
    for (int i = lo; i < hi; ++i) {
        const float4 e = ce[i];
        const float wt = es_kernel_fast(fmaf(csf - e.z, g.inv_h, e.w), g.beta_l2);
        acc.x = fmaf(wt, e.x, acc.x);
        acc.y = fmaf(wt, e.y, acc.y);
    }
    return acc;
}

// Spreading of one grid row, atomic-free.  The row's (point, tap) entries are
// sorted by jx0 (the key) and taken in chunks: every thread stages one
// entry's u = phi_y * V[p], key and -(gx - jx0) / h in shared memory.  The plan holds
// one record per touched cell of the chunk, naming the contiguous range of
// entries whose footprint covers that cell (keys in [cell - w + 1, cell]);
// one thread per record sums u * phi(cell - key - (gx - jx0)) over its range
// and adds it to its cell.  Within a chunk every physical cell has one record
// (the few wrap-around duplicates at the spectrum edge are flagged and added
// serially), so no two threads touch a cell and every cell's summation order
// is fixed: atomic-free and bit-reproducible.
// The per-plan spreading kernel runs slices fastest in its grid (blockIdx.x =
// slice, blockIdx.y = grid row): the CTAs in flight share one row's entry and
// record tables, read once from DRAM per launch instead of once per slice.
// iterations of the spreading pass's entry staging, and of the inverse column
// pass's grid-row loads, unrolled so that their global loads are in flight together
#ifndef TC_ADJ_ROW_STAGE_UNROLL
#define TC_ADJ_ROW_STAGE_UNROLL 2
#endif
#ifndef TC_ADJ_COL_LOAD_UNROLL
#define TC_ADJ_COL_LOAD_UNROLL 4
#endif
constexpr int kAdjRowStageUnroll = TC_ADJ_ROW_STAGE_UNROLL;
constexpr int kAdjColLoadUnroll = TC_ADJ_COL_LOAD_UNROLL;
#ifndef TC_ADJ_ROW_SLICES_FASTEST
#define TC_ADJ_ROW_SLICES_FASTEST 1
#endif
template <int LOGN>
__device__ __forceinline__ void adj_row_body(const float2 *__restrict__ V, float2 *__restrict__ U, const KArgs &g,
                                             int r, int b) {
    extern __shared__ float2 sm[];
    constexpr int N = 1 << LOGN, G = 2 * N;
    constexpr int ts = fft_tstride(N), hsz = 2 * ts;              // grid row: 2 transforms
    // staged entries: (u = phi_y V[p], key, -ex / h); hsz is even, so 16-byte aligned
    float4 *ce = reinterpret_cast<float4 *>(sm + hsz);             // [g.chunk]
    const int e0 = g.row_off[r], e1 = g.row_off[r + 1];
    for (int c = threadIdx.x; c < hsz; c += blockDim.x) sm[c] = make_float2(0.f, 0.f);
    const float2 *Vb = V + (size_t)b * g.w * g.AM;
    const int *roff = g.rec_off + (size_t)r * (2 * g.nch + 1);
    const int chunk = g.chunk;
    for (int kc = 0, c0 = e0; c0 < e1; ++kc, c0 += chunk) {
        const int n = (e1 - c0) < chunk ? (e1 - c0) : chunk;
#pragma unroll kAdjRowStageUnroll
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int4 en = g.ent[c0 + i];
            const float2 u = cscale(Vb[entry_p(en)], entry_wy(en));
            ce[i] = make_float4(u.x, u.y, (float)entry_key(en), -entry_ex(en) * g.inv_h);
        }
        const int rb = roff[2 * kc], rs = roff[2 * kc + 1], re = roff[2 * kc + 2];
#if TC_ADJ_ROW_REC_PREFETCH
        // each thread's next kRecAhead records are read ahead (the first ones
        // before the staging barrier), so a record's table load is not waited for
        const int bd = blockDim.x;
        int q = rb + threadIdx.x;
        int2 rn[kRecAhead];
#pragma unroll
        for (int k = 0; k < kRecAhead; ++k) rn[k] = q + k * bd < rs ? g.rec[q + k * bd] : make_int2(0, 0);
        __syncthreads();
        for (; q < rs; q += bd) {
            const int2 rc = rn[0];
#pragma unroll
            for (int k = 0; k + 1 < kRecAhead; ++k) rn[k] = rn[k + 1];
            if (q + kRecAhead * bd < rs) rn[kRecAhead - 1] = g.rec[q + kRecAhead * bd];
            const int cs = (rc.x & 0x7fff) + g.kmin;
            const float2 acc = spread_record(ce, cs, rc.y & 0xffff, rc.y >> 16, g);
            float2 &hc = sm[cell_slot(0, ts, cs & (G - 1))];
            hc = cadd(hc, acc);
        }
#else
        __syncthreads();
#pragma unroll kAdjRowRecUnroll
        for (int q = rb + threadIdx.x; q < rs; q += blockDim.x) {
            const int2 rc = g.rec[q];
            const int cs = (rc.x & 0x7fff) + g.kmin;
            const float2 acc = spread_record(ce, cs, rc.y & 0xffff, rc.y >> 16, g);
            float2 &hc = sm[cell_slot(0, ts, cs & (G - 1))];
            hc = cadd(hc, acc);
        }
#endif
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = rs; q < re; ++q) {  // seam records, in order
                const int2 rc = g.rec[q];
                const int cs = (rc.x & 0x7fff) + g.kmin;
                const float2 acc = spread_record(ce, cs, rc.y & 0xffff, rc.y >> 16, g);
                float2 &hc = sm[cell_slot(0, ts, cs & (G - 1))];
                hc = cadd(hc, acc);
            }
        }
        __syncthreads();
    }
    float2 *Ur = U + ((size_t)b * g.R + r) * N;
    if constexpr (LOGN % 4 == 3) {
        if (blockDim.x == N / 8) {  // the last FFT stage writes the image row directly
            fft_ct_pair_emit<+1, LOGN>(sm, g.twN, [&](int q, float2 x0, float2 x1) {
                const int ix = (q + N / 2) & (N - 1);
                Ur[ix] = cadd(x0, cmul(x1, cconj(g.twG[ix])));
            });
            return;
        }
    }
    fft_ct<+1, LOGN>(sm, 2, g.twN);
#pragma unroll 4
    for (int ix = threadIdx.x; ix < N; ix += blockDim.x) {
        const int q = (ix - N / 2) & (N - 1);
        Ur[ix] = cadd(sm[spad(q)], cmul(sm[ts + spad(q)], cconj(g.twG[ix])));
    }
}

template <int LOGN>
__global__ void __launch_bounds__(512) k_adj_row(const float2 *__restrict__ V, float2 *__restrict__ U,
                          const KArgs g) {
    adj_row_body<LOGN>(V, U, g, TC_ADJ_ROW_SLICES_FASTEST ? blockIdx.y : blockIdx.x,
                       TC_ADJ_ROW_SLICES_FASTEST ? blockIdx.x : blockIdx.y);
}

// Epilogues of the inverse column pass.
#define COL_DEAPOD 0  // adjoint: x = Re(.) / (psi(x) psi(y))
#define COL_PLAIN 1   // normal operator: out = Re(.)
#define COL_GRAD 2    // normal-operator gradient: out = Re(.) - sub; with xdot, the
                      // block's FP64 partial of <xdot, out - sub> in part

template <int LOGN, int EPI>
__device__ __forceinline__ void adj_col_body(const float2 *__restrict__ U, float *__restrict__ x, const KArgs &g,
                                             int CP, const float *__restrict__ sub, const float *__restrict__ xdot,
                                             double *__restrict__ part, int tile, int b, int nt) {
    extern __shared__ float2 sm[];  // 2CP transforms (stride ts)
    constexpr int N = 1 << LOGN, G = 2 * N, ts = fft_tstride(N);
    const int x0base = tile * CP * 2;
    const float2 *Ub = U + (size_t)b * g.R * N;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // cells jy and G - jy (jy = 0..N) come from the same two grid rows: one
    // pair of loads gives both (the second cell's Hermitian parts are the
    // conjugates of the first's)
#pragma unroll kAdjColLoadUnroll
    for (int idx = threadIdx.x; idx < (N + 1) * CP; idx += blockDim.x) {
        const int pp = idx % CP, jy = idx / CP;
        const int xc = x0base + 2 * pp;
        const int jn = (G - jy) & (G - 1);
        const int js_p = jy <= g.jmax ? jy : jy - G;
        const int js_n = jn <= g.jmax ? jn : jn - G;
        const float4 up = (js_p >= g.jmin)
            ? *reinterpret_cast<const float4 *>(Ub + (size_t)(js_p - g.jmin) * N + xc) : zero4;
        const float4 un = (js_n >= g.jmin)
            ? *reinterpret_cast<const float4 *>(Ub + (size_t)(js_n - g.jmin) * N + xc) : zero4;
        // Hermitian parts of the two columns, packed as H0 + i H1
        const float h0x = 0.5f * (up.x + un.x), h0y = 0.5f * (up.y - un.y);
        const float h1x = 0.5f * (up.z + un.z), h1y = 0.5f * (up.w - un.w);
        sm[cell_slot(pp * 2, ts, jy)] = make_float2(h0x - h1y, h0y + h1x);
        if (jn != jy) sm[cell_slot(pp * 2, ts, jn)] = make_float2(h0x + h1y, h1x - h0y);
    }
    __syncthreads();
    fft_ct<+1, LOGN>(sm, 2 * CP, g.twN);
    const size_t sb = (size_t)b * N * N;
    // blockDim.x is a multiple of CP, so a thread keeps its column pair
    const int pp = threadIdx.x % CP, xc = x0base + 2 * pp;
    float dx0 = 1.f, dx1 = 1.f;
    if constexpr (EPI == COL_DEAPOD) {
        dx0 = g.dea[xc];
        dx1 = g.dea[xc + 1];
    }
    double acc = 0.0;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < N * CP; idx += blockDim.x) {
        const int iy = idx / CP;
        const int q = (iy - N / 2) & (N - 1);
        const float2 v = cadd(sm[(pp * 2) * ts + spad(q)],
                              cmul(sm[(pp * 2 + 1) * ts + spad(q)], cconj(g.twG[iy])));
        const size_t off = sb + (size_t)iy * N + xc;
        float2 o = v;
        if constexpr (EPI == COL_DEAPOD) {
            const float dy = g.dea[iy];
            o = make_float2(v.x * dx0 * dy, v.y * dx1 * dy);
        }
        if constexpr (EPI == COL_GRAD) {
            const float2 r = *reinterpret_cast<const float2 *>(sub + off);
            o = make_float2(v.x - r.x, v.y - r.y);
            if (xdot) {
                const float2 xv = *reinterpret_cast<const float2 *>(xdot + off);
                acc += (double)fmaf(xv.y, o.y - r.y, xv.x * (o.x - r.x));
            }
        }
        *reinterpret_cast<float2 *>(x + off) = o;
    }
    if constexpr (EPI == COL_GRAD) {
        if (xdot) {  // uniform over the grid
            __shared__ double red[32];
            const double tot = block_sum_f64(acc, red);
            if (threadIdx.x == 0) part[(size_t)b * nt + tile] = tot;
        }
    }
}

template <int LOGN, int EPI>
__global__ void __launch_bounds__(512) k_adj_col(const float2 *__restrict__ U, float *__restrict__ x,
                          const KArgs g, int CP, const float *__restrict__ sub,
                          const float *__restrict__ xdot, double *__restrict__ part) {
    adj_col_body<LOGN, EPI>(U, x, g, CP, sub, xdot, part, blockIdx.x, blockIdx.y, gridDim.x);
}

// Row pass of the normal operator A^T A on the 2N-periodic grid (Toeplitz
// plus Hankel embedding; the derivation is in normal.cu).  One grid row ky of
// the column spectra per CTA, in place: FFT_G along x (G outputs from the N
// non-zero inputs, as two N-point FFTs), the embedded kernels applied as
// Y = T^ F + H^ conj(F) (the image is real, so F(-k) = conj F(k)) while the
// inverse transform's first stage loads F, and the inverse FFT_G evaluated at
// the N image columns.  The grid runs over slices fastest (blockIdx.x = slice,
// blockIdx.y = row), so the CTAs in flight share a few table rows in L2.
// For N = 2048 the row passes run N/8 = 256 threads: four CTAs per SM fit in
// 64 registers a thread.
template <int LOGN>
__global__ void __launch_bounds__(LOGN == 11 ? 256 : 512, LOGN == 11 ? 4 : 1)
    k_nrm_row(float2 *__restrict__ U, const float *__restrict__ tt,
                          const float2 *__restrict__ th, const KArgs g) {
    extern __shared__ float2 sm[];  // 2 transforms (stride ts)
    constexpr int N = 1 << LOGN, ts = fft_tstride(N);
    const int b = blockIdx.x, r = blockIdx.y;
    float2 *Ur = U + ((size_t)b * g.R + r) * N;
    fft_first_from_row<-1, LOGN>(sm, Ur, g.twG);
    fft_ct<-1, LOGN, 4>(sm, 2, g.twN);
    // cell c = 2j + t of the row sits in transform t at j; the tables use the same order
    const float *tr = tt + (size_t)r * 2 * N;
    const float2 *hr = th + (size_t)r * 2 * N;
    fft_ct_first_mapped<+1, LOGN>(sm, 2, [&](int t, int j, float2 f) {
        const int i = t * N + j;
        const float2 h = hr[i];
        const float a = tr[i];
        return make_float2(fmaf(a, f.x, fmaf(h.x, f.x, h.y * f.y)), fmaf(a, f.y, fmaf(h.y, f.x, -h.x * f.y)));
    });
    if constexpr (LOGN % 4 == 3) {
        if (blockDim.x == N / 8) {  // the last FFT stage writes the row directly
            fft_ct_pair_emit<+1, LOGN, 4>(sm, g.twN, [&](int q, float2 x0, float2 x1) {
                const int ix = (q + N / 2) & (N - 1);
                Ur[ix] = cadd(x0, cmul(x1, cconj(g.twG[ix])));
            });
            return;
        }
    }
    fft_ct<+1, LOGN, 4>(sm, 2, g.twN);
#pragma unroll 4
    for (int ix = threadIdx.x; ix < N; ix += blockDim.x) {
        const int q = (ix - N / 2) & (N - 1);
        Ur[ix] = cadd(sm[spad(q)], cmul(sm[ts + spad(q)], cconj(g.twG[ix])));
    }
}

// Calls f(std::integral_constant<int, L>) for the supported image sides
// N = 2^L, 16 <= N <= 4096.
template <class F>
int with_logn(int lg, F &&f) {
    switch (lg) {
        case 4: return f(std::integral_constant<int, 4>{});
        case 5: return f(std::integral_constant<int, 5>{});
        case 6: return f(std::integral_constant<int, 6>{});
        case 7: return f(std::integral_constant<int, 7>{});
        case 8: return f(std::integral_constant<int, 8>{});
        case 9: return f(std::integral_constant<int, 9>{});
        case 10: return f(std::integral_constant<int, 10>{});
        case 11: return f(std::integral_constant<int, 11>{});
        case 12: return f(std::integral_constant<int, 12>{});
        default: return TC_ERR_UNSUPPORTED;
    }
}

// Bluestein lengths L = 2^8 .. 2^13 (the plan caps L at 8192) get compile-time
// FFTs; other lengths keep the run-time form.
template <class F>
void with_logl(int lg, F &&f) {
    switch (lg) {
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 9: f(std::integral_constant<int, 9>{}); break;
        case 10: f(std::integral_constant<int, 10>{}); break;
        case 11: f(std::integral_constant<int, 11>{}); break;
        case 12: f(std::integral_constant<int, 12>{}); break;
        case 13: f(std::integral_constant<int, 13>{}); break;
        default: f(std::integral_constant<int, 0>{}); break;
    }
}

}  // namespace
