// qGGMRF prior value and gradient (arXiv 2304.12934, Sec. 3 Eqs. reg2, reg3)
// on a volume [B][N][N] of consecutive slices, and the solver's restart-test
// inner products fused into the same pass.
//
//   H(f) = sum_m sum_{n in N(m)} w_mn rho(f_m - f_n),
//   rho(d) = u^2 / (c + |u|^(2-p)),  u = d / sigma,
// with w_mn proportional to 1/||m - n|| (unit sum over the 8 or 26
// neighbours) and neighbours outside the volume left out.  Every unordered
// pair {m, n} is evaluated once, at its lower voxel m along one of 13 forward
// directions (9 towards z+1, 4 in-plane); it adds 2 w rho'(d) to the gradient
// at m and subtracts it at n (rho' is odd), and 2 w rho(d) to H.
//
// With q = 2 - p, Q = |u|^q / c and i = 1 / (1 + Q):
//   rho'(d) = d i (p + q i) / (sigma^2 c),   rho(d) = d^2 i / (sigma^2 c),
// so a pair costs lg2, ex2 and rcp (one-instruction approximations, relative
// error ~1e-7) and a few products; 2 lambda / (sigma^2 c) is applied once per
// voxel.  The three special-function instructions per pair and voxel bound
// the kernel; everything else is laid out to keep that unit busy.
//
// Layout: one warp owns a strip of R image rows by 60 columns and marches
// along z through the planes of its z chunk.  It holds in registers the strip
// with one halo row below and above and two halo columns on either side (64
// columns, two adjacent cells per lane, so that every pair evaluation works
// on both cells at once with the packed f32x2 arithmetic) for the current and
// the next plane, and the gradient sums of both planes.  A neighbour in the
// same lane is a register; one in the adjacent lane comes by a warp shuffle,
// and so do the closing shares a pair leaves at a cell of the adjacent lane.
// There is no shared memory and no barrier in the march: the warps of an SM
// run independently.  Pairs that join a strip to the halo rows and columns are
// evaluated by both strips they touch, each keeping the shares that land on
// its own cells.
//
// Order within a step (plane z): row by row, bottom to top.  Row r's gradient
// is complete once rows r-1 and r are done (its forward pairs, the closings of
// in-plane pairs from row r-1 and of z+1 pairs from plane z-1), so it is
// written there, and the registers of row r then receive plane z+2.
//
// The grid's third dimension cuts the z range into chunks (a chunk other than
// the first starts one plane below, evaluating that plane's z+1 pairs only).
//
// In the solver (DOTS) the gradient is not stored: the next iterate
// x_{k+1} = f - step g goes in place of x_prev, and the momentum point of an
// iteration without restart, x_{k+1} + beta (x_{k+1} - x_k), in place of g,
// so the solver needs no separate update pass.  Both x_prev and g are read
// only at the warp's own cells, once, before these stores.
//
// Sums: H per step in FP32 (one plane's rows of one lane) added into a
// compensated pair; the restart-test inner products <g, f - x_prev> and
// <g, g> from error-free differences and products (TwoSum, FMA) into
// compensated accumulators, then FP64 from the per-thread totals on, always in
// the same order: deterministic, and as exact as an FP64 reduction of the
// same FP32 vectors.
#pragma once
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "f32x2.cuh"
#include "profile.cuh"
#include "sfu.cuh"

namespace {

#ifndef TC_PRIOR_R
#define TC_PRIOR_R 4
#endif
#ifndef TC_PRIOR_WPB
#define TC_PRIOR_WPB 4
#endif
#ifndef TC_PRIOR_MINB
#define TC_PRIOR_MINB 4
#endif
constexpr int TX = 60;                      // interior columns of a strip
constexpr int R = TC_PRIOR_R;               // interior rows of a strip
constexpr int RR = R + 2;                   // register rows: halo, R interior rows, halo
constexpr int WPB = TC_PRIOR_WPB;           // strips (one warp each) per CTA, stacked along y
constexpr int THREADS = 32 * WPB;
constexpr int TY = R * WPB;                 // rows of a CTA
constexpr int MIN_BLOCKS = TC_PRIOR_MINB;   // CTAs per SM the register budget is cut for
#ifndef TC_PRIOR_GRP
#define TC_PRIOR_GRP 13
#endif
constexpr int GRP = TC_PRIOR_GRP;           // pair directions per scheduling block
constexpr int ZCHUNK_MAX = 8;               // z chunks per tile column (the partial-sum slots are sized for it)

struct PriorArgs {
    int N, B;
    int z0, z1;        // slices whose gradient this launch produces
    int zc;            // planes per z chunk (blockIdx.z)
    // constants as packed pairs (both halves equal) for the f32x2 arithmetic
    unsigned long long ql2;      // multiplier of log2|d|: q, or the least normal float when q = 0
    unsigned long long lk2;      // -q log2(sigma) - log2(c): exponent offset of Q = |d|^q / (sigma^q c)
    unsigned long long one2;     // 1
    unsigned long long wq2[3];   // w q per weight class (distance 1, sqrt 2, sqrt 3)
    unsigned long long wp2[3];   // w p per weight class
    unsigned long long wh2[3];   // w per weight class (the H terms)
    unsigned long long gscale2;  // 2 lambda / (sigma^2 c)
    unsigned long long nstep2;   // DOTS: minus the solver's step (g receives f - step grad)
    const double *scal;          // DOTS: the solver's scalars (momentum t_k at SC_T)
};

// Global accesses under a predicate, without a branch (zeros when off).
__device__ __forceinline__ float2 ldg2_if(const float *p, bool c) {
    float2 v;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\t"
        "@q ld.global.v2.f32 {%0, %1}, [%2];\n\t}"
        : "=f"(v.x), "=f"(v.y) : "l"(p), "r"((int)c));
    return v;
}
__device__ __forceinline__ float ldg1_if(const float *p, bool c) {
    float v;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\tmov.b32 %0, 0;\n\t@q ld.global.f32 %0, [%1];\n\t}"
        : "=f"(v) : "l"(p), "r"((int)c));
    return v;
}
__device__ __forceinline__ void stg2_if(float *p, float2 v, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.global.v2.f32 [%0], {%1, %2};\n\t}"
                 ::"l"(p), "f"(v.x), "f"(v.y), "r"((int)c) : "memory");
}
__device__ __forceinline__ void stg1_if(float *p, float v, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}"
                 ::"l"(p), "f"(v), "r"((int)c) : "memory");
}
__device__ __forceinline__ void prefetch_l2_if(const float *p, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t@q prefetch.global.L2 [%0];\n\t}" ::"l"(p), "r"((int)c));
}

// the next lane's value (lane + 1) and the previous lane's (lane - 1); lanes
// 31 and 0 get their own, which only halo cells consume
__device__ __forceinline__ float from_next(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float from_prev(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// Neighbour weights 1/||m - n|| normalised over the 26 (3D) or 8 (2D)
// neighbours, at distance 1, sqrt 2, sqrt 3.
template <int DIMS>
struct Wts;
template <>
struct Wts<3> {  // Z = 6 + 12/sqrt(2) + 8/sqrt(3)
    static constexpr double w[3] = {1.0 / 19.104083527755576, 0.70710678118654752 / 19.104083527755576,
                                    0.57735026918962576 / 19.104083527755576};
};
template <>
struct Wts<2> {  // Z = 4 + 4/sqrt(2)
    static constexpr double w[3] = {1.0 / 6.8284271247461901, 0.70710678118654752 / 6.8284271247461901, 0.0};
};

// the 13 forward directions: k < 9 the z+1 pairs (dx, dy) = (k % 3 - 1, k / 3 - 1);
// k = 9..12 the in-plane ones (1,0), (-1,1), (0,1), (1,1)
__host__ __device__ constexpr int kdx(int k) { return k < 9 ? k % 3 - 1 : (k == 9 ? 1 : (k == 10 ? -1 : (k == 11 ? 0 : 1))); }
__host__ __device__ constexpr int kdy(int k) { return k < 9 ? k / 3 - 1 : (k == 9 ? 0 : 1); }
__host__ __device__ constexpr int kdz(int k) { return k < 9 ? 1 : 0; }
__host__ __device__ constexpr int kwc(int k) { return (kdx(k) != 0) + (kdy(k) != 0) + (kdz(k) != 0) - 1; }
// does register row i evaluate direction k: interior rows all; the bottom halo
// row those reaching row 1 (dy = +1); the top halo row those reaching row R (dy = -1)
__host__ __device__ constexpr bool row_does(int i, int k) {
    return (i >= 1 && i <= R) ? true : (i == 0 ? kdy(k) == 1 : kdy(k) == -1 && kdz(k) == 1);
}


// one pair direction for both cells of a lane: returns w d i (p + q i), the
// pair value up to 1 / (sigma^2 c); hs += w d^2 i
template <bool WANT_H, bool MK>
__device__ __forceinline__ float2 pair_value(float2 d, bool k0, bool k1, float2 &hs, unsigned long long ql2,
                                             unsigned long long lk2, unsigned long long one2,
                                             unsigned long long wq, unsigned long long wp,
                                             unsigned long long wh) {
    const float2 t = fma2kk(make_float2(lg2a(fabsf(d.x)), lg2a(fabsf(d.y))), ql2, lk2);
    const float2 den = add2k(make_float2(ex2a(t.x), ex2a(t.y)), one2);
    const float2 inv = make_float2(rcpa(den.x), rcpa(den.y));
    float2 di = mul2(d, inv);
    if (MK) {
        di.x = k0 ? di.x : 0.f;
        di.y = k1 ? di.y : 0.f;
    }
    if (WANT_H) hs = fma2k(mul2(d, di), wh, hs);
    return mul2(di, fma2kk(inv, wq, wp));
}

// a row's two cells of a plane (zeros where off)
template <bool EVEN>
__device__ __forceinline__ float2 load_cells(const float *src, bool c0, bool c1) {
    if (EVEN) return ldg2_if(src, c0);
    return make_float2(ldg1_if(src, c0), ldg1_if(src + 1, c1));
}

// the gradient inputs of an interior row (offset o) of the plane being
// written; the same lines two planes on into L2
template <bool EVEN, bool DOTS>
__device__ __forceinline__ void load_inputs(const float *g, const float *xprev, long long o, bool c, bool in0,
                                            bool in1, long long NN, bool pf, float2 &gi, float2 &xi) {
    if (EVEN) {
        gi = ldg2_if(g + o, c && in0);
        if (DOTS) xi = ldg2_if(xprev + o, c && in0);
    } else {
        gi = make_float2(ldg1_if(g + o, c && in0), ldg1_if(g + o + 1, c && in1));
        if (DOTS) xi = make_float2(ldg1_if(xprev + o, c && in0), ldg1_if(xprev + o + 1, c && in1));
    }
    prefetch_l2_if(g + o + 2 * NN, c && in0 && pf);
    if (DOTS) prefetch_l2_if(xprev + o + 2 * NN, c && in0 && pf);
}

// What a warp's march holds fixed: pointers, sizes, its cells' masks and the
// packed constants of the pair evaluation.
struct MarchCtx {
    const float *f;
    float *g;
    float *xprev;
    long long NN, off0;   // plane size; offset of register row 0, cell 0
    int N, B, za, zb, zl;
    bool ilane, in0, in1;
    bool go;                 // true (a runtime value: the blocks of pairs stay separate)
    unsigned xm0, xm1, rm;   // border strips: (cell, neighbour at dx) inside, bit dx + 1; rows inside, bit i
    unsigned long long ql2, lk2, one2, wq[3], wp[3], wh[3], gscale2, nstep2;
    unsigned long long beta2;   // DOTS: the momentum coefficient without restart
};

// One step of the march: plane z in Pc, plane z + 1 in Pn (3D), their
// gradient sums in Ac / An (Ac already holding the z+1 closings from plane
// z - 1).  FAST: plane z is produced by this chunk and (3D) has a plane above,
// so no pair needs a branch.  On return Pc, Pn, Ac hold the next step's.
template <bool WANT_H, bool DOTS, bool GRAD, int DIMS, bool EVEN, bool MK, bool FAST>
__device__ __forceinline__ void prior_step(const MarchCtx &c, int z, float2 (&Pc)[RR], float2 (&Pn)[RR],
                                           float2 (&Ac)[RR], float2 (&An)[RR], float2 (&Gi)[RR],
                                           float2 (&Xi)[RR], Acc2 &ah, Acc2 &ad1, Acc2 &ad2) {
    const bool own = FAST || z >= c.za;                    // else only this plane's z+1 pairs
    const bool up = DIMS == 3 && (FAST || z + 1 < c.B);    // the z+1 pairs exist
    const long long NN = c.NN, N = c.N;
    const long long zo = (long long)z * NN + c.off0;
#define ROW_IN(i) (!MK || ((c.rm >> (i)) & 1u))
    float2 Pq[RR];   // the plane after: z + 2 (3D), z + 1 (2D)
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        Pq[i] = make_float2(0.f, 0.f);
        if (DIMS == 2) {
            const bool cl = z + 1 < c.zl && ROW_IN(i);
            Pq[i] = load_cells<EVEN>(c.f + zo + NN + i * N, cl && c.in0, cl && c.in1);
        }
        if (GRAD) An[i] = make_float2(0.f, 0.f);
    }
    if (GRAD && own) {
        load_inputs<EVEN, DOTS>(c.g, c.xprev, zo + N, c.ilane && ROW_IN(1), c.in0, c.in1, NN, z + 2 < c.zb, Gi[1], Xi[1]);
        if (R >= 2)
            load_inputs<EVEN, DOTS>(c.g, c.xprev, zo + 2 * N, c.ilane && ROW_IN(2), c.in0, c.in1, NN, z + 2 < c.zb,
                                    Gi[2], Xi[2]);
    }
    // closing shares for the next lane's cell 0 (toR) and the previous lane's
    // cell 1 (toL), in this plane (c) and the next (n); the next lane's cell 0
    // (rs) and the previous lane's cell 1 (ls) of a row
    float toRc[RR], toLc[RR], toRn[RR], toLn[RR], rsC[RR], lsC[RR], rsN[RR], lsN[RR];
#pragma unroll
    for (int i = 0; i < RR; ++i) toRc[i] = toLc[i] = toRn[i] = toLn[i] = rsC[i] = lsC[i] = rsN[i] = lsN[i] = 0.f;
    float2 hstep = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const bool intr = i >= 1 && i <= R;
        if (GRAD && intr && i + 2 <= R && own)
            load_inputs<EVEN, DOTS>(c.g, c.xprev, zo + (i + 2) * N, c.ilane && ROW_IN(i + 2), c.in0, c.in1, NN,
                                    z + 2 < c.zb, Gi[i + 2], Xi[i + 2]);
        // shifted copies of the rows this row is the first to need
        if (i + 1 < RR) {
            if (own) {
                rsC[i + 1] = from_next(Pc[i + 1].x);
                lsC[i + 1] = from_prev(Pc[i + 1].y);
            }
            if (up) {
                if (i == 0) {
                    rsN[0] = from_next(Pn[0].x);
                    lsN[0] = from_prev(Pn[0].y);
                }
                rsN[i + 1] = from_next(Pn[i + 1].x);
                lsN[i + 1] = from_prev(Pn[i + 1].y);
            }
        }
        const float2 fm = Pc[i];
        float2 fw = make_float2(0.f, 0.f), hs = make_float2(0.f, 0.f);
        // the row's pairs: the z+1 ones (k < 9), then the in-plane ones, in
        // blocks of GRP directions, each behind a branch the compiler cannot
        // remove, which bounds how many pair evaluations it interleaves (and so
        // the registers they hold)
#pragma unroll
        for (int k0g = 0; k0g < 13; k0g += GRP) {
            if (GRP < 13 && !c.go) continue;
#pragma unroll
            for (int k = k0g; k < (k0g + GRP < 13 ? k0g + GRP : 13); ++k) {
                const int dx = kdx(k), dy = kdy(k), dz = kdz(k), j = i + dy;
                if (!row_does(i, k) || (DIMS == 2 && dz == 1)) continue;
                if (dz ? !up : !own) continue;
                const float2 fn = dz ? Pn[j] : Pc[j];
                float2 d;
                if (dx == 0) d = sub2(fm, fn);
                else if (dx > 0) d = make_float2(fm.x - fn.y, fm.y - (dz ? rsN[j] : rsC[j]));
                else d = make_float2(fm.x - (dz ? lsN[j] : lsC[j]), fm.y - fn.x);
                bool k0 = true, k1 = true;
                if (MK) {
                    const bool rv = ((c.rm >> i) & 1u) && ((c.rm >> j) & 1u);
                    k0 = rv && ((c.xm0 >> (dx + 1)) & 1u);
                    k1 = rv && ((c.xm1 >> (dx + 1)) & 1u);
                }
                const int wc = kwc(k);
                const float2 e =
                    pair_value<WANT_H, MK>(d, k0, k1, hs, c.ql2, c.lk2, c.one2, c.wq[wc], c.wp[wc], c.wh[wc]);
                if (intr) fw = add2(fw, e);
                if (GRAD && j >= 1 && j <= R) {   // the closing share at row j of plane z + dz
                    if (dx == 0) {
                        if (dz) An[j] = sub2(An[j], e);
                        else Ac[j] = sub2(Ac[j], e);
                    } else if (dx > 0) {
                        if (dz) {
                            An[j].y -= e.x;
                            toRn[j] += e.y;
                        } else {
                            Ac[j].y -= e.x;
                            toRc[j] += e.y;
                        }
                    } else {
                        if (dz) {
                            An[j].x -= e.y;
                            toLn[j] += e.x;
                        } else {
                            Ac[j].x -= e.y;
                            toLc[j] += e.x;
                        }
                    }
                }
            }
        }
        if (intr && own) {
            const long long o = zo + i * N;
            const bool m0 = c.ilane && ROW_IN(i) && c.in0, m1 = c.ilane && ROW_IN(i) && c.in1;
            if (GRAD) {
                // row i of plane z is complete once the adjacent lanes' shares are in
                float2 acc = add2(Ac[i], fw);
                acc.x -= from_prev(toRc[i]);
                acc.y -= from_next(toLc[i]);
                const float2 gn = fma2k(acc, c.gscale2, Gi[i]);
                const float2 out = DOTS ? fma2k(gn, c.nstep2, fm) : gn;
                // DOTS: x_{k+1} over x_prev, z_{k+1} = x_{k+1} + beta (x_{k+1} - x_k) over g
                float *const dst = DOTS ? c.xprev : c.g;
                if (EVEN) {
                    stg2_if(dst + o, out, m0);
                } else {
                    stg1_if(dst + o, out.x, m0);
                    stg1_if(dst + o + 1, out.y, m1);
                }
                if (DOTS) {
                    const float2 zn = fma2k(sub2(out, Xi[i]), c.beta2, out);
                    if (EVEN) {
                        stg2_if(c.g + o, zn, m0);
                    } else {
                        stg1_if(c.g + o, zn.x, m0);
                        stg1_if(c.g + o + 1, zn.y, m1);
                    }
                }
                if (DOTS) {
                    // <g, f - x_prev>: f - x_prev exactly as dd + de, then exact products (TwoSum)
                    float2 de;
                    const float2 dd = two_sum2(fm, make_float2(-Xi[i].x, -Xi[i].y), de);
                    const float2 gm = make_float2(m0 ? gn.x : 0.f, m1 ? gn.y : 0.f);
                    const float2 p1 = mul2(gm, dd);
                    ad1.add(p1, fma2(gm, de, fma2(gm, dd, make_float2(-p1.x, -p1.y))));
                    // <g, g>: non-negative terms, so the running sum dominates each new
                    // term after the first and Fast2Sum is exact
                    const float2 p2v = mul2(gm, gm);
                    const float2 e2 = fma2(gm, gm, make_float2(-p2v.x, -p2v.y));
                    const float2 s2 = add2(ad2.s, p2v);
                    ad2.c = add2(ad2.c, add2(add2(sub2(ad2.s, s2), p2v), e2));
                    ad2.s = s2;
                }
            }
            if (WANT_H) hstep = add2(hstep, make_float2(m0 ? hs.x : 0.f, m1 ? hs.y : 0.f));
        }
        // row i - 1 of plane z + 1 has all its z+1 closings from this plane
        if (GRAD && DIMS == 3 && i - 1 >= 1 && i - 1 <= R && up) {
            An[i - 1].x -= from_prev(toRn[i - 1]);
            An[i - 1].y -= from_next(toLn[i - 1]);
        }
        // row i of plane z is no longer needed: plane z + 2 takes its place
        if (DIMS == 3) {
            const bool cl = z + 2 < c.zl && ROW_IN(i);
            Pq[i] = load_cells<EVEN>(c.f + zo + 2 * NN + i * N, cl && c.in0, cl && c.in1);
        }
    }
    if (WANT_H && own) ah.add(hstep, make_float2(0.f, 0.f));
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        if (DIMS == 3) {
            Pc[i] = Pn[i];
            Pn[i] = Pq[i];
            Ac[i] = An[i];
        } else {
            Pc[i] = Pq[i];
            Ac[i] = make_float2(0.f, 0.f);
        }
    }
#undef ROW_IN
}

// The march of one warp over its z chunk.  MK: a border strip (a mask per
// pair); else every cell of the strip, halo included, lies in the volume.
template <bool WANT_H, bool DOTS, bool GRAD, int DIMS, bool EVEN, bool MK>
__device__ __forceinline__ void prior_march(const float *__restrict__ f, float *__restrict__ g,
                                            float *__restrict__ xprev, const PriorArgs &a,
                                            unsigned long long beta2, int gx, int y0, int za, int zb,
                                            Acc2 &ah, Acc2 &ad1, Acc2 &ad2) {
    MarchCtx c;
    c.f = f;
    c.g = g;
    c.xprev = xprev;
    c.N = a.N;
    c.B = a.B;
    c.NN = (long long)a.N * a.N;
    c.za = za;
    c.zb = zb;
    c.zl = DIMS == 3 ? min(a.B, zb + 1) : zb;   // planes below zl are read
    c.off0 = (long long)(y0 - 1) * a.N + gx;
    const int N = a.N;
    const int lane = threadIdx.x & 31;
    c.ilane = lane >= 1 && lane <= 30;   // both cells interior columns
    const bool cx0 = gx >= 0 && gx < N, cx1 = gx + 1 >= 0 && gx + 1 < N;
    c.in0 = !MK || cx0;
    c.in1 = !MK || cx1;
    c.go = a.B > 0;
    c.xm0 = c.xm1 = c.rm = 0;
    if (MK) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (cx0 && gx + dx >= 0 && gx + dx < N) c.xm0 |= 1u << (dx + 1);
            if (cx1 && gx + 1 + dx >= 0 && gx + 1 + dx < N) c.xm1 |= 1u << (dx + 1);
        }
#pragma unroll
        for (int i = 0; i < RR; ++i)
            if (y0 - 1 + i >= 0 && y0 - 1 + i < N) c.rm |= 1u << i;
    }
    c.ql2 = a.ql2;
    c.lk2 = a.lk2;
    c.one2 = a.one2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.wq[k] = a.wq2[k];
        c.wp[k] = a.wp2[k];
        c.wh[k] = a.wh2[k];
    }
    c.gscale2 = a.gscale2;
    c.nstep2 = a.nstep2;
    c.beta2 = beta2;

    const int zs = (DIMS == 3 && za > 0) ? za - 1 : za;
    float2 Pc[RR], Pn[RR], Ac[RR], An[RR], Gi[RR], Xi[RR];
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const bool ri = !MK || ((c.rm >> i) & 1u);
        const float *src = f + (long long)zs * c.NN + c.off0 + (long long)i * N;
        Pc[i] = load_cells<EVEN>(src, zs < c.zl && ri && c.in0, zs < c.zl && ri && c.in1);
        Pn[i] = make_float2(0.f, 0.f);
        if (DIMS == 3)
            Pn[i] = load_cells<EVEN>(src + c.NN, zs + 1 < c.zl && ri && c.in0, zs + 1 < c.zl && ri && c.in1);
        Ac[i] = An[i] = Gi[i] = Xi[i] = make_float2(0.f, 0.f);
    }
    // the steps that produce their plane and (3D) have a plane above run branch-free
    const int zfast_end = DIMS == 3 ? min(zb, a.B - 1) : zb;
    int z = zs;
    if (z < za) {
        prior_step<WANT_H, DOTS, GRAD, DIMS, EVEN, MK, false>(c, z, Pc, Pn, Ac, An, Gi, Xi, ah, ad1, ad2);
        ++z;
    }
#pragma unroll 1
    for (; z < zfast_end; ++z)
        prior_step<WANT_H, DOTS, GRAD, DIMS, EVEN, MK, true>(c, z, Pc, Pn, Ac, An, Gi, Xi, ah, ad1, ad2);
    if (z < zb) prior_step<WANT_H, DOTS, GRAD, DIMS, EVEN, MK, false>(c, z, Pc, Pn, Ac, An, Gi, Xi, ah, ad1, ad2);
}

template <bool WANT_H, bool DOTS, bool GRAD, int DIMS, bool EVEN>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
    k_prior(const float *__restrict__ f, float *__restrict__ g, double *__restrict__ part_h,
            const PriorArgs a, float *__restrict__ xprev, double *__restrict__ pd1,
            double *__restrict__ pd2) {
    __shared__ double red[WPB];
    const int N = a.N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY + wid * R;   // first interior column and row
    const int gx = x0 - 2 + 2 * lane;                                   // the lane's cells gx, gx + 1
    const int za = a.z0 + blockIdx.z * a.zc;
    const int zb = min(a.z1, za + a.zc);
    Acc2 ah, ad1, ad2;
    ah.zero();
    ad1.zero();
    ad2.zero();
    unsigned long long beta2 = 0;
    if (DOTS) {
        // beta of an iteration without restart, as the solver's scalar step
        // forms it from t_k (the restart test that follows this pass may
        // still set beta = 0; the solver then copies x_{k+1} over z_{k+1})
        const double t = a.scal[SC_T];
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const float bf = (float)((t - 1.0) / tn);
        beta2 = f2_pack(make_float2(bf, bf));
    }
    if (y0 < N && za < zb) {
        const bool full = EVEN && x0 >= 2 && x0 + TX + 2 <= N && y0 >= 1 && y0 + R + 1 <= N;
        if (full)
            prior_march<WANT_H, DOTS, GRAD, DIMS, EVEN, false>(f, g, xprev, a, beta2, gx, y0, za, zb, ah, ad1,
                                                              ad2);
        else
            prior_march<WANT_H, DOTS, GRAD, DIMS, EVEN, true>(f, g, xprev, a, beta2, gx, y0, za, zb, ah, ad1, ad2);
    }
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (WANT_H) {
        const double tot = block_sum_f64(ah.total(), red);
        if (threadIdx.x == 0) part_h[bid] = tot;
    }
    if (DOTS) {
        const double t1 = block_sum_f64(ad1.total(), red);
        const double t2 = block_sum_f64(ad2.total(), red);
        if (threadIdx.x == 0) {
            pd1[bid] = t1;
            pd2[bid] = t2;
        }
    }
}

}  // namespace
