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
// voxel.
//
// Layout of a CTA: a tile of 60 x 12 voxel columns marching along z, held
// with its halo in a 64 x 14 ring of shared memory (two halo columns on each
// side, so that every lane's pair of cells starts on an 8-byte boundary).
// One warp per ring row, two cells per lane: every pair evaluation works on
// both cells at once with the packed f32x2 arithmetic.  Each plane is kept
// twice, plain and shifted by one cell, so the neighbours at dx = -1, 0, +1
// are each one aligned 8-byte shared load.
//
// One z step, two barriers:
//   A  store plane z+1 (3D) or z (2D); read the z+1 pair values of the step
//      before (the pairs that end at this plane's voxels)
//   B  evaluate this plane's 13 pair directions; store the pair values
//   C  read the in-plane pair values that end at this plane's voxels; write
//      the gradient (or the solver's next iterate) and the sums
// The z+1 pair values need a single buffer: phase A of step z reads the
// values of step z-1 before the barrier that precedes phase B's writes.
//
// The grid's third dimension cuts the z range into chunks (a chunk other than
// the first starts one plane below, evaluating that plane's pairs only).
//
// Sums: H (positive terms) in FP32 groups of 16 steps added into a
// compensated pair; the restart-test inner products <g, f - x_prev> and
// <g, g> from error-free differences and products (TwoSum, FMA) into
// compensated accumulators, then FP64 from the per-thread totals on, always in
// the same order: deterministic, and as exact as an FP64 reduction of the
// same FP32 vectors.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "f32x2.cuh"
#include "profile.cuh"

namespace {

#ifndef TC_PRIOR_TY
#define TC_PRIOR_TY 12
#endif
#ifndef TC_PRIOR_MINB
#define TC_PRIOR_MINB 2
#endif
constexpr int TX = 60;              // interior columns of a tile
constexpr int TY = TC_PRIOR_TY;     // interior rows of a tile
constexpr int RX = 64;              // ring columns
constexpr int RY = TY + 2;          // ring rows, one warp each
constexpr int THREADS = 32 * RY;    // 448
constexpr int PLANE = RY * RX;      // floats per ring array
constexpr int PAD = 4;              // floats before and after the arrays (reads one slot past either end)
constexpr int MIN_BLOCKS = TC_PRIOR_MINB;  // CTAs per SM the register budget is cut for
constexpr int ZCHUNK_MAX = 8;       // z chunks per tile column (the partial-sum slots are sized for it)

// shared floats: F[2], S[2] (plain and shifted planes), Eu[9] (3D), Ep[3]
__host__ __device__ constexpr int smem_floats(int dims) { return 2 * PAD + (4 + (dims == 3 ? 9 : 0) + 3) * PLANE; }

struct PriorArgs {
    int N, B;
    int z0, z1;        // slices whose gradient this launch produces
    int zc;            // planes per z chunk (blockIdx.z)
    // constants as packed pairs (both halves equal) for the f32x2 arithmetic
    unsigned long long p2, q2;   // p, q = 2 - p
    unsigned long long lk2;      // -q log2(sigma) - log2(c): exponent offset of Q = |d|^q / (sigma^q c)
    unsigned long long one2;     // 1
    unsigned long long gscale2;  // 2 lambda / (sigma^2 c)
    unsigned long long nstep2;   // DOTS: minus the solver's step (g receives f - step grad)
};

__device__ __forceinline__ float lg2a(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2a(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcpa(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// direction u of the z+1 pairs: dx = u % 3 - 1, dy = u / 3 - 1
__host__ __device__ constexpr int udx(int u) { return u % 3 - 1; }
__host__ __device__ constexpr int udy(int u) { return u / 3 - 1; }
// in-plane directions q: (1,0), (-1,1), (0,1), (1,1)
__host__ __device__ constexpr int pdx(int q) { return q == 0 ? 1 : (q == 1 ? -1 : (q == 2 ? 0 : 1)); }
__host__ __device__ constexpr int pdy(int q) { return q == 0 ? 0 : 1; }

// 8-byte shared load of ring cells (c, c+1) at float index i (i even)
__device__ __forceinline__ float2 lds2(const float *s, int i) { return *reinterpret_cast<const float2 *>(s + i); }

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

// Neighbour weights 1/||m - n|| normalised over the 26 (3D) or 8 (2D)
// neighbours, at distance 1, sqrt 2, sqrt 3.
template <int DIMS>
struct Wts;
template <>
struct Wts<3> {  // Z = 6 + 12/sqrt(2) + 8/sqrt(3)
    static constexpr float w1 = (float)(1.0 / 19.104083527755576), w2 = (float)(0.70710678118654752 / 19.104083527755576),
                           w3 = (float)(0.57735026918962576 / 19.104083527755576);
};
template <>
struct Wts<2> {  // Z = 4 + 4/sqrt(2)
    static constexpr float w1 = (float)(1.0 / 6.8284271247461901), w2 = (float)(0.70710678118654752 / 6.8284271247461901),
                           w3 = 0.f;
};

// role of a ring row: interior rows, the bottom halo row (only pairs that reach
// row 1) and the top halo row (only the z+1 pairs that reach row TY)
constexpr int ROLE_IN = 0, ROLE_BOT = 1, ROLE_TOP = 2;
__host__ __device__ constexpr unsigned up_dirs(int role) { return role == ROLE_IN ? 0x1ffu : (role == ROLE_BOT ? 0x1c0u : 0x007u); }
__host__ __device__ constexpr unsigned pl_dirs(int role) { return role == ROLE_IN ? 0xfu : (role == ROLE_BOT ? 0xeu : 0x0u); }

template <bool WANT_H, bool DOTS, bool GRAD, int DIMS, bool EVEN>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS)
    k_prior(const float *__restrict__ f, float *__restrict__ g, double *__restrict__ part_h,
            const PriorArgs a, const float *__restrict__ xprev, double *__restrict__ pd1,
            double *__restrict__ pd2) {
    extern __shared__ float psm[];
    float *F = psm + PAD;                                    // [2][PLANE] plain planes
    float *S = F + 2 * PLANE;                                // [2][PLANE] shifted: (f[c+1], f[c+2]) at c
    float *Eu = S + 2 * PLANE;                               // [9][PLANE] z+1 pair values (3D)
    float *Ep = Eu + (DIMS == 3 ? 9 : 0) * PLANE;            // [3][PLANE] in-plane (-1,1), (0,1), (1,1)
    __shared__ double red[THREADS / 32];
    const int N = a.N, B = a.B;
    const size_t NN = (size_t)N * N;
    const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = x0 - 2 + 2 * lane, gy = y0 - 1 + wr;
    const bool rowin = gy >= 0 && gy < N;
    const bool in0 = rowin && gx >= 0 && gx < N, in1 = rowin && gx + 1 >= 0 && gx + 1 < N;
    const bool iwarp = wr >= 1 && wr <= TY;                  // interior ring row
    const bool ilane = lane >= 1 && lane <= 30;              // both cells interior columns
    const bool own0 = iwarp && ilane && in0, own1 = iwarp && ilane && in1;
    // the whole ring inside the volume (even N): no pair needs the border test
    const bool full = EVEN && x0 >= 2 && x0 + RX - 2 <= N && y0 >= 1 && y0 - 1 + RY <= N;
    // border tiles: bit k of km0 / km1 = pair direction k of cell 0 / 1 valid
    // (k < 9: z+1 pair u = k; k = 9 + q: in-plane q)
    unsigned km0 = 0, km1 = 0;
    if (!full) {
        auto inv_ = [&](int x, int y) { return x >= 0 && x < N && y >= 0 && y < N; };
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            const int dx = k < 9 ? udx(k) : pdx(k - 9), dy = k < 9 ? udy(k) : pdy(k - 9);
            if (in0 && inv_(gx + dx, gy + dy)) km0 |= 1u << k;
            if (in1 && inv_(gx + 1 + dx, gy + dy)) km1 |= 1u << k;
        }
    }
    // z range of this block
    const int za = a.z0 + blockIdx.z * a.zc;
    const int zb = min(a.z1, za + a.zc);
    const int zs = (DIMS == 3 && za > 0) ? za - 1 : za;
    const long long off = (long long)gy * N + gx;
    const int rs = wr * RX + 2 * lane;                       // own slot in a ring array
    // constants of the pair evaluation, held once
    const unsigned long long q2 = a.q2, lk2 = a.lk2, p2 = a.p2, one2 = a.one2;
    const unsigned long long w1 = pack_splat(Wts<DIMS>::w1), w2 = pack_splat(Wts<DIMS>::w2),
                             w3 = pack_splat(Wts<DIMS>::w3);
    auto wup = [&](int u) { return (udx(u) == 0 && udy(u) == 0) ? w1 : ((udx(u) == 0 || udy(u) == 0) ? w2 : w3); };

    auto load_pair = [&](int z) -> float2 {
        const float *src = f + (size_t)z * NN + off;
        const bool c = z < B;
        if (EVEN) return ldg2_if(src, c && in0);
        return make_float2(ldg1_if(src, c && in0), ldg1_if(src + 1, c && in1));
    };
    // plane values into ring array pl: plain and shifted by one cell
    auto store_plane = [&](int pl, float2 v) {
        const float nx = __shfl_down_sync(0xffffffffu, v.x, 1);
        *reinterpret_cast<float2 *>(F + pl * PLANE + rs) = v;
        *reinterpret_cast<float2 *>(S + pl * PLANE + rs) = make_float2(v.y, nx);
    };
    // one pair direction for both cells: d = fm - fn, e = d i (p + q i); dh = d^2 i
    auto pair_eval = [&](auto mk, float2 fm, float2 fn, bool k0, bool k1, float2 &dh) -> float2 {
        const float2 d = sub2(fm, fn);
        const float2 t = fma2kk(make_float2(lg2a(fabsf(d.x)), lg2a(fabsf(d.y))), q2, lk2);
        const float2 den = add2k(make_float2(ex2a(t.x), ex2a(t.y)), one2);
        const float2 inv = make_float2(rcpa(den.x), rcpa(den.y));
        float2 di = mul2(d, inv);
        if (decltype(mk)::value) {
            di.x = k0 ? di.x : 0.f;
            di.y = k1 ? di.y : 0.f;
        }
        if (WANT_H) dh = mul2(d, di);
        return mul2(di, fma2kk(inv, q2, p2));
    };
    if (DIMS == 3) {
        for (int i = threadIdx.x; i < 9 * PLANE; i += THREADS) Eu[i] = 0.f;
    }
    float2 fcur = load_pair(zs), fnx;
    if (DIMS == 3) {
        store_plane(0, fcur);
        fnx = load_pair(zs + 1);
    } else {
        fnx = fcur;
    }
    __syncthreads();   // zeroed z+1 pair values and the first plane before any step reads them
    Acc2 ah, ad1, ad2;
    ah.zero();
    ad1.zero();
    ad2.zero();
    float2 h16 = make_float2(0.f, 0.f);

    // phase B for one role and border mode: this plane's pairs of the lane's
    // two cells, their forward shares in gs (and H terms in hs), the values
    // stored for the voxels that close them
    auto pairs = [&](auto role, auto mk, auto cur_c, bool up, float2 &gs, float2 &hs, float2 &e10) {
        constexpr int ROLE = decltype(role)::value, cur = decltype(cur_c)::value, nxt = cur ^ 1;
        if (DIMS == 3 && up) {
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                if (!((up_dirs(ROLE) >> u) & 1u)) continue;
                const int dx = udx(u), dy = udy(u);
                const int o = nxt * PLANE + (wr + dy) * RX + 2 * lane;
                const float2 fn = dx == 0 ? lds2(F, o) : lds2(S, o + (dx > 0 ? 0 : -2));
                float2 dh;
                const float2 e = pair_eval(mk, fcur, fn, (km0 >> u) & 1, (km1 >> u) & 1, dh);
                gs = fma2k(e, wup(u), gs);
                if (WANT_H) hs = fma2k(dh, wup(u), hs);
                if (GRAD) *reinterpret_cast<float2 *>(Eu + u * PLANE + rs) = e;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!((pl_dirs(ROLE) >> q) & 1u)) continue;
            const int dx = pdx(q), dy = pdy(q);
            const int o = cur * PLANE + (wr + dy) * RX + 2 * lane;
            const float2 fn = dx == 0 ? lds2(F, o) : lds2(S, o + (dx > 0 ? 0 : -2));
            float2 dh;
            const float2 e = pair_eval(mk, fcur, fn, (km0 >> (9 + q)) & 1, (km1 >> (9 + q)) & 1, dh);
            const unsigned long long wq = (dx != 0 && dy != 0) ? w2 : w1;
            gs = fma2k(e, wq, gs);
            if (WANT_H) hs = fma2k(dh, wq, hs);
            if (q == 0) e10 = e;
            else if (GRAD) *reinterpret_cast<float2 *>(Ep + (q - 1) * PLANE + rs) = e;
        }
    };

    auto step = [&](auto par, int z) {
        constexpr int cur = decltype(par)::value, nxt = cur ^ 1;
        const bool own = z >= za;
        const bool up = DIMS == 3 && z + 1 < B;
        const float2 fpf = load_pair(DIMS == 3 ? z + 2 : z + 1);   // the plane the next step stores
        const size_t i = (size_t)z * NN + off;
        const bool mine0 = own && own0, mine1 = own && own1;       // this lane's cells get a gradient
        float2 gold = make_float2(0.f, 0.f), xold = make_float2(0.f, 0.f);
        if (GRAD && own && iwarp) {
            if (EVEN) {
                gold = ldg2_if(g + i, mine0);
                if (DOTS) xold = ldg2_if(xprev + i, mine0);
            } else {
                gold = make_float2(ldg1_if(g + i, mine0), ldg1_if(g + i + 1, mine1));
                if (DOTS) xold = make_float2(ldg1_if(xprev + i, mine0), ldg1_if(xprev + i + 1, mine1));
            }
            // the same lines two planes on, into L2
            prefetch_l2_if(g + i + 2 * NN, mine0 && z + 2 < zb);
            if (DOTS) prefetch_l2_if(xprev + i + 2 * NN, mine0 && z + 2 < zb);
        }
        // ---- A: stage the next plane; close the z+1 pairs of the step before
        if (DIMS == 3) {
            if (up) store_plane(nxt, fnx);
        } else {
            store_plane(cur, fnx);
            fcur = fnx;
        }
        float2 gc = make_float2(0.f, 0.f);   // closing shares (subtracted)
        if (DIMS == 3 && GRAD && own && iwarp) {
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                const int dx = udx(u), dy = udy(u);
                const float *e = Eu + u * PLANE + (wr - dy) * RX + 2 * lane;
                float2 v;
                if (dx == 0) v = lds2(e, 0);
                else if (dx > 0) v = make_float2(e[-1], e[0]);
                else v = make_float2(e[1], e[2]);
                gc = fma2k(v, wup(u), gc);
            }
        }
        __syncthreads();
        // ---- B: this plane's pairs (one branch per warp role and border mode)
        float2 gs = make_float2(0.f, 0.f), hs = make_float2(0.f, 0.f), e10 = make_float2(0.f, 0.f);
        using CUR = std::integral_constant<int, cur>;
        if (iwarp) {
            if (full) pairs(std::integral_constant<int, ROLE_IN>{}, std::false_type{}, CUR{}, up, gs, hs, e10);
            else pairs(std::integral_constant<int, ROLE_IN>{}, std::true_type{}, CUR{}, up, gs, hs, e10);
        } else if (GRAD) {
            if (wr == 0) {
                if (full) pairs(std::integral_constant<int, ROLE_BOT>{}, std::false_type{}, CUR{}, up, gs, hs, e10);
                else pairs(std::integral_constant<int, ROLE_BOT>{}, std::true_type{}, CUR{}, up, gs, hs, e10);
            } else {
                if (full) pairs(std::integral_constant<int, ROLE_TOP>{}, std::false_type{}, CUR{}, up, gs, hs, e10);
                else pairs(std::integral_constant<int, ROLE_TOP>{}, std::true_type{}, CUR{}, up, gs, hs, e10);
            }
        }
        __syncthreads();
        // ---- C: close the in-plane pairs; gradient and sums
        if (own && iwarp) {
            if (GRAD) {
                const float e10l = __shfl_up_sync(0xffffffffu, e10.y, 1);   // cell 2l - 1, lane l - 1
                gc = fma2k(make_float2(e10l, e10.x), w1, gc);
                const float *r1 = Ep + (wr - 1) * RX + 2 * lane;
                gc = fma2k(make_float2(r1[1], r1[2]), w2, gc);                       // (-1,1) from (c+1, y-1)
                gc = fma2k(lds2(r1 + PLANE, 0), w1, gc);                             // (0,1) from (c, y-1)
                gc = fma2k(make_float2(r1[2 * PLANE - 1], r1[2 * PLANE]), w2, gc);   // (1,1) from (c-1, y-1)
                const float2 gn = fma2k(sub2(gs, gc), a.gscale2, gold);
                const float2 out = DOTS ? fma2k(gn, a.nstep2, fcur) : gn;
                if (EVEN) {
                    stg2_if(g + i, out, mine0);
                } else {
                    stg1_if(g + i, out.x, mine0);
                    stg1_if(g + i + 1, out.y, mine1);
                }
                if (DOTS) {
                    // <g, f - x_prev>: f - x_prev exactly as dd + de, then exact products (TwoSum)
                    float2 de;
                    const float2 dd = two_sum2(fcur, make_float2(-xold.x, -xold.y), de);
                    const float2 gm = make_float2(mine0 ? gn.x : 0.f, mine1 ? gn.y : 0.f);
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
            if (WANT_H) h16 = add2(h16, make_float2(mine0 ? hs.x : 0.f, mine1 ? hs.y : 0.f));
        }
        if (WANT_H && (z & 15) == 15) {
            ah.add(h16, make_float2(0.f, 0.f));
            h16 = make_float2(0.f, 0.f);
        }
        if (DIMS == 3) fcur = fnx;
        fnx = fpf;
    };
    int z = zs;
    for (; z + 1 < zb; z += 2) {
        step(std::integral_constant<int, 0>{}, z);
        step(std::integral_constant<int, 1>{}, z + 1);
    }
    if (z < zb) step(std::integral_constant<int, 0>{}, z);
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (WANT_H) {
        ah.add(h16, make_float2(0.f, 0.f));
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

PriorArgs make_prior_args(int n, int nb, const tc_prior *pr, double step = 0.0) {
    PriorArgs a;
    a.N = n;
    a.B = nb;
    a.z0 = 0;
    a.z1 = nb;
    a.zc = nb;
    a.p2 = pack_splat((float)pr->p);
    a.q2 = pack_splat((float)(2.0 - pr->p));
    a.lk2 = pack_splat((float)(-(2.0 - pr->p) * std::log2(pr->sigma) - std::log2(pr->c)));
    a.one2 = pack_splat(1.0f);
    a.gscale2 = pack_splat((float)(2.0 * pr->lambda / (pr->sigma * pr->sigma * pr->c)));
    a.nstep2 = pack_splat((float)-step);
    return a;
}

// lambda H from the block partials of sum w d^2 i over unordered pairs: every
// pair enters H twice (ordered pairs) and rho = d^2 i / (sigma^2 c).
double prior_value_scale(const tc_prior *pr) { return 2.0 * pr->lambda / (pr->sigma * pr->sigma * pr->c); }

dim3 tile_grid(int n) { return dim3((n + TX - 1) / TX, (n + TY - 1) / TY, 1); }

// z chunks for nb slices: about 128 planes each, at most ZCHUNK_MAX and at
// most what max_blocks partial sums allow
int z_chunks(int n, int nb, int max_blocks) {
    const dim3 t = tile_grid(n);
    int c = nb / 128;
    c = c < 1 ? 1 : (c > ZCHUNK_MAX ? ZCHUNK_MAX : c);
    while (c > 1 && (long long)c * t.x * t.y > max_blocks) --c;
    return c;
}

template <bool H, bool DOTS, bool GRAD, int DIMS, bool EVEN>
void launch_one(dim3 grid, cudaStream_t s, bool profiled, const float *x, float *g, double *ph,
                const PriorArgs &a, const float *xp, double *p1, double *p2) {
    const size_t smem = (size_t)smem_floats(DIMS) * sizeof(float);
    if (profiled)
        TC_PROFILED(TCK_PRIOR, s, (k_prior<H, DOTS, GRAD, DIMS, EVEN><<<grid, THREADS, smem, s>>>(x, g, ph, a, xp, p1, p2)));
    else
        k_prior<H, DOTS, GRAD, DIMS, EVEN><<<grid, THREADS, smem, s>>>(x, g, ph, a, xp, p1, p2);
}

// dispatch on (WANT_H, DOTS, DIMS) for the gradient kernels
template <bool EVEN>
void launch_grad(bool h, bool dots, int dims, dim3 grid, cudaStream_t s, bool prof, const float *x, float *g,
                 double *ph, const PriorArgs &a, const float *xp, double *p1, double *p2) {
    if (dims == 3) {
        if (h && dots) launch_one<true, true, true, 3, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else if (h) launch_one<true, false, true, 3, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else if (dots) launch_one<false, true, true, 3, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else launch_one<false, false, true, 3, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
    } else {
        if (h && dots) launch_one<true, true, true, 2, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else if (h) launch_one<true, false, true, 2, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else if (dots) launch_one<false, true, true, 2, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
        else launch_one<false, false, true, 2, EVEN>(grid, s, prof, x, g, ph, a, xp, p1, p2);
    }
}

}  // namespace

int prior_tile_count(int n) {
    const dim3 t = tile_grid(n);
    return (int)(t.x * t.y);
}

// partial-sum slots a plan needs for the prior launches on N x N slices
int prior_block_slots(int n) { return prior_tile_count(n) * ZCHUNK_MAX; }

int launch_prior_grad(tc_plan *p, const float *x, float *g, int nb,
                      const tc_prior *pr, double *h_acc, cudaStream_t s, const float *dot_x,
                      int z0, int z1, double step) {
    PriorArgs a = make_prior_args(p->k.N, nb, pr, step);
    if (z1 < 0) z1 = nb;
    if (z0 < 0 || z0 >= z1 || z1 > nb) return TC_ERR_INVALID_ARG;
    a.z0 = z0;
    a.z1 = z1;
    const int acc = z0 > 0;  // a later slab adds to the sums of the earlier ones
    dim3 grid = tile_grid(a.N);
    grid.z = z_chunks(a.N, z1 - z0, p->slot);
    a.zc = (z1 - z0 + grid.z - 1) / grid.z;
    const int blocks = grid.x * grid.y * grid.z;
    if (blocks > p->slot) return TC_ERR_UNSUPPORTED;
    double *part = p->partials + (size_t)1 * p->slot;
    double *p1 = p->partials + (size_t)2 * p->slot, *p2 = p->partials + (size_t)3 * p->slot;
    launch_grad<true>(h_acc != nullptr, dot_x != nullptr, pr->dims, grid, s, true, x, g, part, a, dot_x,
                      dot_x ? p1 : nullptr, dot_x ? p2 : nullptr);
    TC_LAUNCHED("k_prior");
    if (dot_x) {
        int rc = launch_reduce_finalize(p1, blocks, p->scal + SC_DOT_GZX, acc, 1.0, s);
        if (!rc) rc = launch_reduce_finalize(p2, blocks, p->scal + SC_DOT_GG, acc, 1.0, s);
        if (rc) return rc;
    }
    if (h_acc) return launch_reduce_finalize(part, blocks, h_acc, acc, prior_value_scale(pr), s);
    return TC_OK;
}

int launch_prior_value(tc_plan *p, const float *x, int nb, const tc_prior *pr,
                       double *h_acc, cudaStream_t s) {
    PriorArgs a = make_prior_args(p->k.N, nb, pr);
    dim3 grid = tile_grid(a.N);
    grid.z = z_chunks(a.N, nb, p->slot);
    a.zc = (nb + grid.z - 1) / grid.z;
    const int blocks = grid.x * grid.y * grid.z;
    if (blocks > p->slot) return TC_ERR_UNSUPPORTED;
    double *part = p->partials + (size_t)1 * p->slot;
    if (pr->dims == 3)
        launch_one<true, false, false, 3, true>(grid, s, true, x, nullptr, part, a, nullptr, nullptr, nullptr);
    else
        launch_one<true, false, false, 2, true>(grid, s, true, x, nullptr, part, a, nullptr, nullptr, nullptr);
    TC_LAUNCHED("k_prior");
    return launch_reduce_finalize(part, blocks, h_acc, 0, prior_value_scale(pr), s);
}

// Prior gradient and value with caller-supplied partial-sum storage (the
// no-allocation entry point, prior_noalloc.cu): g += 2 lambda sum w rho',
// *h_out = lambda H.  Same kernel and reduction as launch_prior_grad, any side
// n >= 1; launched without profiler events.
int launch_prior_kernel_into(const float *x, float *g, int n, int nb, const tc_prior *pr,
                             double *partials, int max_partials, double *h_out,
                             cudaStream_t s) {
    PriorArgs a = make_prior_args(n, nb, pr);
    dim3 grid = tile_grid(n);
    grid.z = z_chunks(n, nb, max_partials);
    a.zc = (nb + grid.z - 1) / grid.z;
    const int blocks = grid.x * grid.y * grid.z;
    if (blocks > max_partials) return TC_ERR_INVALID_ARG;
    const bool h = h_out != nullptr, even = n % 2 == 0;
    if (pr->dims == 3) {
        if (even) {
            if (h) launch_one<true, false, true, 3, true>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
            else launch_one<false, false, true, 3, true>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
        } else {
            if (h) launch_one<true, false, true, 3, false>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
            else launch_one<false, false, true, 3, false>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
        }
    } else {
        if (even) {
            if (h) launch_one<true, false, true, 2, true>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
            else launch_one<false, false, true, 2, true>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
        } else {
            if (h) launch_one<true, false, true, 2, false>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
            else launch_one<false, false, true, 2, false>(grid, s, false, x, g, partials, a, nullptr, nullptr, nullptr);
        }
    }
    TC_LAUNCHED("k_prior");
    if (h_out) return launch_reduce_finalize(partials, blocks, h_out, 0, prior_value_scale(pr), s);
    return TC_OK;
}

namespace {

// Opt a kernel into its dynamic shared memory (raise only: the limit is a
// process-wide attribute of the kernel).
template <class F>
int raise_smem(F *fn, int smem) {
    cudaFuncAttributes at;
    TC_CUDA(cudaFuncGetAttributes(&at, fn));
    if (at.maxDynamicSharedSizeBytes < smem)
        TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return TC_OK;
}

template <int DIMS>
int configure_dims() {
    const int sm = smem_floats(DIMS) * (int)sizeof(float);
    int rc;
    if ((rc = raise_smem(k_prior<true, true, true, DIMS, true>, sm)) ||
        (rc = raise_smem(k_prior<true, false, true, DIMS, true>, sm)) ||
        (rc = raise_smem(k_prior<false, true, true, DIMS, true>, sm)) ||
        (rc = raise_smem(k_prior<false, false, true, DIMS, true>, sm)) ||
        (rc = raise_smem(k_prior<true, false, false, DIMS, true>, sm)) ||
        (rc = raise_smem(k_prior<true, false, true, DIMS, false>, sm)) ||
        (rc = raise_smem(k_prior<false, false, true, DIMS, false>, sm)))
        return rc;
    return TC_OK;
}

}  // namespace

int prior_configure_kernels() {
    int rc;
    if ((rc = configure_dims<3>()) || (rc = configure_dims<2>())) return rc;
    return TC_OK;
}
