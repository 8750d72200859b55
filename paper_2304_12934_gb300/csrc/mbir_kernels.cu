// MBIR kernels (arXiv 2304.12934, Sec. 3): the qGGMRF prior value and
// gradient (Eqs. reg2, reg3), FP64 reductions for the objective and the
// restart test, and the accelerated-gradient update with restart.
//
// Vectors are FP32; every reduction accumulates at most a few FP32 products
// per thread before promoting to FP64, then sums per-block FP64 partials in a
// fixed order, so results are bit-reproducible run to run.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "profile.cuh"

namespace {

struct PriorArgs {
    int N, B, dims;
    int z0, z1;        // slices of the volume [0, B) whose gradient this launch produces
    float p, c, qexp;  // qexp = 2 - p
    float cq;          // c (2 - p)
    float lk;          // qexp * log2(1 / sigma)
    float two_c;       // 2 c
    float gscale;      // 2 lambda / sigma^2: scale of the gradient sum
    float step;        // DOTS: the solver's step; g receives z - step * grad instead of grad
    float w1, w2, w3;  // weights at distance 1, sqrt 2, sqrt 3
};

// Hardware approximations (one instruction each, denormals flushed to zero):
// relative errors ~1e-7, far inside the prior's FP32 tolerance.
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// rho(d) = u^2 / (c + |u|^(2-p)), u = d / sigma (Eq. reg3), differentiated by
// hand:  rho'(d) = (d / sigma^2) (p |u|^(2-p) + 2c) / (c + |u|^(2-p))^2
//                = (d / sigma^2) inv (p + c (2 - p) inv),  inv = 1 / (c + |u|^(2-p)).
// Returns sigma^2 rho'(d) (the constant is applied once per voxel) and inv,
// from which sigma^2 rho(d) = d^2 inv.
// |u|^(2-p) = 2^((2-p) log2|d| + (2-p) log2(1/sigma)); at d = 0, log2 gives
// -inf and the power 0.
__device__ __forceinline__ float qggmrf_e(float d, const PriorArgs &a, float &inv_out) {
    const float q = ex2_approx(fmaf(a.qexp, lg2_approx(fabsf(d)), a.lk));
    const float inv = rcp_approx(a.c + q);
    inv_out = inv;
    return (d * inv) * fmaf(a.cq, inv, a.p);
}

// inv alone, for the value sigma^2 rho(d) = d^2 inv
__device__ __forceinline__ float qggmrf_inv(float d, const PriorArgs &a) {
    return rcp_approx(a.c + ex2_approx(fmaf(a.qexp, lg2_approx(fabsf(d)), a.lk)));
}

// qGGMRF prior on a volume [B][N][N] (slices consecutive along z).
// A CTA owns a PTX x PTY column of voxels and marches along z holding a ring
// (tile + 1-voxel halo) of two f planes in shared memory.  Each unordered
// neighbour pair is evaluated once, at its lower voxel, along the 13 forward
// directions (9 towards z+1, 4 in-plane); both voxels read the pair's rho'
// from shared memory (the z+1 pairs are kept for the voxel above).
// Buffers: pair values towards z+1 alternate between two slots (a step's
// gradient phase reads the previous step's), the in-plane ones use one; the
// barrier that opens each step orders all reads of the previous step before
// its writes.  With the plane double buffer that is two barriers per z step.
// dims = 2 skips the z pairs and uses the 8-neighbour weights.
// A CTA whose ring lies inside the volume evaluates every direction at every
// ring cell without per-pair tests (the pairs that leave the ring are never
// read); CTAs at the volume border test each pair against the border rule.
// WANT_H also accumulates H (otherwise only the gradient is produced).
// DOTS also accumulates <g, f - xprev> and <g, g> of the final gradient g (the
// inner products of the solver's restart test), sparing a separate pass, and
// stores the solver's next iterate f - step g in place of g.
// Per-thread sums run in FP32 over 8, 64 and 512 z steps and in FP64 from the
// block sum on (the FP64 pipe of this part is narrow), always in the same order.
#define PTX 32
#define PTY 12
#define PRX (PTX + 2)
#define PRY (PTY + 2)
#define PRS (PRX * PRY)
#define PRIOR_THREADS 480
#define PRIOR_FPAD 36  // front pad: unmasked halo reads reach PRX + 1 cells before a plane
#define PRIOR_UP_SLOTS 2    // buffers of z+1 pair values
#define PRIOR_PL_SLOTS 1    // buffers of in-plane pair values
#define PRIOR_MIN_BLOCKS 4  // 46 KB of shared memory and <= 32 registers: 60 warps per SM
#define PRIOR_SMEM_FLOATS (PRIOR_FPAD + 2 * PRS + PRIOR_UP_SLOTS * 9 * PRS + PRIOR_PL_SLOTS * 4 * PRS)
// the first warp covers only the bottom halo row, the last only the top one
static_assert(PRX >= 32 && (PRIOR_THREADS / 32 - 1) * 32 >= (PRY - 1) * PRX && PRIOR_THREADS >= PRS,
              "halo-row warps");

// z+1 pairs of one ring cell: fc / fn point at the cell in planes z and z+1,
// eu at its slot of the current z+1 buffer.
// gs accumulates the cell's own (forward) share of the gradient sum, w e.
// GRAD = false: the value alone (no pair derivatives, nothing stored).
// DIRS: directions evaluated at all (compile time; the others are skipped and
// their slots left untouched, for rows of the halo that never need them).
template <bool MASKED, bool WANT_H, bool GRAD, unsigned DIRS = 0x1ffu>
__device__ __forceinline__ void prior_up_pairs(const float *fn, float fm, float *eu, unsigned mu,
                                               const PriorArgs &a, float &gs, float &hs) {
#pragma unroll
    for (int u = 0; u < 9; ++u) {
        if (!(DIRS & (1u << u))) continue;
        const int dx = u % 3 - 1, dy = u / 3 - 1;
        const float wu = (dx == 0 && dy == 0) ? a.w1 : ((dx == 0 || dy == 0) ? a.w2 : a.w3);
        float e = 0.f;
        if (!MASKED || (mu & (1u << u))) {
            const float d = fm - fn[dy * PRX + dx];
            if (GRAD) {
                float inv;
                e = qggmrf_e(d, a, inv);
                gs = fmaf(wu, e, gs);
                if (WANT_H) hs = fmaf(wu, d * d * inv, hs);
            } else {
                hs = fmaf(wu, d * d * qggmrf_inv(d, a), hs);
            }
        }
        if (GRAD) eu[u * PRS] = e;
    }
}

// in-plane forward directions (dx, dy): (1,0) (-1,1) (0,1) (1,1)
__device__ __forceinline__ int pl_dx(int q) { return q == 0 ? 1 : (q == 1 ? -1 : (q == 2 ? 0 : 1)); }
__device__ __forceinline__ int pl_dy(int q) { return q == 0 ? 0 : 1; }

template <bool MASKED, bool WANT_H, bool GRAD, unsigned DIRS = 0xfu>
__device__ __forceinline__ void prior_plane_pairs(const float *fc, float fm, float *ep, unsigned mp,
                                                  const PriorArgs &a, float &gs, float &hs) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!(DIRS & (1u << q))) continue;
        const float wq = (q & 1) ? a.w2 : a.w1;
        float e = 0.f;
        if (!MASKED || (mp & (1u << q))) {
            const float d = fm - fc[pl_dy(q) * PRX + pl_dx(q)];
            if (GRAD) {
                float inv;
                e = qggmrf_e(d, a, inv);
                gs = fmaf(wq, e, gs);
                if (WANT_H) hs = fmaf(wq, d * d * inv, hs);
            } else {
                hs = fmaf(wq, d * d * qggmrf_inv(d, a), hs);
            }
        }
        if (GRAD) ep[q * PRS] = e;
    }
}

template <bool WANT_H, bool DOTS, bool GRAD = true>
__global__ void __launch_bounds__(PRIOR_THREADS, PRIOR_MIN_BLOCKS) k_prior(const float *__restrict__ f, float *__restrict__ g,
                                                          double *__restrict__ partials, const PriorArgs a,
                                                          const float *__restrict__ xprev,
                                                          double *__restrict__ pd1, double *__restrict__ pd2) {
    extern __shared__ float psm[];
    float *fpl = psm + PRIOR_FPAD;    // [2][PRS]
    float *Eu = fpl + 2 * PRS;        // [3][9][PRS]
    float *Ep = Eu + PRIOR_UP_SLOTS * 9 * PRS;  // [PRIOR_PL_SLOTS][4][PRS]
    __shared__ double red[32];
    const int N = a.N, B = a.B;
    const size_t NN = (size_t)N * N;
    const int h = threadIdx.x, warp = h >> 5;
    const int hx = h % PRX, hy = h / PRX;
    const int x0 = blockIdx.x * PTX - 1, y0 = blockIdx.y * PTY - 1;
    const int x = x0 + hx, y = y0 + hy;
    const bool ring = h < PRS;
    const bool inb = ring && x >= 0 && x < N && y >= 0 && y < N;
    const bool interior = inb && hx >= 1 && hx <= PTX && hy >= 1 && hy <= PTY;
    const bool three = a.dims == 3;
    // the whole ring inside the volume: no pair needs the border test
    const bool full = x0 >= 0 && y0 >= 0 && x0 + PRX <= N && y0 + PRY <= N;
    auto ring_in = [&](int dx, int dy) {
        const int nx = hx + dx, ny = hy + dy;
        if (nx < 0 || nx >= PRX || ny < 0 || ny >= PRY) return false;
        const int gx = x + dx, gy = y + dy;
        return gx >= 0 && gx < N && gy >= 0 && gy < N;
    };
    auto is_interior = [&](int dx, int dy) {
        const int nx = hx + dx, ny = hy + dy;
        return nx >= 1 && nx <= PTX && ny >= 1 && ny <= PTY && x + dx < N && y + dy < N &&
               x + dx >= 0 && y + dy >= 0;
    };
    // border CTAs: bit u of mup / bit q of mpl says the pair towards (dx, dy)
    // is inside the volume and needed by an interior voxel (the same at every z)
    unsigned mup = 0, mpl = 0;
    if (!full) {
#pragma unroll
        for (int u = 0; u < 9; ++u) {
            const int dx = u % 3 - 1, dy = u / 3 - 1;
            if (inb && ring_in(dx, dy) && (interior || is_interior(dx, dy))) mup |= 1u << u;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (inb && ring_in(pl_dx(q), pl_dy(q)) && (interior || is_interior(pl_dx(q), pl_dy(q))))
                mpl |= 1u << q;
    }
    // A slab [z0, z1) of a 3D volume starts one plane below, at the halo plane,
    // whose step only evaluates the pairs towards z0 (no gradient, no sums).
    const int zs = (three && a.z0 > 0) ? a.z0 - 1 : a.z0;
    const size_t off = (size_t)y * N + x;
    if (ring) {
        for (int u = 0; u < 9; ++u)
            for (int sl = 0; sl < PRIOR_UP_SLOTS; ++sl) Eu[(sl * 9 + u) * PRS + h] = 0.f;
        fpl[h] = inb ? f[(size_t)zs * NN + off] : 0.f;
    }
    // register prefetch: the plane the next step stores (3D: z + 2, 2D: z + 1)
    float f_nx = (inb && zs + 1 < B) ? f[(size_t)(zs + 1) * NN + off] : 0.f;
    // per-thread sums: FP32 over 8, 64 and 512 z steps (a level never adds
    // more than 8 terms for volumes up to 4096 slices), FP64 from the block sum on
    float h8 = 0.f, h64 = 0.f, h512 = 0.f, a8 = 0.f, a64 = 0.f, a512 = 0.f, b8 = 0.f, b64 = 0.f, b512 = 0.f;
    static_assert(PRIOR_UP_SLOTS == 2 && PRIOR_PL_SLOTS == 1, "buffer slots alternate with the z parity");
    // One z step; PAR = (z - zs) & 1 fixes every buffer (planes, z+1 pair
    // slots) at compile time, so the march runs two steps per iteration.
    auto step = [&](auto par, int z) {
        constexpr int cur = decltype(par)::value, nxt = cur ^ 1;
        constexpr int s3 = cur, p3 = nxt;  // this step's / previous step's z+1 slot
        const bool own = z >= a.z0;
        const bool up = three && z + 1 < B;
        const int pz = three ? z + 2 : z + 1;
        const float f_pf = (inb && pz < B) ? f[(size_t)pz * NN + off] : 0.f;
        const size_t i = (size_t)z * NN + off;
        const float g_old = (GRAD && own && interior) ? g[i] : 0.f;
        const float x_old = (DOTS && own && interior) ? xprev[i] : 0.f;
        if (GRAD && interior && z + 2 < a.z1) {  // the same lines two planes on, into L2
            asm volatile("prefetch.global.L2 [%0];" ::"l"(g + i + 2 * NN));
            if (DOTS) asm volatile("prefetch.global.L2 [%0];" ::"l"(xprev + i + 2 * NN));
        }
        if (ring) {
            if (up) fpl[nxt * PRS + h] = f_nx;                 // 3D: plane z + 1
            else if (!three && z > zs) fpl[cur * PRS + h] = f_nx;  // 2D: slices are independent
        }
        __syncthreads();
        float hs = 0.f, fm = 0.f, gs = 0.f;
        // the value alone needs the pairs of interior cells only (a pair
        // enters H at its lower voxel); the gradient also needs the halo's
        if (GRAD ? ring : interior) {
            const float *fc = fpl + cur * PRS + h;
            fm = *fc;
            float *eu = Eu + (s3 * 9) * PRS + h;
            float *ep = Ep + h;
            const float *fn = fpl + nxt * PRS + h;
            if (GRAD && three && !up) {
#pragma unroll
                for (int u = 0; u < 9; ++u) eu[u * PRS] = 0.f;
            }
            if (!full) {
                if (up) prior_up_pairs<true, WANT_H, GRAD>(fn, fm, eu, mup, a, gs, hs);
                prior_plane_pairs<true, WANT_H, GRAD>(fc, fm, ep, mpl, a, gs, hs);
            } else if (GRAD && warp == 0) {
                // bottom halo row: only pairs towards dy = +1 reach the interior
                if (up) prior_up_pairs<false, WANT_H, GRAD, 0x1c0u>(fn, fm, eu, 0u, a, gs, hs);
                prior_plane_pairs<false, WANT_H, GRAD, 0xeu>(fc, fm, ep, 0u, a, gs, hs);
            } else if (GRAD && warp == PRIOR_THREADS / 32 - 1) {
                // top halo row: only the z+1 pairs towards dy = -1
                if (up) prior_up_pairs<false, WANT_H, GRAD, 0x007u>(fn, fm, eu, 0u, a, gs, hs);
            } else {
                if (up) prior_up_pairs<false, WANT_H, GRAD>(fn, fm, eu, 0u, a, gs, hs);
                prior_plane_pairs<false, WANT_H, GRAD>(fc, fm, ep, 0u, a, gs, hs);
            }
        }
        __syncthreads();
        if (!GRAD) {
            if (own && interior) h8 += hs;
        } else if (own && interior) {
            // minus the shares of the pairs this voxel closes (evaluated at
            // their lower voxels: in-plane this step, towards z+1 the last)
            if (three) {
                const float *epv = Eu + (p3 * 9) * PRS + h;
#pragma unroll
                for (int u = 0; u < 9; ++u) {
                    const int dx = u % 3 - 1, dy = u / 3 - 1;
                    const float wu = (dx == 0 && dy == 0) ? a.w1 : ((dx == 0 || dy == 0) ? a.w2 : a.w3);
                    gs = fmaf(-wu, epv[u * PRS - dy * PRX - dx], gs);
                }
            }
            const float *ep = Ep + h;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                gs = fmaf((q & 1) ? -a.w2 : -a.w1, ep[q * PRS - pl_dy(q) * PRX - pl_dx(q)], gs);
            const float gn = fmaf(a.gscale, gs, g_old);
            // the solver needs x_{k+1} = z_k - step grad, not grad itself
            g[i] = DOTS ? fmaf(-a.step, gn, fm) : gn;
            if (WANT_H) h8 += hs;
            if (DOTS) {
                a8 = fmaf(gn, fm - x_old, a8);
                b8 = fmaf(gn, gn, b8);
            }
        }
        if ((z & 7) == 7) {
            h64 += h8; a64 += a8; b64 += b8;
            h8 = a8 = b8 = 0.f;
            if ((z & 63) == 63) {
                h512 += h64; a512 += a64; b512 += b64;
                h64 = a64 = b64 = 0.f;
            }
        }
        f_nx = f_pf;
    };
    int z = zs;
    for (; z + 1 < a.z1; z += 2) {
        step(std::integral_constant<int, 0>{}, z);
        step(std::integral_constant<int, 1>{}, z + 1);
    }
    if (z < a.z1) step(std::integral_constant<int, 0>{}, z);
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (WANT_H) {
        const double tot = block_sum_f64((double)h512 + ((double)h64 + (double)h8), red);
        if (threadIdx.x == 0) partials[bid] = tot;
    }
    if (DOTS) {
        const double t1 = block_sum_f64((double)a512 + ((double)a64 + (double)a8), red);
        const double t2 = block_sum_f64((double)b512 + ((double)b64 + (double)b8), red);
        if (threadIdx.x == 0) {
            pd1[bid] = t1;
            pd2[bid] = t2;
        }
    }
}

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
    if (restart && dot > 0.0) {
        t = 1.0;
        sc[SC_RESTARTS] += 1.0;
    }
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

PriorArgs make_prior_args(int n, int nb, const tc_prior *pr) {
    PriorArgs a;
    a.N = n;
    a.B = nb;
    a.z0 = 0;
    a.z1 = nb;
    a.dims = pr->dims;
    a.p = (float)pr->p;
    a.c = (float)pr->c;
    a.qexp = (float)(2.0 - pr->p);
    a.cq = (float)(pr->c * (2.0 - pr->p));
    a.lk = (float)((2.0 - pr->p) * std::log2(1.0 / pr->sigma));
    a.two_c = (float)(2.0 * pr->c);
    a.gscale = (float)(2.0 * pr->lambda / (pr->sigma * pr->sigma));
    a.step = 0.f;
    // w_mn proportional to 1/distance, normalised over the full neighbourhood
    double z;
    if (pr->dims == 3) z = 6.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    else z = 4.0 + 4.0 / sqrt(2.0);
    a.w1 = (float)(1.0 / z);
    a.w2 = (float)(1.0 / (sqrt(2.0) * z));
    a.w3 = (float)(1.0 / (sqrt(3.0) * z));
    return a;
}

// lambda H from the block partials of sum w d^2 inv over unordered pairs:
// every pair enters H twice (ordered pairs) and rho = d^2 inv / sigma^2.
double prior_value_scale(const tc_prior *pr) { return 2.0 * pr->lambda / (pr->sigma * pr->sigma); }

}  // namespace

int prior_tile_count(int n) { return ((n + PTX - 1) / PTX) * ((n + PTY - 1) / PTY); }

int launch_prior_grad(tc_plan *p, const float *x, float *g, int nb,
                      const tc_prior *pr, double *h_acc, cudaStream_t s, const float *dot_x,
                      int z0, int z1, double step) {
    PriorArgs a = make_prior_args(p->k.N, nb, pr);
    a.step = (float)step;
    if (z1 < 0) z1 = nb;
    if (z0 < 0 || z0 >= z1 || z1 > nb) return TC_ERR_INVALID_ARG;
    a.z0 = z0;
    a.z1 = z1;
    const int acc = z0 > 0;  // a later slab adds to the sums of the earlier ones
    dim3 grid((a.N + PTX - 1) / PTX, (a.N + PTY - 1) / PTY);
    const int blocks = grid.x * grid.y;
    if (blocks > p->slot) return TC_ERR_UNSUPPORTED;
    double *part = p->partials + (size_t)1 * p->slot;
    const size_t smem = PRIOR_SMEM_FLOATS * sizeof(float);
    double *p1 = p->partials + (size_t)2 * p->slot, *p2 = p->partials + (size_t)3 * p->slot;
    if (dot_x) {
        if (h_acc)
            TC_PROFILED(TCK_PRIOR, s, (k_prior<true, true><<<grid, PRIOR_THREADS, smem, s>>>(x, g, part, a, dot_x, p1, p2)));
        else
            TC_PROFILED(TCK_PRIOR, s, (k_prior<false, true><<<grid, PRIOR_THREADS, smem, s>>>(x, g, part, a, dot_x, p1, p2)));
    } else {
        if (h_acc)
            TC_PROFILED(TCK_PRIOR, s, (k_prior<true, false><<<grid, PRIOR_THREADS, smem, s>>>(x, g, part, a, nullptr, nullptr, nullptr)));
        else
            TC_PROFILED(TCK_PRIOR, s, (k_prior<false, false><<<grid, PRIOR_THREADS, smem, s>>>(x, g, part, a, nullptr, nullptr, nullptr)));
    }
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
    const PriorArgs a = make_prior_args(p->k.N, nb, pr);
    dim3 grid((a.N + PTX - 1) / PTX, (a.N + PTY - 1) / PTY);
    const int blocks = grid.x * grid.y;
    if (blocks > p->slot) return TC_ERR_UNSUPPORTED;
    double *part = p->partials + (size_t)1 * p->slot;
    const size_t smem = PRIOR_SMEM_FLOATS * sizeof(float);
    TC_PROFILED(TCK_PRIOR, s, (k_prior<true, false, false><<<grid, PRIOR_THREADS, smem, s>>>(
                                  x, nullptr, part, a, nullptr, nullptr, nullptr)));
    TC_LAUNCHED("k_prior");
    return launch_reduce_finalize(part, blocks, h_acc, 0, prior_value_scale(pr), s);
}

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

// Prior gradient and value with caller-supplied partial-sum storage (used by
// the no-allocation entry point in prior_noalloc.cu): g += 2 lambda sum w rho',
// *h_out = lambda H.  Same kernel and reduction as launch_prior_grad.
int launch_prior_kernel_into(const float *x, float *g, int n, int nb, const tc_prior *pr,
                             double *partials, int max_partials, double *h_out,
                             cudaStream_t s) {
    const PriorArgs a = make_prior_args(n, nb, pr);
    dim3 grid((n + PTX - 1) / PTX, (n + PTY - 1) / PTY);
    const int blocks = grid.x * grid.y;
    if (blocks > max_partials) return TC_ERR_INVALID_ARG;
    const size_t smem = PRIOR_SMEM_FLOATS * sizeof(float);
    if (h_out)
        TC_PROFILED(TCK_PRIOR, s, (k_prior<true, false><<<grid, PRIOR_THREADS, smem, s>>>(x, g, partials, a, nullptr, nullptr, nullptr)));
    else
        TC_PROFILED(TCK_PRIOR, s, (k_prior<false, false><<<grid, PRIOR_THREADS, smem, s>>>(x, g, partials, a, nullptr, nullptr, nullptr)));
    TC_LAUNCHED("k_prior");
    if (h_out) return launch_reduce_finalize(partials, blocks, h_out, 0, prior_value_scale(pr), s);
    return TC_OK;
}

// Opt the prior kernel into its dynamic shared memory (raise only: the limit
// is a process-wide attribute of the kernel).
template <class F>
int raise_prior_smem(F *fn, int smem) {
    cudaFuncAttributes at;
    TC_CUDA(cudaFuncGetAttributes(&at, fn));
    if (at.maxDynamicSharedSizeBytes < smem)
        TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return TC_OK;
}

int prior_configure_kernels() {
    const int smem = (int)(PRIOR_SMEM_FLOATS * sizeof(float));
    int rc;
    if ((rc = raise_prior_smem(k_prior<true, false>, smem)) || (rc = raise_prior_smem(k_prior<false, false>, smem)) ||
        (rc = raise_prior_smem(k_prior<true, true>, smem)) || (rc = raise_prior_smem(k_prior<false, true>, smem)) ||
        (rc = raise_prior_smem(k_prior<true, false, false>, smem)))
        return rc;
    return TC_OK;
}
