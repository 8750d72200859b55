// Batches of slices with uneven geometry (image side, angle count, detector
// width) in persistent launches over work lists.
//
// A plan group holds one plan per geometry, sized for all of that geometry's
// slices.  Per pipeline stage, the geometries fall into classes that share a
// launch shape: the image side for the column and row passes, the detector
// transform (Bluestein length, or mixed radix) for the detector passes.  Each
// (stage, class) runs as one persistent launch of as many CTAs as fit on the
// GPU; every CTA takes the next (geometry, slice, tile) item of the class's
// work list from an atomic ticket -- a column strip, a grid row or an angle
// pair -- runs the same pass body as the per-plan kernels (radon_passes.cuh)
// with that item's geometry, and takes another until the list is empty.
// Items are listed largest geometry first, so the small ones fill the tail.
// Stage boundaries are kernel boundaries: no CTA ever waits for another.
// The arithmetic is the per-plan kernels'; results agree with the
// per-geometry plans to FP32 rounding (separately compiled kernels may fuse a
// multiply and an add differently), and the data term's FP64 partials are
// summed in the per-plan order.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "profile.cuh"
#include "radon_passes.cuh"

int tc_plan_build(const tc_geom *geom, int max_batch, tc_plan **out);
void tc_plan_free(tc_plan *p);

namespace {

enum { GS_FWD_COL = 0, GS_FWD_ROW, GS_FWD_DET, GS_ADJ_DET, GS_ADJ_ROW, GS_ADJ_COL, GS_COUNT };

// One geometry of a group, as the grouped kernels see it.
struct GroupGeom {
    KArgs k;
    float2 *tu, *pv;          // the geometry's plan scratch (all its slices)
    float *sr;                // weighted residual sinograms
    double *part;             // FP64 partials of the data term [count][angle pairs]
    int cp;                   // column pairs per CTA of the column passes
    int count;                // slices
    long long xoff, yoff;     // first element of its slices in the concatenated images / sinograms
    int tiles[GS_COUNT];      // items per slice of each stage
};

// The persistent loop over the items [first, end) of one class: take tickets
// until the list is exhausted; f runs item (geometry G, tile t, slice b) with
// the whole block.  starts[pos] is the first item of the pos-th geometry of the
// stage's list (geo[pos] its index in gg); the class's geometries begin at
// position pos0.
template <class F>
__device__ __forceinline__ void run_items(const GroupGeom *__restrict__ gg, const int *__restrict__ starts,
                                          const int *__restrict__ geo, int pos0, int stage, int first, int end,
                                          int *__restrict__ ticket, F &&f) {
    __shared__ int item_s;
    for (;;) {
        __syncthreads();  // the previous item is done with shared memory and item_s
        if (threadIdx.x == 0) item_s = first + atomicAdd(ticket, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= end) return;
        int pos = pos0;
        while (item >= starts[pos + 1]) ++pos;
        const GroupGeom &G = gg[geo[pos]];
        const int local = item - starts[pos], nt = G.tiles[stage];
        f(G, local % nt, local / nt);
    }
}

#define GK_ARGS const GroupGeom *__restrict__ gg, const int *__restrict__ starts, const int *__restrict__ geo, \
                int pos0, int first, int end, int *__restrict__ ticket

template <int LOGN>
__global__ void __launch_bounds__(512) gk_fwd_col(GK_ARGS, const float *__restrict__ x) {
    run_items(gg, starts, geo, pos0, GS_FWD_COL, first, end, ticket, [&](const GroupGeom &G, int t, int b) {
        fwd_col_body<LOGN, false>(x + G.xoff, G.tu, G.k, G.cp, nullptr, nullptr, t, b);
    });
}

template <int LOGN>
__global__ void __launch_bounds__(LOGN == 11 ? 256 : 512, LOGN == 11 ? 5 : 1) gk_fwd_row(GK_ARGS) {
    run_items(gg, starts, geo, pos0, GS_FWD_ROW, first, end, ticket,
              [&](const GroupGeom &G, int t, int b) { fwd_row_body<LOGN>(G.tu, G.pv, G.k, t, b); });
}

// y (sinograms out, may be null), bs and ws (may be null): mode as k_fwd_det
template <bool BLUE, int LOGL>
__global__ void __launch_bounds__(512) gk_fwd_det(GK_ARGS, float *__restrict__ y, const float *__restrict__ bs,
                                                  const float *__restrict__ ws, int mode) {
    run_items(gg, starts, geo, pos0, GS_FWD_DET, first, end, ticket, [&](const GroupGeom &G, int t, int b) {
        fwd_det_body<BLUE, LOGL>(G.pv, y ? y + G.yoff : nullptr, bs ? bs + G.yoff : nullptr,
                                 ws ? ws + G.yoff : nullptr, G.sr, G.part, G.k, mode, t, b, G.tiles[GS_FWD_DET]);
    });
}

// the adjoint's input: y (concatenated sinograms), or each geometry's residual when y is null
template <bool BLUE, int LOGL>
__global__ void __launch_bounds__(512) gk_adj_det(GK_ARGS, const float *__restrict__ y) {
    run_items(gg, starts, geo, pos0, GS_ADJ_DET, first, end, ticket, [&](const GroupGeom &G, int t, int b) {
        adj_det_body<BLUE, LOGL>(y ? y + G.yoff : G.sr, G.pv, G.k, t, b);
    });
}

template <int LOGN>
__global__ void __launch_bounds__(512) gk_adj_row(GK_ARGS) {
    run_items(gg, starts, geo, pos0, GS_ADJ_ROW, first, end, ticket,
              [&](const GroupGeom &G, int t, int b) { adj_row_body<LOGN>(G.pv, G.tu, G.k, t, b); });
}

template <int LOGN>
__global__ void __launch_bounds__(512) gk_adj_col(GK_ARGS, float *__restrict__ x) {
    run_items(gg, starts, geo, pos0, GS_ADJ_COL, first, end, ticket, [&](const GroupGeom &G, int t, int b) {
        adj_col_body<LOGN, COL_DEAPOD>(G.tu, x + G.xoff, G.k, G.cp, nullptr, nullptr, nullptr, t, b,
                                       G.tiles[GS_ADJ_COL]);
    });
}

// obj[2 i] = the data term of geometry i (caller's order): its FP64 partials
// summed in the order the per-plan reduction uses (k_reduce_finalize), one
// block each.
__global__ void gk_data_finalize(const GroupGeom *__restrict__ gg, double *__restrict__ obj) {
    __shared__ double red[32];
    const GroupGeom &G = gg[blockIdx.x];
    const int n = G.count * G.tiles[GS_FWD_DET];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += G.part[i];
    const double tot = block_sum_f64(s, red);
    if (threadIdx.x == 0) obj[2 * blockIdx.x] = 0.0 + 1.0 * tot;
}

}  // namespace

// One persistent launch: the items [first, end) of one class of one stage.
struct ClassLaunch {
    int stage;
    int key;        // log2 N (column / row passes); Bluestein log2 L, 0 run-time L, -1 mixed radix (detector)
    int pos0;       // first position of the class in the stage's geometry order
    int first, end; // item range
    int grid, threads;
    size_t smem;
};

struct tc_plan_group {
    int device = 0, ng = 0;
    std::vector<tc_plan *> plans;    // caller's order
    std::vector<int> counts;
    std::vector<long long> xoff, yoff;
    GroupGeom *dgeoms = nullptr;     // caller's order
    int *dstarts = nullptr;          // [GS_COUNT][ng + 1] first item of each position of the stage's order
    int *dgeo = nullptr;             // [GS_COUNT][ng] position -> geometry
    int *tickets = nullptr;          // one per class launch
    std::vector<ClassLaunch> launches;
    long long bytes = 0;
};

namespace {

void group_free(tc_plan_group *g) {
    if (!g) return;
    for (tc_plan *p : g->plans) tc_plan_free(p);
    for (void *q : {(void *)g->dgeoms, (void *)g->dstarts, (void *)g->dgeo, (void *)g->tickets})
        if (q) cudaFree(q);
    delete g;
}

int det_key(const KArgs &k) {
    if (!k.blue) return -1;
    return (k.log2L >= 8 && k.log2L <= 13) ? k.log2L : 0;
}

template <class F>
void with_det_key(int key, F &&f) {
    switch (key) {
        case -1: f(std::false_type{}, std::integral_constant<int, 0>{}); break;
        case 8: f(std::true_type{}, std::integral_constant<int, 8>{}); break;
        case 9: f(std::true_type{}, std::integral_constant<int, 9>{}); break;
        case 10: f(std::true_type{}, std::integral_constant<int, 10>{}); break;
        case 11: f(std::true_type{}, std::integral_constant<int, 11>{}); break;
        case 12: f(std::true_type{}, std::integral_constant<int, 12>{}); break;
        case 13: f(std::true_type{}, std::integral_constant<int, 13>{}); break;
        default: f(std::true_type{}, std::integral_constant<int, 0>{}); break;
    }
}

// The kernel of one class launch, handed to f as a function pointer.
template <class F>
int with_class_kernel(int stage, int key, F &&f) {
    int rc = TC_OK;
    switch (stage) {
        case GS_FWD_COL: return with_logn(key, [&](auto L) { return f(gk_fwd_col<decltype(L)::value>); });
        case GS_FWD_ROW: return with_logn(key, [&](auto L) { return f(gk_fwd_row<decltype(L)::value>); });
        case GS_ADJ_ROW: return with_logn(key, [&](auto L) { return f(gk_adj_row<decltype(L)::value>); });
        case GS_ADJ_COL: return with_logn(key, [&](auto L) { return f(gk_adj_col<decltype(L)::value>); });
        case GS_FWD_DET:
            with_det_key(key, [&](auto blue, auto L) { rc = f(gk_fwd_det<decltype(blue)::value, decltype(L)::value>); });
            return rc;
        case GS_ADJ_DET:
            with_det_key(key, [&](auto blue, auto L) { rc = f(gk_adj_det<decltype(blue)::value, decltype(L)::value>); });
            return rc;
    }
    return TC_ERR_INVALID_ARG;
}

// Occupancy-sized grid of one class launch (and its shared-memory opt-in).
int class_config(ClassLaunch &c, int device) {
    return with_class_kernel(c.stage, c.key, [&](auto *kern) -> int {
        cudaFuncAttributes at;
        TC_CUDA(cudaFuncGetAttributes(&at, kern));
        if ((size_t)at.maxDynamicSharedSizeBytes < c.smem)
            TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
        int per_sm = 0, sms = 0;
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c.threads, c.smem));
        TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        if (per_sm < 1) return TC_ERR_UNSUPPORTED;
        c.grid = std::max(1, std::min(c.end - c.first, per_sm * sms));
        return TC_OK;
    });
}

// Runs every class launch of one stage (x: images in; y: sinograms in or
// out; b, w, mode: the forward detector pass's epilogue; xo: images out).
int launch_stage(tc_plan_group *g, int st, cudaStream_t s, const float *x, float *y, const float *b,
                 const float *w, int mode, float *xo) {
    const int *starts = g->dstarts + (size_t)st * (g->ng + 1), *geo = g->dgeo + (size_t)st * g->ng;
    for (size_t li = 0; li < g->launches.size(); ++li) {
        const ClassLaunch &c = g->launches[li];
        if (c.stage != st) continue;
        int *tk = g->tickets + li;
        const dim3 grid(c.grid), blk(c.threads);
        const size_t sm = c.smem;
#define GK_PASS g->dgeoms, starts, geo, c.pos0, c.first, c.end, tk
        int rc = TC_OK;
        switch (st) {
            case GS_FWD_COL:
                rc = with_logn(c.key, [&](auto L) {
                    TC_PROFILED(TCK_FWD_COL, s, (gk_fwd_col<decltype(L)::value><<<grid, blk, sm, s>>>(GK_PASS, x)));
                    return TC_OK;
                });
                break;
            case GS_FWD_ROW:
                rc = with_logn(c.key, [&](auto L) {
                    TC_PROFILED(TCK_FWD_ROW, s, (gk_fwd_row<decltype(L)::value><<<grid, blk, sm, s>>>(GK_PASS)));
                    return TC_OK;
                });
                break;
            case GS_FWD_DET:
                with_det_key(c.key, [&](auto blue, auto L) {
                    TC_PROFILED(TCK_FWD_DET, s,
                                (gk_fwd_det<decltype(blue)::value, decltype(L)::value>
                                 <<<grid, blk, sm, s>>>(GK_PASS, y, b, w, mode)));
                });
                break;
            case GS_ADJ_DET:
                with_det_key(c.key, [&](auto blue, auto L) {
                    TC_PROFILED(TCK_ADJ_DET, s,
                                (gk_adj_det<decltype(blue)::value, decltype(L)::value><<<grid, blk, sm, s>>>(GK_PASS, y)));
                });
                break;
            case GS_ADJ_ROW:
                rc = with_logn(c.key, [&](auto L) {
                    TC_PROFILED(TCK_ADJ_ROW, s, (gk_adj_row<decltype(L)::value><<<grid, blk, sm, s>>>(GK_PASS)));
                    return TC_OK;
                });
                break;
            case GS_ADJ_COL:
                rc = with_logn(c.key, [&](auto L) {
                    TC_PROFILED(TCK_ADJ_COL, s, (gk_adj_col<decltype(L)::value><<<grid, blk, sm, s>>>(GK_PASS, xo)));
                    return TC_OK;
                });
                break;
        }
#undef GK_PASS
        if (rc) return rc;
        TC_LAUNCHED("grouped pass");
    }
    return TC_OK;
}

struct GroupDevice {
    int prev = -1;
    bool ok = true;
    explicit GroupDevice(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess || (prev != dev && cudaSetDevice(dev) != cudaSuccess)) ok = false;
    }
    ~GroupDevice() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

int tc_plan_group_create(const tc_geom *geoms, const int *counts, int n_geoms, tc_plan_group **out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!geoms || !counts || n_geoms < 1 || n_geoms > 256) return TC_ERR_INVALID_ARG;
    for (int i = 0; i < n_geoms; ++i)
        if (counts[i] < 1 || counts[i] > 65535) return TC_ERR_INVALID_ARG;
    tc_plan_group *g = new tc_plan_group();
    const int n = n_geoms;
    g->ng = n;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return TC_ERR_CUDA;
    }
    long long xo = 0, yo = 0;
    std::vector<GroupGeom> hg(n);
    for (int i = 0; i < n; ++i) {
        tc_plan *p = nullptr;
        const int rc = tc_plan_create(&geoms[i], counts[i], &p);
        if (rc) {
            group_free(g);
            return rc;
        }
        g->plans.push_back(p);
        g->counts.push_back(counts[i]);
        g->xoff.push_back(xo);
        g->yoff.push_back(yo);
        GroupGeom &G = hg[i];
        std::memset(&G, 0, sizeof(G));
        G.k = p->k;
        G.tu = p->tu;
        G.pv = p->pv;
        G.sr = p->sr;
        G.part = p->partials;
        G.cp = p->cp_col;
        G.count = counts[i];
        G.xoff = xo;
        G.yoff = yo;
        const int col = p->k.N / (2 * p->cp_col), rows = p->k.R, det = (p->k.A + 1) / 2;
        const int tiles[GS_COUNT] = {col, rows, det, det, rows, col};
        for (int st = 0; st < GS_COUNT; ++st) G.tiles[st] = tiles[st];
        xo += (long long)counts[i] * p->k.N * p->k.N;
        yo += (long long)counts[i] * p->k.A * p->k.D;
        g->bytes += p->bytes;
    }
    // per stage: geometries ordered by class, then largest first; one launch per class
    std::vector<int> starts((size_t)GS_COUNT * (n + 1)), geo((size_t)GS_COUNT * n);
    for (int st = 0; st < GS_COUNT; ++st) {
        const bool det = st == GS_FWD_DET || st == GS_ADJ_DET;
        auto key = [&](int i) { return det ? det_key(g->plans[i]->k) : g->plans[i]->k.log2N; };
        auto cost = [&](int i) { return (long long)hg[i].tiles[st] * hg[i].count; };
        std::vector<int> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
            return key(a) != key(b) ? key(a) < key(b) : cost(a) > cost(b);
        });
        long long item = 0;
        for (int pos = 0; pos < n; ++pos) {
            geo[(size_t)st * n + pos] = ord[pos];
            starts[(size_t)st * (n + 1) + pos] = (int)item;
            item += cost(ord[pos]);
            if (item >= (1LL << 31)) {
                group_free(g);
                return TC_ERR_UNSUPPORTED;
            }
        }
        starts[(size_t)st * (n + 1) + n] = (int)item;
        for (int p0 = 0; p0 < n;) {
            int p1 = p0;
            ClassLaunch c{};
            c.stage = st;
            c.key = key(ord[p0]);
            c.pos0 = p0;
            while (p1 < n && key(ord[p1]) == c.key) {
                const tc_plan *p = g->plans[ord[p1]];
                if (st == GS_FWD_COL || st == GS_ADJ_COL) {
                    c.threads = std::max(c.threads, p->threads_col);
                    c.smem = std::max(c.smem, p->smem_col);
                } else if (st == GS_FWD_ROW || st == GS_ADJ_ROW) {
                    c.threads = std::max(c.threads, p->threads_row);
                    c.smem = std::max(c.smem, st == GS_FWD_ROW ? p->smem_row_fwd : p->smem_row_adj);
                } else {
                    c.threads = std::max(c.threads, p->threads_det);
                    c.smem = std::max(c.smem, p->smem_det);
                }
                ++p1;
            }
            c.first = starts[(size_t)st * (n + 1) + p0];
            c.end = starts[(size_t)st * (n + 1) + p1];
            if (c.end > c.first) g->launches.push_back(c);
            p0 = p1;
        }
    }
    int rc = TC_OK;
    if (cudaMalloc(&g->dgeoms, sizeof(GroupGeom) * n) != cudaSuccess ||
        cudaMalloc(&g->dstarts, sizeof(int) * starts.size()) != cudaSuccess ||
        cudaMalloc(&g->dgeo, sizeof(int) * geo.size()) != cudaSuccess ||
        cudaMalloc(&g->tickets, sizeof(int) * std::max<size_t>(1, g->launches.size())) != cudaSuccess) {
        cudaGetLastError();
        group_free(g);
        return TC_ERR_OOM;
    }
    if (cudaMemcpy(g->dgeoms, hg.data(), sizeof(GroupGeom) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->dstarts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->dgeo, geo.data(), sizeof(int) * geo.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = tc_cuda_fail(cudaGetLastError(), "tc_plan_group_create");
    for (ClassLaunch &c : g->launches)
        if (!rc) rc = class_config(c, g->device);
    if (rc) {
        group_free(g);
        return rc;
    }
    *out = g;
    return TC_OK;
}

int tc_plan_group_destroy(tc_plan_group *g) {
    if (!g) return TC_OK;
    GroupDevice dg(g->device);
    cudaDeviceSynchronize();
    group_free(g);
    return TC_OK;
}

long long tc_plan_group_device_bytes(const tc_plan_group *g) { return g ? g->bytes : 0; }

int radon_fwd_group(tc_plan_group *g, const float *x, float *y, void *stream) {
    if (!g || !x || !y || !aligned16(x) || !aligned16(y)) return TC_ERR_INVALID_ARG;
    GroupDevice dg(g->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * g->launches.size(), s));
    int rc;
    if ((rc = launch_stage(g, GS_FWD_COL, s, x, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_ROW, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_DET, s, nullptr, y, nullptr, nullptr, DET_WRITE_Y, nullptr)))
        return rc;
    return TC_OK;
}

int radon_adj_group(tc_plan_group *g, const float *y, float *x, void *stream) {
    if (!g || !x || !y || !aligned16(x) || !aligned16(y)) return TC_ERR_INVALID_ARG;
    GroupDevice dg(g->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * g->launches.size(), s));
    int rc;
    if ((rc = launch_stage(g, GS_ADJ_DET, s, nullptr, const_cast<float *>(y), nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_ADJ_ROW, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_ADJ_COL, s, nullptr, nullptr, nullptr, nullptr, 0, x)))
        return rc;
    return TC_OK;
}

int mbir_grad_group(tc_plan_group *g, const float *x, const float *b, const float *w, const tc_prior *prior,
                    float *grad, double *obj, void *stream) {
    if (!g || !x || !b || !grad || !aligned16(x) || !aligned16(b) || !aligned16(grad) || (w && !aligned16(w)))
        return TC_ERR_INVALID_ARG;
    if (prior && (!(prior->dims == 2 || prior->dims == 3) || !(prior->sigma > 0) || !(prior->c > 0) ||
                  !(prior->p >= 1.0 && prior->p <= 2.0) || !(prior->lambda >= 0)))
        return TC_ERR_INVALID_ARG;
    GroupDevice dg(g->device);
    if (!dg.ok) return TC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * g->launches.size(), s));
    if (obj) TC_CUDA(cudaMemsetAsync(obj, 0, sizeof(double) * 2 * g->ng, s));
    const int mode = DET_RESID | (obj ? DET_OBJ : 0);
    int rc;
    if ((rc = launch_stage(g, GS_FWD_COL, s, x, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_ROW, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_DET, s, nullptr, nullptr, b, w, mode, nullptr)))
        return rc;
    if (obj) {
        TC_PROFILED(TCK_REDUCE, s, gk_data_finalize<<<g->ng, 256, 0, s>>>(g->dgeoms, obj));
        TC_LAUNCHED("gk_data_finalize");
    }
    if ((rc = launch_stage(g, GS_ADJ_DET, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_ADJ_ROW, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_ADJ_COL, s, nullptr, nullptr, nullptr, nullptr, 0, grad)))
        return rc;
    if (prior && prior->lambda != 0.0) {
        for (int i = 0; i < g->ng; ++i) {
            tc_plan *p = g->plans[i];
            if ((rc = launch_prior_grad(p, x + g->xoff[i], grad + g->xoff[i], g->counts[i], prior,
                                        obj ? obj + 2 * i + 1 : nullptr, s)))
                return rc;
        }
    }
    return TC_OK;
}

}  // extern "C"
