// Batches of slices with uneven geometry (image side, angle count, detector
// width) in one persistent launch per pipeline stage.
//
// A plan group holds one plan per geometry, sized for all of that geometry's
// slices, and a work list per stage: every (geometry, slice, tile) item of
// the stage -- column strips for the column passes, grid rows for the row
// passes, angle pairs for the detector passes.  A stage runs as one launch of
// as many CTAs as fit on the GPU at once; each CTA takes the next item from an
// atomic ticket, runs the same pass body as the per-plan kernels
// (radon_passes.cuh) with that item's geometry, and takes another until the
// list is empty.  Items are listed largest geometry first, so the small ones
// fill the tail.  Stage boundaries are kernel boundaries: no CTA ever waits
// for another, so nothing can stall on a dependency.  Results equal the
// per-plan path bit for bit (same bodies, same inputs; the data term's FP64
// partials are summed in the same order).
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
    int start[GS_COUNT];      // first item of each stage's work list
};

template <class F>
__device__ __forceinline__ int with_logn_dev(int lg, F &&f) {
    switch (lg) {
        case 4: f(std::integral_constant<int, 4>{}); return 0;
        case 5: f(std::integral_constant<int, 5>{}); return 0;
        case 6: f(std::integral_constant<int, 6>{}); return 0;
        case 7: f(std::integral_constant<int, 7>{}); return 0;
        case 8: f(std::integral_constant<int, 8>{}); return 0;
        case 9: f(std::integral_constant<int, 9>{}); return 0;
        case 10: f(std::integral_constant<int, 10>{}); return 0;
        case 11: f(std::integral_constant<int, 11>{}); return 0;
        case 12: f(std::integral_constant<int, 12>{}); return 0;
        default: return 1;
    }
}

// Detector-pass dispatch: Bluestein at a compile-time length, Bluestein at a
// run-time length, or the mixed-radix DFT.
template <class F>
__device__ __forceinline__ void with_det_dev(const KArgs &k, F &&f) {
    if (!k.blue) {
        f(std::false_type{}, std::integral_constant<int, 0>{});
        return;
    }
    switch (k.log2L) {
        case 8: f(std::true_type{}, std::integral_constant<int, 8>{}); break;
        case 9: f(std::true_type{}, std::integral_constant<int, 9>{}); break;
        case 10: f(std::true_type{}, std::integral_constant<int, 10>{}); break;
        case 11: f(std::true_type{}, std::integral_constant<int, 11>{}); break;
        case 12: f(std::true_type{}, std::integral_constant<int, 12>{}); break;
        case 13: f(std::true_type{}, std::integral_constant<int, 13>{}); break;
        default: f(std::true_type{}, std::integral_constant<int, 0>{}); break;
    }
}

// The persistent loop: take tickets until the stage's list is exhausted; f
// runs the item (geometry G, tile t, slice b) with the whole block.
template <class F>
__device__ __forceinline__ void run_items(const GroupGeom *__restrict__ gg, int ng, int stage, int total,
                                          int *__restrict__ ticket, F &&f) {
    __shared__ int item_s;
    for (;;) {
        __syncthreads();  // the previous item is done with shared memory and item_s
        if (threadIdx.x == 0) item_s = atomicAdd(ticket, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= total) return;
        int gi = 0;
        while (gi + 1 < ng && item >= gg[gi + 1].start[stage]) ++gi;
        const GroupGeom &G = gg[gi];
        const int local = item - G.start[stage], nt = G.tiles[stage];
        f(G, local % nt, local / nt);
    }
}

__global__ void __launch_bounds__(512) gk_fwd_col(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket, const float *__restrict__ x) {
    run_items(gg, ng, GS_FWD_COL, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_logn_dev(G.k.log2N, [&](auto L) {
            fwd_col_body<decltype(L)::value, false>(x + G.xoff, G.tu, G.k, G.cp, nullptr, nullptr, t, b);
        });
    });
}

__global__ void __launch_bounds__(512) gk_fwd_row(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket) {
    run_items(gg, ng, GS_FWD_ROW, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_logn_dev(G.k.log2N, [&](auto L) { fwd_row_body<decltype(L)::value>(G.tu, G.pv, G.k, t, b); });
    });
}

// y (images' sinograms, may be null), b and w (may be null): mode as k_fwd_det
__global__ void __launch_bounds__(512) gk_fwd_det(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket, float *__restrict__ y,
                                                  const float *__restrict__ bs, const float *__restrict__ ws,
                                                  int mode) {
    run_items(gg, ng, GS_FWD_DET, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_det_dev(G.k, [&](auto blue, auto L) {
            fwd_det_body<decltype(blue)::value, decltype(L)::value>(
                G.pv, y ? y + G.yoff : nullptr, bs ? bs + G.yoff : nullptr, ws ? ws + G.yoff : nullptr, G.sr,
                G.part, G.k, mode, t, b, G.tiles[GS_FWD_DET]);
        });
    });
}

// the adjoint's input: y (concatenated sinograms), or each geometry's residual when y is null
__global__ void __launch_bounds__(512) gk_adj_det(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket, const float *__restrict__ y) {
    run_items(gg, ng, GS_ADJ_DET, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_det_dev(G.k, [&](auto blue, auto L) {
            adj_det_body<decltype(blue)::value, decltype(L)::value>(y ? y + G.yoff : G.sr, G.pv, G.k, t, b);
        });
    });
}

__global__ void __launch_bounds__(512) gk_adj_row(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket) {
    run_items(gg, ng, GS_ADJ_ROW, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_logn_dev(G.k.log2N, [&](auto L) { adj_row_body<decltype(L)::value>(G.pv, G.tu, G.k, t, b); });
    });
}

__global__ void __launch_bounds__(512) gk_adj_col(const GroupGeom *__restrict__ gg, int ng, int total,
                                                  int *__restrict__ ticket, float *__restrict__ x) {
    run_items(gg, ng, GS_ADJ_COL, total, ticket, [&](const GroupGeom &G, int t, int b) {
        with_logn_dev(G.k.log2N, [&](auto L) {
            adj_col_body<decltype(L)::value, COL_DEAPOD>(G.tu, x + G.xoff, G.k, G.cp, nullptr, nullptr, nullptr, t,
                                                         b, G.tiles[GS_ADJ_COL]);
        });
    });
}

// obj[2 gi] = the data term of geometry gi: its FP64 partials summed in the
// order the per-plan reduction uses (k_reduce_finalize), one block each.
__global__ void gk_data_finalize(const GroupGeom *__restrict__ gg, const int *__restrict__ caller_index,
                                 double *__restrict__ obj) {
    __shared__ double red[32];
    const GroupGeom &G = gg[blockIdx.x];
    const int n = G.count * G.tiles[GS_FWD_DET];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += G.part[i];
    const double tot = block_sum_f64(s, red);
    if (threadIdx.x == 0) obj[2 * caller_index[blockIdx.x]] = 0.0 + 1.0 * tot;
}

}  // namespace

struct tc_plan_group {
    int device = 0, ng = 0;
    std::vector<tc_plan *> plans;    // caller's order
    std::vector<int> counts;
    std::vector<long long> xoff, yoff;
    std::vector<int> order;          // work-list position -> caller index
    GroupGeom *dgeoms = nullptr;     // work-list order
    int *dorder = nullptr;           // work-list position -> caller index (device)
    int *tickets = nullptr;          // [GS_COUNT]
    int total[GS_COUNT] = {};
    int grid[GS_COUNT] = {}, threads[GS_COUNT] = {};
    size_t smem[GS_COUNT] = {};
    long long bytes = 0;
};

namespace {

void group_free(tc_plan_group *g) {
    if (!g) return;
    for (tc_plan *p : g->plans) tc_plan_free(p);
    if (g->dgeoms) cudaFree(g->dgeoms);
    if (g->dorder) cudaFree(g->dorder);
    if (g->tickets) cudaFree(g->tickets);
    delete g;
}

template <class K>
int stage_config(tc_plan_group *g, int st, K *kern, int threads, size_t smem) {
    cudaFuncAttributes at;
    TC_CUDA(cudaFuncGetAttributes(&at, kern));
    if ((size_t)at.maxDynamicSharedSizeBytes < smem)
        TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, sms = 0;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    if (per_sm < 1) return TC_ERR_UNSUPPORTED;
    g->threads[st] = threads;
    g->smem[st] = smem;
    g->grid[st] = std::max(1, std::min(g->total[st], per_sm * sms));
    return TC_OK;
}

int launch_stage(tc_plan_group *g, int st, cudaStream_t s, const float *x, float *y, const float *b,
                 const float *w, int mode, float *xo) {
    const dim3 grid(g->grid[st]), blk(g->threads[st]);
    const size_t sm = g->smem[st];
    int *tk = g->tickets + st;
    switch (st) {
        case GS_FWD_COL:
            TC_PROFILED(TCK_FWD_COL, s, gk_fwd_col<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk, x));
            break;
        case GS_FWD_ROW:
            TC_PROFILED(TCK_FWD_ROW, s, gk_fwd_row<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk));
            break;
        case GS_FWD_DET:
            TC_PROFILED(TCK_FWD_DET, s,
                        gk_fwd_det<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk, y, b, w, mode));
            break;
        case GS_ADJ_DET:
            TC_PROFILED(TCK_ADJ_DET, s, gk_adj_det<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk, y));
            break;
        case GS_ADJ_ROW:
            TC_PROFILED(TCK_ADJ_ROW, s, gk_adj_row<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk));
            break;
        case GS_ADJ_COL:
            TC_PROFILED(TCK_ADJ_COL, s, gk_adj_col<<<grid, blk, sm, s>>>(g->dgeoms, g->ng, g->total[st], tk, xo));
            break;
    }
    TC_LAUNCHED("grouped pass");
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
    g->ng = n_geoms;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return TC_ERR_CUDA;
    }
    long long xo = 0, yo = 0;
    for (int i = 0; i < n_geoms; ++i) {
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
        xo += (long long)counts[i] * p->k.N * p->k.N;
        yo += (long long)counts[i] * p->k.A * p->k.D;
        g->bytes += p->bytes;
    }
    // work list: largest geometries (by image work) first
    g->order.resize(n_geoms);
    std::iota(g->order.begin(), g->order.end(), 0);
    std::stable_sort(g->order.begin(), g->order.end(), [&](int a, int b) {
        const tc_plan *pa = g->plans[a], *pb = g->plans[b];
        return (long long)pa->k.N * pa->k.N * g->counts[a] > (long long)pb->k.N * pb->k.N * g->counts[b];
    });
    std::vector<GroupGeom> hg(n_geoms);
    int thr_col = 0, thr_row = 0, thr_det = 0;
    size_t sm_col = 0, sm_rowf = 0, sm_rowa = 0, sm_det = 0;
    for (int j = 0; j < n_geoms; ++j) {
        const int i = g->order[j];
        tc_plan *p = g->plans[i];
        GroupGeom &G = hg[j];
        std::memset(&G, 0, sizeof(G));
        G.k = p->k;
        G.tu = p->tu;
        G.pv = p->pv;
        G.sr = p->sr;
        G.part = p->partials;
        G.cp = p->cp_col;
        G.count = g->counts[i];
        G.xoff = g->xoff[i];
        G.yoff = g->yoff[i];
        const int col = p->k.N / (2 * p->cp_col), rows = p->k.R, det = (p->k.A + 1) / 2;
        const int tiles[GS_COUNT] = {col, rows, det, det, rows, col};
        for (int st = 0; st < GS_COUNT; ++st) {
            G.tiles[st] = tiles[st];
            G.start[st] = g->total[st];
            const long long t = (long long)g->total[st] + (long long)tiles[st] * G.count;
            if (t >= (1LL << 31)) {
                group_free(g);
                return TC_ERR_UNSUPPORTED;
            }
            g->total[st] = (int)t;
        }
        thr_col = std::max(thr_col, p->threads_col);
        thr_row = std::max(thr_row, p->threads_row);
        thr_det = std::max(thr_det, p->threads_det);
        sm_col = std::max(sm_col, p->smem_col);
        sm_rowf = std::max(sm_rowf, p->smem_row_fwd);
        sm_rowa = std::max(sm_rowa, p->smem_row_adj);
        sm_det = std::max(sm_det, p->smem_det);
    }
    int rc = TC_OK;
    if (cudaMalloc(&g->dgeoms, sizeof(GroupGeom) * n_geoms) != cudaSuccess ||
        cudaMalloc(&g->dorder, sizeof(int) * n_geoms) != cudaSuccess ||
        cudaMalloc(&g->tickets, sizeof(int) * GS_COUNT) != cudaSuccess) {
        cudaGetLastError();
        group_free(g);
        return TC_ERR_OOM;
    }
    if (cudaMemcpy(g->dgeoms, hg.data(), sizeof(GroupGeom) * n_geoms, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->dorder, g->order.data(), sizeof(int) * n_geoms, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = tc_cuda_fail(cudaGetLastError(), "tc_plan_group_create");
    if (!rc) rc = stage_config(g, GS_FWD_COL, gk_fwd_col, thr_col, sm_col);
    if (!rc) rc = stage_config(g, GS_FWD_ROW, gk_fwd_row, thr_row, sm_rowf);
    if (!rc) rc = stage_config(g, GS_FWD_DET, gk_fwd_det, thr_det, sm_det);
    if (!rc) rc = stage_config(g, GS_ADJ_DET, gk_adj_det, thr_det, sm_det);
    if (!rc) rc = stage_config(g, GS_ADJ_ROW, gk_adj_row, thr_row, sm_rowa);
    if (!rc) rc = stage_config(g, GS_ADJ_COL, gk_adj_col, thr_col, sm_col);
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
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * GS_COUNT, s));
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
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * GS_COUNT, s));
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
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, sizeof(int) * GS_COUNT, s));
    if (obj) TC_CUDA(cudaMemsetAsync(obj, 0, sizeof(double) * 2 * g->ng, s));
    const int mode = DET_RESID | (obj ? DET_OBJ : 0);
    int rc;
    if ((rc = launch_stage(g, GS_FWD_COL, s, x, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_ROW, s, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) ||
        (rc = launch_stage(g, GS_FWD_DET, s, nullptr, nullptr, b, w, mode, nullptr)))
        return rc;
    if (obj) {
        TC_PROFILED(TCK_REDUCE, s, gk_data_finalize<<<g->ng, 256, 0, s>>>(g->dgeoms, g->dorder, obj));
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
