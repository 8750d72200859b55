// Batches of slices with uneven geometry (image side, angle count, detector
// width): one launch per pipeline stage and geometry class over a work list.
//
// A plan group holds one plan per geometry, sized for all of that geometry's
// slices.  Per stage, the geometries fall into classes that share a launch
// shape: the image side for the column and row passes, the detector transform
// (Bluestein length, or mixed radix) for the detector passes.  Each class
// (up to GK_MAXG geometries) runs as one launch whose work list is every
// (geometry, slice, tile) item of the class -- column strips, grid rows or
// angle pairs -- largest geometry first; CTA i runs item i, and the GPU's
// block scheduler hands the items out in list order as SMs free up, so the
// small geometries fill the tail of the large ones.  The geometries travel in
// the launch's parameter block and a switch picks the item's one, so every
// pass body reads its geometry from the constant bank at a fixed offset, as
// the per-plan kernels do.  (A software work queue -- CTAs looping over
// tickets -- made the compiler keep each body's geometry-derived values live
// across items: 600 to 2,500 bytes of register spills per thread at the
// per-plan kernels' occupancy, where one item per CTA needs 44 registers.)
// The class launches of one stage touch disjoint geometries, so they run side
// by side on the group's streams (forked from the caller's stream by an event
// and joined back before the next stage), as do the per-geometry prior
// launches; the small geometries' launches then fill the SMs that the large
// ones leave idle in their tails.  Stage boundaries are kernel boundaries: no
// CTA ever waits for another.
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

// One class launch: its geometries and the first item of each.
constexpr int GK_MAXG = 4;
constexpr int GK_SIDE = 7;   // side streams of a group (besides the caller's)
struct ClassParams {
    int ng;                    // geometries of this launch (1..GK_MAXG)
    int starts[GK_MAXG + 1];   // first item of each geometry; starts[ng] = items of the launch
    GroupGeom geo[GK_MAXG];
};

// Item blockIdx.x of the launch: f(G, tile, slice) with G the item's
// geometry, chosen by a switch so each branch reads its geometry at a fixed
// parameter offset.
template <class F>
__device__ __forceinline__ void run_item(const ClassParams &cp, int stage, F &&f) {
    const int item = blockIdx.x;
    int pos = 0;
    while (pos + 1 < cp.ng && item >= cp.starts[pos + 1]) ++pos;
    const int local = item - cp.starts[pos];
    auto go = [&](const GroupGeom &G) { f(G, local % G.tiles[stage], local / G.tiles[stage]); };
    switch (pos) {
        case 0: go(cp.geo[0]); break;
        case 1: go(cp.geo[1]); break;
        case 2: go(cp.geo[2]); break;
        default: go(cp.geo[3]); break;
    }
}
static_assert(GK_MAXG == 4, "run_item's switch covers GK_MAXG geometries");

// launch bounds as the per-plan kernels of the same passes
template <int LOGN>
__global__ void __launch_bounds__(512) gk_fwd_col(const __grid_constant__ ClassParams cp, const float *__restrict__ x) {
    run_item(cp, GS_FWD_COL, [&](const GroupGeom &G, int t, int b) {
        fwd_col_body<LOGN, false>(x + G.xoff, G.tu, G.k, G.cp, nullptr, nullptr, t, b);
    });
}

template <int LOGN>
__global__ void __launch_bounds__(LOGN == 11 ? 256 : 512, LOGN == 11 ? 5 : 1)
    gk_fwd_row(const __grid_constant__ ClassParams cp) {
    run_item(cp, GS_FWD_ROW, [&](const GroupGeom &G, int t, int b) { fwd_row_body<LOGN>(G.tu, G.pv, G.k, t, b); });
}

// y (sinograms out, may be null), bs and ws (may be null): mode as k_fwd_det
template <bool BLUE, int LOGL>
__global__ void __launch_bounds__(512, 2) gk_fwd_det(const __grid_constant__ ClassParams cp, float *__restrict__ y,
                                                  const float *__restrict__ bs, const float *__restrict__ ws,
                                                  int mode) {
    run_item(cp, GS_FWD_DET, [&](const GroupGeom &G, int t, int b) {
        fwd_det_body<BLUE, LOGL>(G.pv, y ? y + G.yoff : nullptr, bs ? bs + G.yoff : nullptr,
                                 ws ? ws + G.yoff : nullptr, G.sr, G.part, G.k, mode, t, b, G.tiles[GS_FWD_DET]);
    });
}

// the adjoint's input: y (concatenated sinograms), or each geometry's residual when y is null
template <bool BLUE, int LOGL>
__global__ void __launch_bounds__(512, 2) gk_adj_det(const __grid_constant__ ClassParams cp, const float *__restrict__ y) {
    run_item(cp, GS_ADJ_DET, [&](const GroupGeom &G, int t, int b) {
        adj_det_body<BLUE, LOGL>(y ? y + G.yoff : G.sr, G.pv, G.k, t, b);
    });
}

template <int LOGN>
__global__ void __launch_bounds__(512) gk_adj_row(const __grid_constant__ ClassParams cp) {
    run_item(cp, GS_ADJ_ROW, [&](const GroupGeom &G, int t, int b) { adj_row_body<LOGN>(G.pv, G.tu, G.k, t, b); });
}

template <int LOGN>
__global__ void __launch_bounds__(512) gk_adj_col(const __grid_constant__ ClassParams cp, float *__restrict__ x) {
    run_item(cp, GS_ADJ_COL, [&](const GroupGeom &G, int t, int b) {
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

// One launch: up to GK_MAXG geometries of one class of one stage, one CTA per item.
struct ClassLaunch {
    int stage;
    int key;        // log2 N (column / row passes); Bluestein log2 L, 0 run-time L, -1 mixed radix (detector)
    int items;
    int grid, threads;
    size_t smem;
    ClassParams par;
};

struct tc_plan_group {
    int device = 0, ng = 0;
    std::vector<tc_plan *> plans;    // caller's order
    std::vector<int> counts;
    std::vector<long long> xoff, yoff;
    GroupGeom *dgeoms = nullptr;     // caller's order
    std::vector<ClassLaunch> launches;
    long long bytes = 0;
    // the class launches of one stage, and the per-geometry prior launches,
    // are independent: they run side by side on these streams, forked from
    // and joined back into the caller's stream with events (so a captured
    // call stays one graph)
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

namespace {

void group_free(tc_plan_group *g) {
    if (!g) return;
    for (cudaStream_t q : g->side)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : g->join)
        if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    for (tc_plan *p : g->plans) tc_plan_free(p);
    for (void *q : {(void *)g->dgeoms})
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

// A class launch's shared-memory opt-in (raise only: the limit is a
// process-wide attribute of the kernel).
int class_config(ClassLaunch &c) {
    return with_class_kernel(c.stage, c.key, [&](auto *kern) -> int {
        cudaFuncAttributes at;
        TC_CUDA(cudaFuncGetAttributes(&at, kern));
        if ((size_t)at.maxDynamicSharedSizeBytes < c.smem)
            TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem));
        c.grid = c.items;
        return TC_OK;
    });
}

// Runs every class launch of one stage (x: images in; y: sinograms in or
// out; b, w, mode: the forward detector pass's epilogue; xo: images out).
// Runs f(q, j) for j = 0..n-1, the first on s and the others on the group's
// side streams (round robin), each side stream forked from s before and
// joined into s after.
template <class F>
int fan_out(tc_plan_group *g, cudaStream_t s, int n, F &&f) {
    const int ns = (int)g->side.size();
    if (n <= 1 || ns == 0) {
        for (int j = 0; j < n; ++j) {
            const int rc = f(s, j);
            if (rc) return rc;
        }
        return TC_OK;
    }
    const int used = n - 1 < ns ? n - 1 : ns;
    TC_CUDA(cudaEventRecord(g->fork, s));
    for (int k = 0; k < used; ++k) TC_CUDA(cudaStreamWaitEvent(g->side[k], g->fork, 0));
    int rc = TC_OK;
    for (int j = 0; j < n && !rc; ++j) rc = f(j == 0 ? s : g->side[(j - 1) % ns], j);
    // join even after a failed launch, so no side stream is left forked
    for (int k = 0; k < used; ++k) {
        TC_CUDA(cudaEventRecord(g->join[k], g->side[k]));
        TC_CUDA(cudaStreamWaitEvent(s, g->join[k], 0));
    }
    return rc;
}

int launch_stage(tc_plan_group *g, int st, cudaStream_t s0, const float *x, float *y, const float *b,
                 const float *w, int mode, float *xo) {
    std::vector<int> mine;
    for (size_t li = 0; li < g->launches.size(); ++li)
        if (g->launches[li].stage == st) mine.push_back((int)li);
    return fan_out(g, s0, (int)mine.size(), [&](cudaStream_t s, int j) -> int {
        const ClassLaunch &c = g->launches[mine[j]];
        const dim3 grid(c.grid), blk(c.threads);
        const size_t sm = c.smem;
#define GK_PASS c.par
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
        return TC_OK;
    });
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
    // per stage: geometries grouped by class, largest first; one launch per
    // class (per GK_MAXG geometries of a class)
    for (int st = 0; st < GS_COUNT; ++st) {
        const bool det = st == GS_FWD_DET || st == GS_ADJ_DET;
        auto key = [&](int i) { return det ? det_key(g->plans[i]->k) : g->plans[i]->k.log2N; };
        auto cost = [&](int i) { return (long long)hg[i].tiles[st] * hg[i].count; };
        std::vector<int> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
            return key(a) != key(b) ? key(a) < key(b) : cost(a) > cost(b);
        });
        for (int p0 = 0; p0 < n;) {
            ClassLaunch c{};
            c.stage = st;
            c.key = key(ord[p0]);
            long long item = 0;
            int p1 = p0;
            while (p1 < n && key(ord[p1]) == c.key && c.par.ng < GK_MAXG) {
                const int i = ord[p1];
                const tc_plan *p = g->plans[i];
                c.par.starts[c.par.ng] = (int)item;
                c.par.geo[c.par.ng++] = hg[i];
                item += cost(i);
                if (item >= (1LL << 31)) {
                    group_free(g);
                    return TC_ERR_UNSUPPORTED;
                }
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
            c.par.starts[c.par.ng] = (int)item;
            c.items = (int)item;
            if (c.items > 0) g->launches.push_back(c);
            p0 = p1;
        }
    }
    int rc = TC_OK;
    if (cudaMalloc(&g->dgeoms, sizeof(GroupGeom) * n) != cudaSuccess) {
        cudaGetLastError();
        group_free(g);
        return TC_ERR_OOM;
    }
    if (cudaMemcpy(g->dgeoms, hg.data(), sizeof(GroupGeom) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = tc_cuda_fail(cudaGetLastError(), "tc_plan_group_create");
    for (ClassLaunch &c : g->launches)
        if (!rc) rc = class_config(c);
    // side streams: as many as the widest stage (or the geometries, for the
    // priors) needs beyond the caller's stream, at most GK_SIDE
    int width = n;
    for (int st = 0; st < GS_COUNT; ++st) {
        int k = 0;
        for (const ClassLaunch &c : g->launches) k += c.stage == st;
        width = std::max(width, k);
    }
    const int nside = std::min(width - 1, GK_SIDE);
    if (!rc && nside > 0) {
        if (cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) rc = TC_ERR_CUDA;
        for (int k = 0; k < nside && !rc; ++k) {
            cudaStream_t q = nullptr;
            cudaEvent_t e = nullptr;
            if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) {
                rc = TC_ERR_CUDA;
                break;
            }
            g->side.push_back(q);
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                rc = TC_ERR_CUDA;
                break;
            }
            g->join.push_back(e);
        }
        if (rc) cudaGetLastError();
    }
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
        // one prior launch (and its value reduction) per geometry, side by side
        rc = fan_out(g, s, g->ng, [&](cudaStream_t q, int i) -> int {
            tc_plan *p = g->plans[i];
            return launch_prior_grad(p, x + g->xoff[i], grad + g->xoff[i], g->counts[i], prior,
                                     obj ? obj + 2 * i + 1 : nullptr, q);
        });
        if (rc) return rc;
    }
    return TC_OK;
}

}  // extern "C"
