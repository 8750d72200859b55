// qGGMRF prior launches (arXiv 2304.12934, Sec. 3 Eqs. reg2, reg3): the host
// side of the prior kernel in prior_kernel.cuh -- its constants, grid and z
// chunks, and the FP64 reductions of its block partials.
#include "prior_kernel.cuh"

namespace {

PriorArgs make_prior_args(int n, int nb, const tc_prior *pr, double step = 0.0) {
    PriorArgs a;
    a.N = n;
    a.B = nb;
    a.z0 = 0;
    a.z1 = nb;
    a.zc = nb;
    const double p = pr->p, q = 2.0 - p;
    // q = 0 (p = 2): Q = 1/c for every d; a zero difference still gives a
    // zero pair value, which log2|0| times the least normal float keeps finite
    a.ql2 = pack_splat(q > 0.0 ? (float)q : FLT_MIN);
    a.lk2 = pack_splat((float)(-q * std::log2(pr->sigma) - std::log2(pr->c)));
    a.one2 = pack_splat(1.0f);
    const double *w = pr->dims == 3 ? Wts<3>::w : Wts<2>::w;
    for (int c = 0; c < 3; ++c) {
        a.wq2[c] = pack_splat((float)(w[c] * q));
        a.wp2[c] = pack_splat((float)(w[c] * p));
        a.wh2[c] = pack_splat((float)w[c]);
    }
    a.gscale2 = pack_splat((float)(2.0 * pr->lambda / (pr->sigma * pr->sigma * pr->c)));
    a.nstep2 = pack_splat((float)-step);
    a.scal = nullptr;
    return a;
}

// lambda H from the block partials of sum w d^2 i over unordered pairs: every
// pair enters H twice (ordered pairs) and rho = d^2 i / (sigma^2 c).
double prior_value_scale(const tc_prior *pr) { return 2.0 * pr->lambda / (pr->sigma * pr->sigma * pr->c); }

dim3 tile_grid(int n) { return dim3((n + TX - 1) / TX, (n + TY - 1) / TY, 1); }

// z chunks for nb slices: about 128 planes each, or more chunks (down to 32
// planes) where that is needed for 8 waves of CTAs on 152 SMs (a launch over a
// 64-slice slab); at most ZCHUNK_MAX and at most what max_blocks partial sums
// allow
int z_chunks(int n, int nb, int max_blocks) {
    const dim3 t = tile_grid(n);
    const long long tiles = (long long)t.x * t.y, waves8 = 8LL * 152 * MIN_BLOCKS;
    int c = nb / 128;
    const int c_fill = (int)((waves8 + tiles - 1) / tiles), c_cap = nb / 32;
    if (c < c_fill) c = c_fill < c_cap ? c_fill : c_cap;
    c = c < 1 ? 1 : (c > ZCHUNK_MAX ? ZCHUNK_MAX : c);
    while (c > 1 && (long long)c * tiles > max_blocks) --c;
    return c;
}

template <bool H, bool DOTS, bool GRAD, int DIMS, bool EVEN>
void launch_one(dim3 grid, cudaStream_t s, bool profiled, const float *x, float *g, double *ph,
                const PriorArgs &a, float *xp, double *p1, double *p2) {
    if (profiled)
        TC_PROFILED(DOTS ? TCK_PRIOR_NEXT : TCK_PRIOR, s,
                    (k_prior<H, DOTS, GRAD, DIMS, EVEN><<<grid, THREADS, 0, s>>>(x, g, ph, a, xp, p1, p2)));
    else
        k_prior<H, DOTS, GRAD, DIMS, EVEN><<<grid, THREADS, 0, s>>>(x, g, ph, a, xp, p1, p2);
}

// dispatch on (WANT_H, DOTS, DIMS) for the gradient kernels
template <bool EVEN>
void launch_grad(bool h, bool dots, int dims, dim3 grid, cudaStream_t s, bool prof, const float *x, float *g,
                 double *ph, const PriorArgs &a, float *xp, double *p1, double *p2) {
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
                      const tc_prior *pr, double *h_acc, cudaStream_t s, float *dot_x,
                      int z0, int z1, double step) {
    PriorArgs a = make_prior_args(p->k.N, nb, pr, step);
    a.scal = p->scal;
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

// The prior kernels use no dynamic shared memory: nothing to opt into.
int prior_configure_kernels() { return TC_OK; }
