// Per-plan launchers of the NUFFT Radon passes (radon_passes.cuh): one
// launch per pass over a (tile, slice) grid for a chunk of slices of one
// geometry, and the kernels' shared-memory configuration.
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "profile.cuh"
#include "radon_passes.cuh"

int launch_radon_fwd_chunk(tc_plan *p, const float *x, float *y, int nb,
                           const float *b, const float *w, float *resid,
                           double *obj_acc, cudaStream_t s) {
    const KArgs &g = p->k;
    dim3 gc(g.N / (2 * p->cp_col), nb);
    dim3 gr(g.R, nb);
    // the image strips by TMA when the plan allows it and the map encodes
    CUtensorMap tmx;
    std::memset(&tmx, 0, sizeof(tmx));
    const bool use_tma = p->smem_col_tma > 0 &&
                         tma_encode_f32_3d(&tmx, x, g.N, g.N, nb, 2 * p->cp_col, g.N < 256 ? g.N : 256) == TC_OK;
    int rc = with_logn(g.log2N, [&](auto L) {
        constexpr int LG = decltype(L)::value;
        if (use_tma)
            TC_PROFILED(TCK_FWD_COL, s, k_fwd_col<LG, true><<<gc, p->threads_col, p->smem_col_tma, s>>>(
                                            x, p->tu, g, p->cp_col, tmx, p->dev_err));
        else
            TC_PROFILED(TCK_FWD_COL, s, k_fwd_col<LG, false><<<gc, p->threads_col, p->smem_col, s>>>(
                                            x, p->tu, g, p->cp_col, tmx, p->dev_err));
        TC_LAUNCHED("k_fwd_col");
        TC_PROFILED(TCK_FWD_ROW, s, k_fwd_row<LG><<<gr, p->threads_row, p->smem_row_fwd, s>>>(p->tu, p->pv, g));
        TC_LAUNCHED("k_fwd_row");
        return TC_OK;
    });
    if (rc) return rc;
    dim3 gd((g.A + 1) / 2, nb);
    int mode = 0;
    if (y) mode |= DET_WRITE_Y;
    if (resid) mode |= DET_RESID;
    if (resid && obj_acc) mode |= DET_OBJ;
    if (g.blue)
        with_logl(g.log2L, [&](auto L) {
            TC_PROFILED(TCK_FWD_DET, s, k_fwd_det<true, decltype(L)::value><<<gd, p->threads_det, p->smem_det, s>>>(
                                            p->pv, y, b, w, resid, p->partials, g, mode));
        });
    else
        TC_PROFILED(TCK_FWD_DET, s, k_fwd_det<false><<<gd, p->threads_det, p->smem_det, s>>>(p->pv, y, b, w, resid, p->partials, g, mode));
    TC_LAUNCHED("k_fwd_det");
    if (mode & DET_OBJ) {
        rc = launch_reduce_finalize(p->partials, gd.x * gd.y, obj_acc, 1, 1.0, s);
        if (rc) return rc;
    }
    return TC_OK;
}

int launch_radon_adj_chunk(tc_plan *p, const float *y, float *x, int nb,
                           cudaStream_t s) {
    const KArgs &g = p->k;
    dim3 gd((g.A + 1) / 2, nb);
    if (g.blue)
        with_logl(g.log2L, [&](auto L) {
            TC_PROFILED(TCK_ADJ_DET, s, k_adj_det<true, decltype(L)::value><<<gd, p->threads_det, p->smem_det, s>>>(
                                            y, p->pv, g));
        });
    else
        TC_PROFILED(TCK_ADJ_DET, s, k_adj_det<false><<<gd, p->threads_det, p->smem_det, s>>>(y, p->pv, g));
    TC_LAUNCHED("k_adj_det");
    const dim3 gr = TC_ADJ_ROW_SLICES_FASTEST ? dim3(nb, g.R) : dim3(g.R, nb);
    dim3 gc(g.N / (2 * p->cp_col), nb);
    return with_logn(g.log2N, [&](auto L) {
        constexpr int LG = decltype(L)::value;
        TC_PROFILED(TCK_ADJ_ROW, s, k_adj_row<LG><<<gr, p->threads_row, p->smem_row_adj, s>>>(p->pv, p->tu, g));
        TC_LAUNCHED("k_adj_row");
        TC_PROFILED(TCK_ADJ_COL, s, k_adj_col<LG, COL_DEAPOD><<<gc, p->threads_col, p->smem_col, s>>>(
                                        p->tu, x, g, p->cp_col, nullptr, nullptr, nullptr));
        TC_LAUNCHED("k_adj_col");
        return TC_OK;
    });
}

int launch_radon_normal_chunk(tc_plan *p, const float *x, float *out, int nb, const float *sub,
                              const float *xdot, double *obj_acc, cudaStream_t s) {
    const KArgs &kn = p->kn;
    float2 *tu = p->nrm_tu ? p->nrm_tu : p->tu;
    dim3 gc(kn.N / (2 * p->cp_col), nb);
    dim3 gr(nb, kn.R);  // slices fastest: the CTAs in flight share table rows
    CUtensorMap tmx;
    std::memset(&tmx, 0, sizeof(tmx));
    const bool use_tma = p->smem_col_tma > 0 &&
                         tma_encode_f32_3d(&tmx, x, kn.N, kn.N, nb, 2 * p->cp_col, kn.N < 256 ? kn.N : 256) == TC_OK;
    const bool dot = sub && xdot && obj_acc;
    return with_logn(kn.log2N, [&](auto L) {
        constexpr int LG = decltype(L)::value;
        if (use_tma)
            TC_PROFILED(TCK_NRM_COL_FWD, s, k_fwd_col<LG, true><<<gc, p->threads_col, p->smem_col_tma, s>>>(
                                                x, tu, kn, p->cp_col, tmx, p->dev_err));
        else
            TC_PROFILED(TCK_NRM_COL_FWD, s, k_fwd_col<LG, false><<<gc, p->threads_col, p->smem_col, s>>>(
                                                x, tu, kn, p->cp_col, tmx, p->dev_err));
        TC_LAUNCHED("k_fwd_col (normal)");
        TC_PROFILED(TCK_NRM_ROW, s, k_nrm_row<LG><<<gr, p->threads_row, p->smem_row_fwd, s>>>(
                                        tu, p->nrm_t, p->nrm_h, kn));
        TC_LAUNCHED("k_nrm_row");
        if (sub)
            TC_PROFILED(TCK_NRM_COL_ADJ, s, k_adj_col<LG, COL_GRAD><<<gc, p->threads_col, p->smem_col, s>>>(
                                                tu, out, kn, p->cp_col, sub, dot ? xdot : nullptr, p->nrm_part));
        else
            TC_PROFILED(TCK_NRM_COL_ADJ, s, k_adj_col<LG, COL_PLAIN><<<gc, p->threads_col, p->smem_col, s>>>(
                                                tu, out, kn, p->cp_col, nullptr, nullptr, nullptr));
        TC_LAUNCHED("k_adj_col (normal)");
        if (dot) return launch_reduce_finalize(p->nrm_part, (int)(gc.x * gc.y), obj_acc, 1, 0.5, s);
        return TC_OK;
    });
}

// The dynamic shared-memory limit is an attribute of the kernel (process
// wide, per device), shared by every plan: only ever raise it.
template <class F>
int raise_smem_limit(F *fn, size_t bytes) {
    cudaFuncAttributes at;
    TC_CUDA(cudaFuncGetAttributes(&at, fn));
    if ((size_t)at.maxDynamicSharedSizeBytes < bytes)
        TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return TC_OK;
}

int radon_configure_kernels(tc_plan *p) {
    // the column passes may be retuned to up to 4 column pairs per CTA
    size_t col_max = p->smem_col, tma_max = p->smem_col_tma;
    for (int cp = 1; cp <= 4; cp <<= 1) {
        const size_t sm = (size_t)(2 * cp * fft_tstride(p->k.N)) * 8;
        if (sm <= 200 * 1024 && sm > col_max) col_max = sm;
        const size_t st = sm + col_strip_bytes(p->k.N, cp);
        if (cp >= 2 && st <= 200 * 1024 && st > tma_max) tma_max = st;
    }
    int rc = with_logn(p->k.log2N, [&](auto L) {
        constexpr int LG = decltype(L)::value;
        int e;
        if ((e = raise_smem_limit(k_fwd_col<LG, false>, col_max)) ||
            (e = raise_smem_limit(k_adj_col<LG, COL_DEAPOD>, col_max)) ||
            (e = raise_smem_limit(k_adj_col<LG, COL_PLAIN>, col_max)) ||
            (e = raise_smem_limit(k_adj_col<LG, COL_GRAD>, col_max)) ||
            (e = raise_smem_limit(k_nrm_row<LG>, p->smem_row_fwd)) ||
            (p->smem_col_tma && (e = raise_smem_limit(k_fwd_col<LG, true>, tma_max))) ||
            (e = raise_smem_limit(k_fwd_row<LG>, p->smem_row_fwd)) ||
            (e = raise_smem_limit(k_adj_row<LG>, p->smem_row_adj)))
            return e;
        return TC_OK;
    });
    if (rc ||
        (rc = raise_smem_limit(k_fwd_det<true>, p->smem_det)) ||
        (rc = raise_smem_limit(k_adj_det<true>, p->smem_det)) ||
        (rc = raise_smem_limit(k_fwd_det<false>, p->smem_det)) ||
        (rc = raise_smem_limit(k_adj_det<false>, p->smem_det)))
        return rc;
    if (p->k.blue)
        with_logl(p->k.log2L, [&](auto L) {
            constexpr int LL = decltype(L)::value;
            if (!rc) rc = raise_smem_limit(k_fwd_det<true, LL>, p->smem_det);
            if (!rc) rc = raise_smem_limit(k_adj_det<true, LL>, p->smem_det);
        });
    return rc;
}
