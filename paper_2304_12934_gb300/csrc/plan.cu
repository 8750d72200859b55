// Plan construction for the NUFFT Radon operators (host side).
//
// Everything geometric is computed here once, in FP64, and uploaded:
//   * deapodisation factors 1/psi(x), psi the Fourier transform of the
//     spreading kernel (Sec. 2.2 Eq. nufft3's "division by the Fourier
//     transform of the kernel"), by Gauss-Legendre quadrature;
//   * the polar points k = (m/D)(cos theta, sin theta), m = 0..D/2, on the
//     2x oversampled grid g = k G (Sec. 2.2, Fig. gridding), reduced to the
//     upper half plane (theta in [0, pi)) using conj symmetry of real data;
//   * per grid row, the list of (point, tap) pairs whose w x w footprint
//     touches that row, sorted by the point's first column jx0 -- the sorted
//     bins that make spreading a deterministic gather;
//   * twiddle tables and the mixed-radix factorisation of D.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

int radon_configure_kernels(tc_plan *p);
int prior_configure_kernels();

namespace {

const double kPi = 3.14159265358979323846264338327950288;

double es_phi(double z, double beta) {
    const double q = 1.0 - z * z;
    return q > 0.0 ? std::exp(beta * (std::sqrt(q) - 1.0)) : 0.0;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// Odd primes (largest first), then radix 4, then one radix 2.
bool factor_radices(int n, RadixPlan &rp) {
    rp.n = n;
    rp.nrad = 0;
    std::vector<int> odd;
    int m = n, twos = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++twos;
    }
    for (int p = 3; (long long)p * p <= m; p += 2)
        while (m % p == 0) {
            odd.push_back(p);
            m /= p;
        }
    if (m > 1) odd.push_back(m);
    std::sort(odd.rbegin(), odd.rend());
    std::vector<int> r(odd.begin(), odd.end());
    while (twos >= 2) {
        r.push_back(4);
        twos -= 2;
    }
    if (twos) r.push_back(2);
    if ((int)r.size() > TC_MAX_RADICES) return false;
    for (size_t i = 0; i < r.size(); ++i) rp.rad[i] = r[i];
    rp.nrad = (int)r.size();
    return true;
}

// In-place FP64 radix-2 FFT (sign -1) of a power-of-two length, host side.
void fft64(std::vector<double> &re, std::vector<double> &im) {
    const size_t n = re.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * kPi / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const double wr = std::cos(ang * k), wi = std::sin(ang * k);
                const size_t u = i + k, v = i + k + len / 2;
                const double xr = re[v] * wr - im[v] * wi, xi = re[v] * wi + im[v] * wr;
                re[v] = re[u] - xr;
                im[v] = im[u] - xi;
                re[u] += xr;
                im[u] += xi;
            }
    }
}

// Per-stage twiddle tables of a length-2^log2n FFT in the layout fft_pow2
// reads: for each stage after the first, W^(q k n / (Ns R)) at [(q-1) Ns + k].
std::vector<float2> stage_twiddles(int log2n) {
    const int n = 1 << log2n;
    std::vector<float2> out;
    int logNs = 0;
    while (log2n - logNs > 0) {
        const int lr = std::min(4, log2n - logNs);
        const int R = 1 << lr, Ns = 1 << logNs;
        if (logNs > 0)
            for (int q = 1; q < R; ++q)
                for (int k = 0; k < Ns; ++k) {
                    const long long e = (long long)q * k * (n / (Ns * R));
                    const double a = -2.0 * kPi * (double)e / (double)n;
                    out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
                }
        logNs += lr;
    }
    return out;
}

// Largest prime factor of n.
int largest_prime(int n) {
    int lp = 1;
    for (int q = 2; (long long)q * q <= n; ++q)
        while (n % q == 0) {
            lp = q;
            n /= q;
        }
    return n > 1 ? std::max(lp, n) : lp;
}

struct Entry {
    int key, p, s;
    float ex, wy;
};

template <class T>
int upload(T **dst, const std::vector<T> &src, long long &bytes) {
    const size_t nb = src.size() * sizeof(T);
    *dst = nullptr;
    if (nb == 0) return TC_OK;
    cudaError_t e = cudaMalloc((void **)dst, nb);
    if (e != cudaSuccess) return tc_cuda_fail(e, "cudaMalloc(plan table)");
    bytes += (long long)nb;
    TC_CUDA(cudaMemcpy(*dst, src.data(), nb, cudaMemcpyHostToDevice));
    return TC_OK;
}

int alloc_dev(void **dst, size_t nb, long long &bytes) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc(dst, nb ? nb : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TC_ERR_OOM : tc_cuda_fail(e, "cudaMalloc(scratch)");
    }
    bytes += (long long)nb;
    return TC_OK;
}

// Spreading records of one chunk size.  Within each row the key-sorted
// entries are cut into chunks of `chunk`; for every chunk and every signed cell
// cs touched by one of its entries (cs in [key, key + w - 1]), the entries that
// touch cs are those with key in [cs - w + 1, cs]: a contiguous range [lo, hi)
// of the chunk.  A record (cs, lo, hi) lets one thread compute the chunk's
// whole contribution to cell cs mod G.  When two signed cells of a chunk share
// a physical cell (the spectrum edge wraps, cs and cs + G), the later record is
// flagged "seam" and added serially.  Per row, roff holds [start_0, seam_0,
// start_1, seam_1, ..., start_nch]; the seam records of chunk k are
// [seam_k, start_{k+1}), after its regular ones.  Returns nch, the chunks per
// row (the maximum over rows).
int build_spread_records(const std::vector<int> &keys, const std::vector<int> &cnt, int R, int w, int G, int kmin,
                         int chunk, std::vector<int2> &recs, std::vector<int> &roff) {
    recs.clear();
    int nch = 1;
    for (int r = 0; r < R; ++r) nch = std::max(nch, (cnt[r + 1] - cnt[r] + chunk - 1) / chunk);
    roff.assign((size_t)R * (2 * nch + 1), 0);
    std::vector<int> last_use(G, -1);
    std::vector<int2> seams;
    int stamp = 0;
    for (int r = 0; r < R; ++r) {
        const int e0 = cnt[r], e1 = cnt[r + 1];
        for (int kc = 0; kc <= nch; ++kc) {
            int *ro = &roff[(size_t)r * (2 * nch + 1)];
            ro[2 * kc] = (int)recs.size();
            if (kc == nch) continue;
            ro[2 * kc + 1] = (int)recs.size();
            const int c0 = e0 + kc * chunk;
            if (c0 >= e1) continue;
            seams.clear();
            const int n = std::min(chunk, e1 - c0);
            ++stamp;
            // signed cells touched, in increasing order: walk the sorted keys
            int lo = 0, hi = 0;
            int cs = keys[c0];
            const int cs_end = keys[c0 + n - 1] + w - 1;
            while (cs <= cs_end) {
                while (lo < n && keys[c0 + lo] < cs - w + 1) ++lo;
                while (hi < n && keys[c0 + hi] <= cs) ++hi;
                if (hi > lo) {
                    const int cp = cs & (G - 1);
                    const int seam = last_use[cp] == stamp ? 1 : 0;
                    last_use[cp] = stamp;
                    int2 rc;
                    rc.x = (cs - kmin) | (seam << 15);
                    rc.y = lo | (hi << 16);
                    (seam ? seams : recs).push_back(rc);
                    ++cs;
                } else {
                    // no entry touches cs: jump to the next key's window
                    cs = (lo < n) ? std::max(cs + 1, keys[c0 + lo]) : cs_end + 1;
                }
            }
            // longest ranges first: the threads that take them start early
            std::stable_sort(recs.begin() + ro[2 * kc], recs.end(), [](const int2 &u, const int2 &v) {
                return ((u.y >> 16) - (u.y & 0xffff)) > ((v.y >> 16) - (v.y & 0xffff));
            });
            ro[2 * kc + 1] = (int)recs.size();
            recs.insert(recs.end(), seams.begin(), seams.end());
        }
    }
    return nch;
}

}  // namespace

// Entries per spreading chunk: rebuild the record tables for `chunk` (256,
// 512 or 1024) and replace them on the device (synchronous).
int plan_set_spread_chunk(tc_plan *p, int chunk) {
    if (!(chunk == 256 || chunk == 512 || chunk == 1024) || !p->host) return TC_ERR_INVALID_ARG;
    if (chunk == p->k.chunk) return TC_OK;
    KArgs &k = p->k;
    std::vector<int2> recs;
    std::vector<int> roff;
    const int nch = build_spread_records(p->host->keys, p->host->row_off, k.R, k.w, k.G, k.kmin, chunk, recs, roff);
    int2 *nrec = nullptr;
    int *nroff = nullptr;
    long long bytes = 0;
    int rc = upload(&nrec, recs, bytes);
    if (!rc) rc = upload(&nroff, roff, bytes);
    if (rc) {
        if (nrec) cudaFree(nrec);
        return rc;
    }
    TC_CUDA(cudaDeviceSynchronize());  // no launch may still read the old tables
    const long long old = (long long)((size_t)p->host->n_rec * sizeof(int2) + (size_t)p->host->n_roff * sizeof(int));
    cudaFree(p->rec);
    cudaFree(p->rec_off);
    p->rec = nrec;
    p->rec_off = nroff;
    p->bytes += bytes - old;
    p->host->n_rec = recs.size();
    p->host->n_roff = roff.size();
    k.rec = nrec;
    k.rec_off = nroff;
    k.nch = nch;
    k.chunk = chunk;
    p->smem_row_adj = p->smem_row_fwd + (size_t)chunk * sizeof(float4);
    return radon_configure_kernels(p);
}

// Column pairs per CTA of the column passes: threads, shared memory (the
// kernels' dynamic-smem limit is raised to the largest candidate at build).
int plan_set_col_pairs(tc_plan *p, int cp) {
    const int N = p->k.N;
    if (cp < 1 || cp > 4 || 2 * cp > N || 2 * cp * N / 16 > 512) return TC_ERR_INVALID_ARG;
    const size_t smem = (size_t)(2 * cp * fft_tstride(N)) * sizeof(float2);
    if (smem > 200 * 1024) return TC_ERR_INVALID_ARG;
    p->cp_col = cp;
    p->threads_col = std::max(64, 2 * cp * N / 16);
    p->smem_col = smem;
    // TMA staging of the image strip needs rows of >= 16 bytes (cp >= 2)
    p->smem_col_tma = cp >= 2 ? smem + col_strip_bytes(N, cp) : 0;
    if (p->smem_col_tma > 200 * 1024) p->smem_col_tma = 0;
    return TC_OK;
}

void tc_plan_free(tc_plan *p) {
    if (!p) return;
    void *ptrs[] = {p->dea64, p->dea, p->twN, p->twG, p->twD, p->row_off, p->ent, p->rec, p->rec_off,
                    p->tu, p->pv, p->sr, p->partials, p->scal, p->dev_err, p->angle_flip, p->shiftD,
                    p->chirp, p->bhat, p->twL, p->cs64, p->nrm_t, p->nrm_h, p->nrm_one, p->nrm_tu,
                    p->nrm_part};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p->host;
    delete p;
}

int tc_plan_build(const tc_geom *geom, int max_batch, tc_plan **out) {
    const int N = geom->n, A = geom->n_angles, D = geom->n_det, w = geom->kernel_width;
    tc_plan *p = new tc_plan();
    std::memset(p, 0, sizeof(*p));
    *out = nullptr;
    TC_CUDA(cudaGetDevice(&p->device));
    p->max_batch = max_batch;
    KArgs &k = p->k;
    k.N = N;
    k.log2N = ilog2(N);
    k.G = 2 * N;
    k.A = A;
    k.D = D;
    k.Mh = D / 2 + 1;
    k.AM = A * k.Mh;
    k.w = w;
    const double h = 0.5 * w;
    const double beta = 2.30 * w;  // ES shape parameter for sigma = 2 (Barnett et al. 2019)
    k.beta = (float)beta;
    k.beta_l2 = (float)(beta / std::log(2.0));
    k.inv_h = (float)(1.0 / h);
    k.invD = (float)(1.0 / D);
    if (!factor_radices(D, k.rp)) {
        tc_plan_free(p);
        return TC_ERR_UNSUPPORTED;
    }
    const int G = k.G;

    // angles reduced to [0, pi); a flipped angle uses conj symmetry of real data
    std::vector<double> th(A), cs64(2 * (size_t)A);
    std::vector<unsigned char> flip(A, 0);
    for (int a = 0; a < A; ++a) {
        double t = geom->angles ? geom->angles[a] : a * kPi / A;
        if (!std::isfinite(t)) {
            tc_plan_free(p);
            return TC_ERR_INVALID_ARG;
        }
        cs64[2 * a] = std::cos(t);  // the angle as given (normal-operator tables)
        cs64[2 * a + 1] = std::sin(t);
        t = std::fmod(t, 2.0 * kPi);
        if (t < 0.0) t += 2.0 * kPi;
        if (t >= kPi) {
            t -= kPi;
            flip[a] = 1;
        }
        th[a] = t;
    }

    // deapodisation: psi(x) = int_{-h}^{h} phi(u/h) cos(2 pi u x / G) du
    std::vector<double> gx, gw;
    gauss_legendre(4 * w + 48, gx, gw);
    std::vector<double> dea64(N);
    std::vector<float> dea(N);
    for (int i = 0; i < N; ++i) {
        const double xv = i - N / 2;
        double s = 0.0;
        for (size_t q = 0; q < gx.size(); ++q) {
            const double u = gx[q] * h;
            s += gw[q] * h * es_phi(gx[q], beta) * std::cos(2.0 * kPi * u * xv / G);
        }
        dea64[i] = 1.0 / s;
        dea[i] = (float)dea64[i];
    }

    // polar points and per-row entries
    const int Mh = k.Mh;
    const long long npts = (long long)A * Mh;
    std::vector<int> jx0(npts), jy0(npts);
    std::vector<double> exv(npts), eyv(npts);
    int jymin = 1 << 30, jymax = -(1 << 30), kmin = 1 << 30, kmax = -(1 << 30);
    for (int a = 0; a < A; ++a) {
        const double c = std::cos(th[a]), s = std::sin(th[a]);
        for (int m = 0; m < Mh; ++m) {
            const long long pidx = (long long)a * Mh + m;
            const double r = (double)m * G / D;
            const double gxv = r * c, gyv = r * s;
            const int x0 = (int)std::floor(gxv - h) + 1;
            const int y0 = (int)std::floor(gyv - h) + 1;
            jx0[pidx] = x0;
            jy0[pidx] = y0;
            exv[pidx] = gxv - x0;
            eyv[pidx] = gyv - y0;
            jymin = std::min(jymin, y0);
            jymax = std::max(jymax, y0 + w - 1);
            kmin = std::min(kmin, x0);
            kmax = std::max(kmax, x0);
        }
    }
    k.jmin = (int)std::floor(-h) + 1;
    k.jmax = (int)std::floor(N - h) + w;
    if (jymin < k.jmin || jymax > k.jmax || k.jmax - k.jmin + 1 > G) {
        tc_plan_free(p);
        return TC_ERR_INVALID_ARG;
    }
    k.R = k.jmax - k.jmin + 1;
    k.kmin = kmin;
    k.kmax = kmax;
    const int R = k.R;
    std::vector<int> cnt(R + 1, 0);
    for (long long q = 0; q < npts; ++q)
        for (int s = 0; s < w; ++s) cnt[jy0[q] + s - k.jmin + 1]++;
    for (int r = 0; r < R; ++r) cnt[r + 1] += cnt[r];
    std::vector<Entry> ents((size_t)cnt[R]);
    std::vector<int> fillp(cnt.begin(), cnt.end() - 1);
    for (long long q = 0; q < npts; ++q)
        for (int s = 0; s < w; ++s) {
            const int r = jy0[q] + s - k.jmin;
            Entry &e = ents[fillp[r]++];
            e.key = jx0[q];
            e.p = (int)q;
            e.s = s;
            e.ex = (float)exv[q];
            e.wy = (float)es_phi((s - eyv[q]) / h, beta);
        }
    for (int r = 0; r < R; ++r)
        std::sort(ents.begin() + cnt[r], ents.begin() + cnt[r + 1],
                  [](const Entry &u, const Entry &v) { return u.key != v.key ? u.key < v.key : u.p < v.p; });
    const size_t E = ents.size();
    std::vector<int4> epk(E);
    for (size_t i = 0; i < E; ++i) {
        int4 v;
        v.x = ents[i].p;
        std::memcpy(&v.y, &ents[i].ex, 4);
        std::memcpy(&v.z, &ents[i].wy, 4);
        v.w = (int)((unsigned)(unsigned short)(short)ents[i].key | ((unsigned)ents[i].s << 16));
        epk[i] = v;
    }
    p->n_entries = (long long)E;

    // spreading records for the default chunk; the entry keys and row offsets
    // stay on the host so the chunk can be changed later (tc_plan_set_spread_chunk)
    p->host = new PlanHost();
    p->host->keys.resize(E);
    for (size_t i = 0; i < E; ++i) p->host->keys[i] = ents[i].key;
    p->host->row_off = cnt;
    if ((long long)kmax + w - 1 - kmin >= (1 << 15)) {
        tc_plan_free(p);
        return TC_ERR_UNSUPPORTED;
    }
    std::vector<int2> recs;
    std::vector<int> roff;
    k.chunk = TC_SPREAD_CHUNK_DEFAULT;
    k.nch = build_spread_records(p->host->keys, cnt, R, w, G, kmin, k.chunk, recs, roff);

    // Bluestein tables when D has a large prime factor (and L stays <= 8192)
    std::vector<float2> chirp, bhat, twL;
    {
        int L = 1, lg = 0;
        while (L < 2 * D - 1) {
            L <<= 1;
            ++lg;
        }
        k.blue = (largest_prime(D) > 32 && L <= 8192) ? 1 : 0;
        k.L = L;
        k.log2L = lg;
        if (k.blue) {
            chirp.resize(D);
            std::vector<double> br(L, 0.0), bi(L, 0.0);
            for (int n = 0; n < D; ++n) {
                const long long q = ((long long)n * n) % (2LL * D);
                const double a = -kPi * (double)q / (double)D;
                chirp[n] = make_float2((float)std::cos(a), (float)std::sin(a));
                // b_m = conj(chirp_|m|) at m and L - m
                br[n] = std::cos(a);
                bi[n] = -std::sin(a);
                if (n > 0) {
                    br[L - n] = std::cos(a);
                    bi[L - n] = -std::sin(a);
                }
            }
            fft64(br, bi);
            bhat.resize(L);
            for (int i = 0; i < L; ++i) bhat[i] = make_float2((float)(br[i] / L), (float)(bi[i] / L));
            twL = stage_twiddles(lg);
            if ((int)twL.size() != fft_twiddle_count(lg)) {
                tc_plan_free(p);
                return TC_ERR_UNSUPPORTED;
            }
        }
    }

    // twiddles
    std::vector<float2> twN = stage_twiddles(k.log2N), twG(N), twD(D);
    k.ntwN = (int)twN.size();
    if (k.ntwN != fft_twiddle_count(k.log2N)) {
        tc_plan_free(p);
        return TC_ERR_UNSUPPORTED;
    }
    for (int i = 0; i < N; ++i) {
        const double a2 = -2.0 * kPi * (i - N / 2) / G;
        twG[i] = make_float2((float)std::cos(a2), (float)std::sin(a2));
    }
    for (int i = 0; i < D; ++i) {
        const double a3 = -2.0 * kPi * i / D;
        twD[i] = make_float2((float)std::cos(a3), (float)std::sin(a3));
    }
    // rotation-axis offset: exp(-2 pi i m delta / D), the phase reduced in FP64
    const double delta = geom->center_offset;
    std::vector<float2> shiftD;
    if (delta != 0.0) {
        shiftD.resize(k.Mh);
        for (int m = 0; m < k.Mh; ++m) {
            double cyc = std::fmod((double)m * delta, (double)D) / D;
            const double a4 = -2.0 * kPi * cyc;
            shiftD[m] = make_float2((float)std::cos(a4), (float)std::sin(a4));
        }
    }

    long long bytes = 0;
    int rc = TC_OK;
#define UP(dst, src)                              \
    if ((rc = upload(&(dst), (src), bytes))) {    \
        tc_plan_free(p);                          \
        return rc;                                \
    }
    UP(p->dea64, dea64);
    UP(p->dea, dea);
    UP(p->twN, twN);
    UP(p->twG, twG);
    UP(p->twD, twD);
    UP(p->row_off, cnt);
    UP(p->ent, epk);
    UP(p->rec, recs);
    UP(p->rec_off, roff);
    p->host->n_rec = recs.size();
    p->host->n_roff = roff.size();
    UP(p->angle_flip, flip);
    UP(p->shiftD, shiftD);
    UP(p->chirp, chirp);
    UP(p->bhat, bhat);
    UP(p->twL, twL);
    UP(p->cs64, cs64);
#undef UP
    p->delta = delta;
    k.dea = p->dea;
    k.twN = p->twN;
    k.twG = p->twG;
    k.twD = p->twD;
    k.row_off = p->row_off;
    k.ent = p->ent;
    k.rec = p->rec;
    k.rec_off = p->rec_off;
    k.angle_flip = p->angle_flip;
    k.shiftD = p->shiftD;
    k.chirp = p->chirp;
    k.bhat = p->bhat;
    k.twL = p->twL;

    // launch configuration (column pairs per CTA may be retuned by tc_plan_autotune)
    int cp = 4;
    while (cp > 1 && (cp * 2 * N * 8 > 96 * 1024 || 2 * cp * N / 16 > 512 || 2 * cp > N)) cp >>= 1;
    p->chunk = max_batch;
    if (plan_set_col_pairs(p, cp)) {
        tc_plan_free(p);
        return TC_ERR_UNSUPPORTED;
    }
    p->threads_row = std::max(128, N / 8);
    p->threads_det = k.blue ? std::max(256, k.L / 16) : 256;
    p->smem_row_fwd = (size_t)(2 * fft_tstride(N)) * sizeof(float2);
    p->smem_row_adj = p->smem_row_fwd + (size_t)k.chunk * sizeof(float4);
    p->smem_det = k.blue ? (size_t)spad_size(k.L) * sizeof(float2)
                         : (size_t)(3 * D + k.rp.rad[0]) * sizeof(float2);
    if (p->threads_row > 512 || p->smem_det > 200 * 1024 || p->smem_row_adj > 200 * 1024) {
        tc_plan_free(p);
        return TC_ERR_UNSUPPORTED;
    }

    // scratch
    const size_t MB = (size_t)max_batch;
    p->slot = std::max(std::max(TC_RED_BLOCKS, (int)(((A + 1) / 2) * MB)),
                       prior_block_slots(N));
    if ((rc = alloc_dev((void **)&p->tu, MB * R * N * sizeof(float2), bytes)) ||
        (rc = alloc_dev((void **)&p->pv, MB * w * (size_t)k.AM * sizeof(float2), bytes)) ||
        (rc = alloc_dev((void **)&p->sr, MB * (size_t)A * D * sizeof(float), bytes)) ||
        (rc = alloc_dev((void **)&p->partials, (size_t)TC_N_SLOTS * p->slot * sizeof(double), bytes)) ||
        (rc = alloc_dev((void **)&p->scal, SC_COUNT * sizeof(double), bytes)) ||
        (rc = alloc_dev((void **)&p->dev_err, sizeof(int), bytes))) {
        tc_plan_free(p);
        return rc;
    }
    TC_CUDA(cudaMemset(p->scal, 0, SC_COUNT * sizeof(double)));
    TC_CUDA(cudaMemset(p->dev_err, 0, sizeof(int)));
    p->bytes = bytes;
    if ((rc = radon_configure_kernels(p)) || (rc = prior_configure_kernels())) {
        tc_plan_free(p);
        return rc;
    }
    *out = p;
    return TC_OK;
}
