// Plans, shared tables and the C ABI of the spectral-transform library.
//
// The transform, its steps and the on-device transposition are described in
// include/st.h.  The host side here computes:
//   - the grid rings;
//   - the Gauss-Legendre nodes, by Newton iteration in the colatitude, so
//     that sin(theta) and the polar weights keep full relative precision;
//   - the per-m ring ranges and the Bluestein chirps;
//   - the CTA work lists.
// The Legendre tables and the Bluestein filters are built on the device.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "st_internal.cuh"

namespace st {

static thread_local char g_err[512];

// allocation failure injection: the n-th dev_malloc from the arming call fails
static std::atomic<int> g_fail_alloc{0};

cudaError_t dev_malloc(void** p, size_t bytes)
{
    if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------ Gauss nodes
// Nodes of P_nlat in colatitude: theta <- theta + P(cos t)/(sin t P'(cos t)).
// Weights 2 / (sin^2(theta) P'(mu)^2) with P' from the derivative identity.
static void gauss_colatitude(int nlat, std::vector<double>& mu, std::vector<double>& w,
                             std::vector<double>& sinth, std::vector<double>& th_hi, std::vector<double>& th_lo)
{
    mu.assign(nlat, 0.0);
    w.assign(nlat, 0.0);
    sinth.assign(nlat, 0.0);
    th_hi.assign((nlat + 1) / 2, 0.0);
    th_lo.assign((nlat + 1) / 2, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < (nlat + 1) / 2; k++) {
        long double th = pi * (k + 0.75L) / (nlat + 0.5L);
        long double dpdmu = 0;
        for (int it = 0; it < 60; it++) {
            long double x = cosl(th), s = sinl(th);
            long double p0 = 1, p1 = x;
            for (int j = 1; j < nlat; j++) {
                long double p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
                p0 = p1;
                p1 = p2;
            }
            // P'(x) = n (P_{n-1} - x P_n) / (1 - x^2)
            dpdmu = nlat * (p0 - x * p1) / (s * s);
            long double dth = p1 / (s * dpdmu);
            th += dth;
            if (fabsl(dth) < 1e-19L) break;
        }
        long double s = sinl(th);
        if (2 * k + 1 == nlat) th = pi / 2, s = 1;
        long double wk = 2.0L / (s * s * dpdmu * dpdmu);
        th_hi[k] = (double)th;
        th_lo[k] = (double)(th - (long double)th_hi[k]);
        mu[k] = (double)cosl(th);
        if (2 * k + 1 == nlat) mu[k] = 0.0;
        mu[nlat - 1 - k] = -mu[k];
        w[k] = w[nlat - 1 - k] = (double)wk;
        sinth[k] = sinth[nlat - 1 - k] = (double)s;
    }
}

// ------------------------------------------------------------ shared tables
static std::mutex g_tab_mu;
static std::vector<Tables*> g_tabs;

template <typename X>
static int upload(X** d, const std::vector<X>& h)
{
    size_t n = std::max<size_t>(h.size(), 1);
    if (dev_malloc((void**)d, n * sizeof(X)) != cudaSuccess) return ST_ERR_NOMEM;
    if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice) != cudaSuccess)
        return ST_ERR_CUDA;
    return ST_OK;
}

// eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)) in long double
static long double epsl(long double n, long double m) { return sqrtl((n * n - m * m) / (4 * n * n - 1)); }

static void tables_free(Tables* t)
{
    void* ptrs[] = {t->d_nlon, t->d_mmax, t->d_k0, t->d_L, t->d_Lp, t->d_logM, t->d_roff,
                    t->d_foff, t->d_toff, t->d_aoff, t->d_goff, t->d_choff, t->d_floff, t->d_coslat,
                    t->d_w, t->d_mu, t->d_eps, t->d_sc64, t->d_sc32, t->d_bc, t->d_hc, t->d_bc32, t->d_hc32, t->d_poff, t->d_ptab, t->d_fac, t->d_gtab, t->d_ptab32, t->d_gtab32, t->d_fac32, t->d_pw1, t->P64, t->P32, t->Phi, t->Plo, t->Plo2, t->chirp64, t->filt64, t->tw64,
                    t->chirp32, t->filt32, t->tw32, t->tmaps, t->d_Q, t->d_reps, t->ckpt, t->d_ckoff};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete t;
}

static int tables_build_geometry(Tables* t)
{
    const int T = t->T, N = t->N, nlat = 2 * N;
    t->nlat = nlat;
    std::vector<double> sinth;
    gauss_colatitude(nlat, t->mu, t->w, sinth, t->theta_hi, t->theta_lo);
    t->coslat = sinth;  // cos(latitude) = sin(colatitude)
    t->nlon.resize(nlat);
    t->mmax.resize(nlat);
    t->roff.resize(nlat + 1);
    t->foff.resize(nlat + 1);
    t->roff[0] = t->foff[0] = 0;
    for (int k = 0; k < nlat; k++) {
        int i = k < N ? k + 1 : nlat - k;
        int nl = t->kind == ST_GRID_OCTAHEDRAL ? 4 * i + 16 : 4 * N;
        t->nlon[k] = nl;
        t->mmax[k] = std::min(T, nl / 2 - 1);
        t->roff[k + 1] = t->roff[k] + nl;
        t->foff[k + 1] = t->foff[k] + t->mmax[k] + 1;
    }
    t->npts = t->roff[nlat];
    t->nfour_rows = t->foff[nlat];
    // per m: northern rings carrying m, Legendre block sizes (n = m..T+1)
    t->k0.resize(T + 1);
    t->L.resize(T + 1);
    t->Lp.resize(T + 1);
    t->K.resize(2 * (T + 1));
    t->toff.resize(2 * (T + 1) + 1);
    t->aoff.resize(2 * (T + 1) + 1);
    t->goff.resize(2 * (T + 1) + 1);
    t->toff[0] = t->aoff[0] = t->goff[0] = 0;
    for (int m = 0; m <= T; m++) {
        int k0 = 0;
        while (k0 < N && t->mmax[k0] < m) k0++;
        t->k0[m] = k0;
        t->L[m] = N - k0;
        t->Lp[m] = (int)round_up(t->L[m], 8);
        int Kt = T + 2 - m;
        for (int p = 0; p < 2; p++) {
            int K = p == 0 ? (Kt + 1) / 2 : Kt / 2;
            int b = 2 * m + p;
            t->K[b] = K;
            t->toff[b + 1] = t->toff[b] + (long)K * t->Lp[m];
            t->aoff[b + 1] = t->aoff[b] + K;
            t->goff[b + 1] = t->goff[b] + t->L[m];
        }
    }
    t->ntab = t->toff[2 * (T + 1)];
    t->nops_rows = t->aoff[2 * (T + 1)];
    t->ngop_rows = t->goff[2 * (T + 1)];
    // chirp-z plans: one per ring pair (north ring k and its mirror)
    t->logM.resize(N);
    t->choff.resize(N);
    t->floff.resize(N);
    long ch = 0, fl = 0;
    int Mmax = 32;
    for (int k = 0; k < N; k++) {
        const int lm = fft_log_len(t->nlon[k], t->mmax[k] + 1);
        t->logM[k] = lm;
        t->choff[k] = ch;
        t->floff[k] = fl;
        ch += t->nlon[k] / 2 + 1;
        fl += 1L << lm;
        Mmax = std::max(Mmax, 1 << lm);
    }
    t->nchirp = ch;
    t->nfilt = fl;
    t->Mmax = Mmax;
    return ST_OK;
}

static int tables_upload(Tables* t)
{
    int rc = ST_OK;
    std::vector<double> mu = t->mu;
    rc |= upload(&t->d_nlon, t->nlon);
    rc |= upload(&t->d_mmax, t->mmax);
    rc |= upload(&t->d_k0, t->k0);
    rc |= upload(&t->d_L, t->L);
    rc |= upload(&t->d_Lp, t->Lp);
    rc |= upload(&t->d_logM, t->logM);
    rc |= upload(&t->d_roff, t->roff);
    rc |= upload(&t->d_foff, t->foff);
    rc |= upload(&t->d_toff, t->toff);
    rc |= upload(&t->d_aoff, t->aoff);
    rc |= upload(&t->d_goff, t->goff);
    rc |= upload(&t->d_choff, t->choff);
    rc |= upload(&t->d_floff, t->floff);
    rc |= upload(&t->d_coslat, t->coslat);
    rc |= upload(&t->d_w, t->w);
    rc |= upload(&t->d_mu, mu);
    // per-ring scale factors of the ring FFTs, so that no kernel divides in FP64
    std::vector<double> sc64(4 * (size_t)t->nlat);
    std::vector<float> sc32(4 * (size_t)t->nlat);
    for (int k = 0; k < t->nlat; k++) {
        const double wn = t->w[k] / (double)t->nlon[k];
        const double v[4] = {1.0, 1.0 / t->coslat[k], wn, wn / t->coslat[k]};
        for (int j = 0; j < 4; j++) {
            sc64[4 * k + j] = v[j];
            sc32[4 * k + j] = (float)v[j];
        }
    }
    rc |= upload(&t->d_sc64, sc64);
    rc |= upload(&t->d_sc32, sc32);
    // eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)), n = m..T+2, for the derivative
    // and wind recurrences of the spectral pre/post kernels
    std::vector<double> eps(eps_off(t->T, t->T + 1));
    for (int m = 0; m <= t->T; m++)
        for (int n = m; n <= t->T + 2; n++) {
            long double nn = (long double)n * n, mm = (long double)m * m;
            eps[eps_off(t->T, m) + n - m] = n == m ? 0.0 : (double)sqrtl((nn - mm) / (4 * nn - 1));
        }
    rc |= upload(&t->d_eps, eps);
    // 1/eps_n^m (0 at n = m) and Q_m = prod_{k=1}^m sqrt((2k+1)/(2k)) as (mantissa,
    // exponent), both from long double: inputs of the on-the-fly recurrence
    {
        std::vector<double> reps(eps.size(), 0.0);
        for (int m = 0; m <= t->T; m++)
            for (int n = m + 1; n <= t->T + 2; n++) {
                long double nn = (long double)n * n, mm = (long double)m * m;
                reps[eps_off(t->T, m) + n - m] = (double)(1.0L / sqrtl((nn - mm) / (4 * nn - 1)));
            }
        rc |= upload(&t->d_reps, reps);
        std::vector<double2> Q(t->T + 1);
        long double q = 1.0L;
        long qe = 0;
        for (int m = 0; m <= t->T; m++) {
            if (m > 0) q *= sqrtl((long double)(2 * m + 1) / (long double)(2 * m));
            int e;
            q = frexpl(q, &e);
            qe += e;
            Q[m] = make_double2((double)q, (double)qe);
        }
        rc |= upload(&t->d_Q, Q);
    }
    // recurrence coefficients of the spectral pre/post kernels, same index:
    // b_k = (k+2) eps_{k+1} s_{k+1} - (k-1) eps_k s_{k-1} (d/dphi), and
    // h_n = -n eps_{n+1} c_{n+1} + (n+1) eps_n c_{n-1} (wind recombination)
    std::vector<double2> bc(eps.size()), hc(eps.size());
    std::vector<float2> bc32(eps.size());
    std::vector<float4> hc32(eps.size());
    for (int m = 0; m <= t->T; m++)
        for (int n = m; n <= t->T + 1; n++) {
            const long i = eps_off(t->T, m) + n - m;
            bc[i] = make_double2((n + 2) * eps[i + 1], (n - 1) * eps[i]);
            hc[i] = make_double2(-n * eps[i + 1], (n + 1) * eps[i]);
            bc32[i] = make_float2((float)bc[i].x, (float)bc[i].y);
            const float hx = (float)hc[i].x, hy = (float)hc[i].y;
            hc32[i] = make_float4(hx, (float)(hc[i].x - hx), hy, (float)(hc[i].y - hy));
        }
    // FP64 Legendre table of the polar rings (long double recurrence on the
    // host, at the long-double node: rounding mu to FP64 moves a polar node by
    // up to 0.5 ulp / sin(theta) in colatitude, 1e-13 on the first O1280
    // ring, which shifts the phase n theta of the degree-T functions by 1e-10
    // and is what limited the FP64 polar rows before), and beside it the
    // table of G_n^m = cos(phi) dP_n^m/dphi, in the
    // form (n+1) eps_n P_{n-1} - n eps_{n+1} P_{n+1} that the d/dphi
    // recurrence sums, also formed in long double: near the poles its two
    // terms cancel to O(cos(phi)), and rounding them to FP64 first would cost
    // the digits that the 1/cos(phi) of d/dphi and the winds then amplifies.
    {
        int np = 0;
        while (np < t->N && np < 32 && t->coslat[np] < ST_POLAR_COS) np++;
        t->npolar = np;
        std::vector<long> poff((size_t)std::max(np, 1) * (t->T + 1), 0);
        std::vector<double> pt, gt;
        std::vector<long double> pl(t->T + 3);
        for (int k = 0; k < np; k++) {
            const long double th = (long double)t->theta_hi[k] + (long double)t->theta_lo[k];
            const long double x = cosl(th), sn = sinl(th);
            long double pmm = sqrtl(0.5L);  // P_0^0
            for (int m = 0; m <= t->mmax[k]; m++) {
                if (m > 0) pmm *= sqrtl((long double)(2 * m + 1) / (long double)(2 * m)) * sn;
                poff[(size_t)k * (t->T + 1) + m] = (long)pt.size();
                // pl[n - m + 1] = P_n^m for n = m-1 (zero) .. T+1
                pl[0] = 0;
                for (int n = m; n <= t->T + 1; n++) {
                    long double pn;
                    if (n == m) pn = pmm;
                    else if (n == m + 1) pn = sqrtl((long double)(2 * m + 3)) * x * pmm;
                    else pn = (x * pl[n - m] - epsl(n - 1, m) * pl[n - m - 1]) / epsl(n, m);
                    pl[n - m + 1] = pn;
                    pt.push_back((double)pn);
                }
                for (int n = m; n <= t->T + 1; n++) {
                    long double g = 0;
                    if (n <= t->T)
                        g = (n + 1) * epsl(n, m) * pl[n - m] - n * epsl(n + 1, m) * pl[n - m + 2];
                    gt.push_back((double)g);
                }
            }
        }
        rc |= upload(&t->d_poff, poff);
        rc |= upload(&t->d_ptab, pt);
        rc |= upload(&t->d_gtab, gt);
        std::vector<double> fac(t->T + 2, 0.0);
        for (int n = 1; n <= t->T + 1; n++) fac[n] = -1.0 / ((double)n * (n + 1));
        rc |= upload(&t->d_fac, fac);
        // FP32 copies for the polar rows of the FP32 and split plans
        std::vector<float> pt32(pt.begin(), pt.end()), gt32(gt.begin(), gt.end()), fac32(fac.begin(), fac.end());
        rc |= upload(&t->d_ptab32, pt32);
        rc |= upload(&t->d_gtab32, gt32);
        rc |= upload(&t->d_fac32, fac32);
    }
    rc |= upload(&t->d_bc, bc);
    rc |= upload(&t->d_bc32, bc32);
    rc |= upload(&t->d_hc32, hc32);
    rc |= upload(&t->d_hc, hc);
    if (rc) return ST_ERR_NOMEM;
    // chirps c_u = exp(i pi u^2 / n), u = 0..n/2, n = nlon of the ring pair:
    // exact integer reduction of the angle (u^2 mod 2n), then long-double
    // sin/cos.  Stage twiddles exp(-2 pi i j k / L) likewise (j k mod L).
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double2> c64(t->nchirp);
    std::vector<float2> c32(t->nchirp);
    for (int k = 0; k < t->N; k++) {
        const long n = t->nlon[k];
        for (long u = 0; u <= n / 2; u++) {
            const long r = (u * u) % (2 * n);
            const long double a = pi * (long double)r / (long double)n;
            const double2 v = make_double2((double)cosl(a), (double)sinl(a));
            c64[t->choff[k] + u] = v;
            c32[t->choff[k] + u] = make_float2((float)v.x, (float)v.y);
        }
    }
    // per-stage twiddle blocks [k][j] (see fft.cu), spans 2^1 .. 2^13, radix <= 32
    const int logLmax = 13;
    const size_t ntw = 5 * (((size_t)1 << (logLmax + 1)) - 2);
    std::vector<double2> w64(ntw);
    std::vector<float2> w32(ntw);
    for (int logL = 1; logL <= logLmax; logL++) {
        const long L = 1L << logL;
        for (int lr = 1; lr <= 5 && lr <= logL; lr++) {
            const long R = 1L << lr, q = L / R;
            const size_t off = 5 * ((size_t)L - 2) + (size_t)(lr - 1) * L;
            for (long r = 0; r < R; r++)
                for (long j = 0; j < q; j++) {
                    const long e = (j * r) % L;
                    const long double a = -2 * pi * (long double)e / (long double)L;
                    const double2 v = make_double2((double)cosl(a), (double)sinl(a));
                    w64[off + r * q + j] = v;
                    w32[off + r * q + j] = make_float2((float)v.x, (float)v.y);
                }
        }
    }
    rc |= upload(&t->chirp64, c64);
    rc |= upload(&t->chirp32, c32);
    rc |= upload(&t->tw64, w64);
    rc |= upload(&t->tw32, w32);
    if (rc) return ST_ERR_NOMEM;
    if (dev_malloc((void**)&t->filt64, t->nfilt * sizeof(double2)) != cudaSuccess) return ST_ERR_NOMEM;
    if (dev_malloc((void**)&t->filt32, t->nfilt * sizeof(float2)) != cudaSuccess) return ST_ERR_NOMEM;
    return launch_fft_filters(t);
}

// P_n^1 at every northern ring that carries m = 1, n = 0..T+1, for the
// double-float m = 1 sums of the direct winds on the FP32 and split paths:
// the long-double recurrence at the long-double nodes, each value stored as
// FP32 hi + lo (about 48 significant bits).
static int tables_build_wind_m1(Tables* t)
{
    const int T = t->T, N = t->N;
    const int k0 = t->k0[1], nl = N - k0, NP = T + 2;
    std::vector<float2> pw((size_t)std::max(nl, 0) * NP, make_float2(0.f, 0.f));
    std::vector<long double> e(T + 2, 0.0L);
    for (int n = 2; n <= T + 1; n++) e[n] = epsl(n, 1);
    for (int l = 0; l < nl; l++) {
        const int k = k0 + l;
        const long double th = (long double)t->theta_hi[k] + (long double)t->theta_lo[k];
        const long double x = cosl(th), sn = sinl(th);
        long double p2 = 0, p1 = 0;  // P_{n-2}, P_{n-1} (P_0^1 = 0)
        for (int n = 1; n <= T + 1; n++) {
            const long double pn = n == 1 ? sqrtl(0.75L) * sn : (x * p1 - e[n - 1] * p2) / e[n];
            const float hi = (float)pn;
            pw[(size_t)l * NP + n] = make_float2(hi, (float)(pn - (long double)hi));
            p2 = p1;
            p1 = pn;
        }
    }
    return upload(&t->d_pw1, pw);
}

Tables* tables_acquire(int T, int kind, int N, st_prec prec, bool otf, int* status)
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    Tables* t = nullptr;
    for (Tables* c : g_tabs)
        if (c->T == T && c->kind == kind && c->N == N) t = c;
    if (!t) {
        t = new Tables();
        memset((void*)&t->refcount, 0, sizeof(int));
        t->T = T;
        t->kind = kind;
        t->N = N;
        t->refcount = 0;
        t->d_nlon = t->d_mmax = t->d_k0 = t->d_L = t->d_Lp = t->d_logM = nullptr;
        t->d_roff = t->d_foff = t->d_toff = t->d_aoff = t->d_goff = t->d_choff = t->d_floff = nullptr;
        t->d_coslat = t->d_w = t->d_mu = t->d_eps = t->d_sc64 = nullptr;
        t->d_sc32 = nullptr;
        t->d_bc = t->d_hc = nullptr;
        t->d_bc32 = nullptr;
        t->d_hc32 = nullptr;
        t->d_poff = nullptr;
        t->d_ptab = t->d_fac = t->d_gtab = nullptr;
        t->d_ptab32 = t->d_gtab32 = t->d_fac32 = nullptr;
        t->d_pw1 = nullptr;
        t->npolar = 0;
        t->P64 = nullptr;
        t->P32 = nullptr;
        t->Phi = t->Plo = t->Plo2 = nullptr;
        t->chirp64 = t->filt64 = t->tw64 = nullptr;
        t->chirp32 = t->filt32 = t->tw32 = nullptr;
        t->tmaps = nullptr;
        t->d_Q = nullptr;
        t->d_reps = nullptr;
        t->ckpt = nullptr;
        t->d_ckoff = nullptr;
        t->nckpt = 0;
        int rc = tables_build_geometry(t);
        if (rc == ST_OK) rc = tables_upload(t);
        if (rc != ST_OK) {
            if (rc == ST_ERR_NOMEM) set_error("out of device memory building tables for T=%d", T);
            tables_free(t);
            *status = rc;
            return nullptr;
        }
        g_tabs.push_back(t);
    }
    bool need = otf ? !t->ckpt
                    : (prec == ST_PREC_FP64 && !t->P64) || (prec == ST_PREC_FP32 && !t->P32) || (is_split(prec) && !t->Phi);
    const bool need_w1 = prec != ST_PREC_FP64 && T >= 1 && !t->d_pw1;
    if (need || need_w1) {
        int rc = ST_OK;
        if (need) rc = otf ? launch_otf_ckpt(t) : launch_table_gen(t, prec);
        if (rc == ST_OK && need_w1) {
            rc = tables_build_wind_m1(t);
            if (rc != ST_OK) {  // a partial upload leaves the pointer set: drop it
                if (t->d_pw1) cudaFree(t->d_pw1);
                t->d_pw1 = nullptr;
                cudaGetLastError();
            }
        }
        if (rc != ST_OK) {
            // launch_table_gen freed what it allocated; a table that no plan
            // holds yet is dropped, so that no later plan finds it half built
            if (t->refcount == 0) {
                g_tabs.erase(std::remove(g_tabs.begin(), g_tabs.end(), t), g_tabs.end());
                tables_free(t);
            }
            *status = rc;
            return nullptr;
        }
    }
    t->refcount++;
    *status = ST_OK;
    return t;
}

void tables_release(Tables* t)
{
    if (!t) return;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (--t->refcount > 0) return;
    g_tabs.erase(std::remove(g_tabs.begin(), g_tabs.end(), t), g_tabs.end());
    tables_free(t);
}

// -------------------------------------------------------------- work lists
static int elt_bytes(st_prec p) { return p == ST_PREC_FP64 ? 8 : 4; }

void leg_tiles(const Plan* p, int cls, int bn_inv, int bn_dir, std::vector<LegTile>& inv, std::vector<LegTile>& dir)
{
    const Tables* t = p->tab;
    const int bm = leg_bm(p->opts.prec);
    const int ncol = 2 * (cls ? 2 * p->nfld : p->nfld);
    inv.clear();
    dir.clear();
    const bool otf = (p->opts.flags & ST_FLAG_OTF) != 0;
    for (int m = 0; m <= p->T; m++) {
        if (!owns_m(p, m)) continue;
        for (int r = 0; r < t->L[m]; r += bm)
            for (int c = 0; c < ncol; c += bn_inv) inv.push_back({m, 0, r, c, 0});
        if (otf) {  // a direct tile covers the rows r..r+bm-1 of both parities
            for (int r = 0; r < t->K[2 * m]; r += bm)
                for (int c = 0; c < ncol; c += bn_dir) dir.push_back({m, 0, r, c, 0});
            continue;
        }
        for (int pp = 0; pp < 2; pp++)
            for (int r = 0; r < t->K[2 * m + pp]; r += bm)
                for (int c = 0; c < ncol; c += bn_dir) dir.push_back({m, pp, r, c, 0});
    }
    // longest first: the inverse tile costs K_m = T+2-m (already descending), the direct L_m
    std::stable_sort(dir.begin(), dir.end(), [&](const LegTile& a, const LegTile& b) { return t->L[a.m] > t->L[b.m]; });
}

void free_leg_worklists(Plan* p)
{
    for (int c = 0; c < 2; c++) {
        if (p->d_inv_tiles[c]) cudaFree(p->d_inv_tiles[c]);
        if (p->d_dir_tiles[c]) cudaFree(p->d_dir_tiles[c]);
        p->d_inv_tiles[c] = p->d_dir_tiles[c] = nullptr;
    }
}

static int build_tile_lists(Plan* p)
{
    for (int cls = 0; cls < 2; cls++) {
        std::vector<LegTile> inv, dir;
        leg_tiles(p, cls, p->leg_bn[0], p->leg_bn[1], inv, dir);
        int rc = upload(&p->d_inv_tiles[cls], inv) | upload(&p->d_dir_tiles[cls], dir);
        if (rc) return ST_ERR_NOMEM;
        p->n_inv_tiles[cls] = (int)inv.size();
        p->n_dir_tiles[cls] = (int)dir.size();
    }
    return ST_OK;
}

// ---------------------------------------------------------------- autotuner
// Chooses the Legendre tile width of each direction by timing the candidate
// launches on the plan's own workspaces (zeroed first).  With a tune_cache
// path, a line "legendre T=.. N=.. kind=.. nfld=.. prec=.. inv=.. dir=.." is
// looked up before timing and appended after it.
static void tune_key(const Plan* p, char* key, size_t n)
{
    snprintf(key, n, "legendre T=%d N=%d kind=%d nfld=%d prec=%d", p->T, p->grid.N, (int)p->grid.kind, p->nfld,
             (int)p->opts.prec);
}

static bool tune_cache_read(const char* path, const char* key, int* bi, int* bd)
{
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    const size_t kl = strlen(key);
    while (fgets(line, sizeof line, f)) {
        int a, b;
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ' && sscanf(line + kl, " inv=%d dir=%d", &a, &b) == 2) {
            *bi = a;
            *bd = b;
            found = true;  // the last entry wins
        }
    }
    fclose(f);
    return found;
}

static int autotune_leg(Plan* p, const char* cache)
{
    char key[160];
    tune_key(p, key, sizeof key);
    int bi, bd;
    if (cache && tune_cache_read(cache, key, &bi, &bd) && (bi == leg_bn_candidate(p->opts.prec, 0) ||
                                                            bi == leg_bn_candidate(p->opts.prec, 1)) &&
        (bd == leg_bn_candidate(p->opts.prec, 0) || bd == leg_bn_candidate(p->opts.prec, 1))) {
        p->leg_bn[0] = bi;
        p->leg_bn[1] = bd;
        return ST_OK;
    }
    // defined contents for the timing runs
    const size_t eb = p->opts.prec == ST_PREC_FP64 ? 8 : 4;
    const Tables* t = p->tab;
    ST_CUDA_TRY(cudaMemset(p->ws_four, 0, std::max((size_t)t->nfour_rows * p->ncolp * eb,
                                                   (size_t)t->ngop_rows * p->ncolp * (is_split(p->opts.prec) ? 2 : eb))));
    ST_CUDA_TRY(cudaMemset(p->ws_op, 0, (size_t)t->nops_rows * p->ncolp * eb));
    if (p->ws_op_lo) ST_CUDA_TRY(cudaMemset(p->ws_op_lo, 0, (size_t)std::max(t->ngop_rows, t->nops_rows) * p->ncolp * 2));
    if (p->ws_op_lo2) ST_CUDA_TRY(cudaMemset(p->ws_op_lo2, 0, (size_t)std::max(t->ngop_rows, t->nops_rows) * p->ncolp * 2));
    for (int dirn = 0; dirn < 2; dirn++) {
        float best = 1e30f;
        int best_bn = p->leg_bn[dirn];
        for (int v = 0; v < 2; v++) {
            const int bn = leg_bn_candidate(p->opts.prec, v);
            std::vector<LegTile> inv, dir;
            leg_tiles(p, 0, bn, bn, inv, dir);
            std::vector<LegTile>& tl = dirn == 0 ? inv : dir;
            LegTile* d_tiles = nullptr;
            if (upload(&d_tiles, tl)) return ST_ERR_NOMEM;
            LegArgs A;
            memset(&A, 0, sizeof A);
            A.d0 = leg_desc(p, dirn == 0, p->nfld, p->T);
            A.tiles = d_tiles;
            const float ms = time_leg(dirn == 0, p->opts.prec, A, (int)tl.size(), bn, 3);
            cudaFree(d_tiles);
            if (ms < 0) return ST_ERR_CUDA;
            if (ms < best) {
                best = ms;
                best_bn = bn;
            }
        }
        p->leg_bn[dirn] = best_bn;
    }
    if (cache) {
        FILE* f = fopen(cache, "a");
        if (f) {
            fprintf(f, "%s inv=%d dir=%d\n", key, p->leg_bn[0], p->leg_bn[1]);
            fclose(f);
        }
    }
    return ST_OK;
}

int build_leg_worklists(Plan* p)
{
    int rc = build_tile_lists(p);
    if (rc) return rc;
    std::vector<int2> ch;
    for (int m = 0; m <= p->T; m++)
        if (owns_m(p, m))
            for (int n0 = m; n0 <= p->T + 1; n0 += 32) ch.push_back(make_int2(m, n0));
    if (upload(&p->d_spec_chunks, ch)) return ST_ERR_NOMEM;
    p->n_spec_chunks = (int)ch.size();
    return build_fft_worklists(p);
}

// Every stage is also an NVTX range (host side, around its launches), named
// as st_plan_stage_times names the stages; without a tool attached NVTX does
// nothing.
static const char* const k_stage_names[ST_NSTAGES] = {"st pre", "st legendre inverse", "st c2r", "st r2c",
                                                      "st legendre direct", "st post"};

void stage_begin(Plan* p, int stage, cudaStream_t s)
{
    nvtxRangePushA(stage >= 0 && stage < ST_NSTAGES ? k_stage_names[stage] : "st");
    if (!p->ev) return;
    if (p->ev_used >= ST_EV_POOL) {
        p->ev_overflow = 1;
        return;
    }
    cudaEventRecord(p->ev[2 * p->ev_used], s);
}

void stage_fail(Plan*) { nvtxRangePop(); }

void stage_end(Plan* p, int stage, cudaStream_t s)
{
    nvtxRangePop();
    if (!p->ev || p->ev_used >= ST_EV_POOL) return;
    cudaEventRecord(p->ev[2 * p->ev_used + 1], s);
    p->ev_stage[p->ev_used++] = stage;
}

}  // namespace st

using namespace st;

// ------------------------------------------------------------------- C ABI
extern "C" {

const char* st_last_error(void) { return g_err; }

static void plan_free(Plan* p)
{
    if (!p) return;
    if (p->ev) {
        for (int i = 0; i < 2 * ST_EV_POOL; i++)
            if (p->ev[i]) cudaEventDestroy(p->ev[i]);
        delete[] p->ev;
        delete[] p->ev_stage;
    }
    void* ptrs[] = {p->ws_four, p->ws_op, p->ws_op_lo, p->ws_op_lo2, p->ws_gop32, p->d_status, p->d_spec_chunks, p->amaps, p->gmaps};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    free_leg_worklists(p);
    if (p->d_fft_items) cudaFree(p->d_fft_items);
    if (p->d_fft_ctas) cudaFree(p->d_fft_ctas);
    part_free(p);
    tables_release(p->tab);
    delete p;
}

int st_plan_create(st_plan** out, int T, st_grid grid, int nfld, const st_opts* opts)
{
    g_err[0] = 0;
    if (!out) { set_error("st_plan_create: out is NULL"); return ST_ERR_ARG; }
    *out = nullptr;
    if (T < 1 || T > 4000) { set_error("st_plan_create: T=%d outside [1, 4000]", T); return ST_ERR_ARG; }
    if (nfld < 1 || nfld > (1 << 20)) { set_error("st_plan_create: nfld=%d", nfld); return ST_ERR_ARG; }
    if (grid.kind != ST_GRID_OCTAHEDRAL && grid.kind != ST_GRID_FULL_GAUSSIAN) {
        set_error("st_plan_create: unknown grid kind %d", (int)grid.kind);
        return ST_ERR_ARG;
    }
    if (grid.kind == ST_GRID_OCTAHEDRAL && grid.N < T + 1) {
        set_error("st_plan_create: octahedral grid needs N >= T+1 (N=%d, T=%d)", grid.N, T);
        return ST_ERR_ARG;
    }
    if (grid.kind == ST_GRID_FULL_GAUSSIAN && (4 * grid.N < 2 * T + 2 || 2 * grid.N < T + 2)) {
        set_error("st_plan_create: full Gaussian grid N=%d too coarse for T=%d", grid.N, T);
        return ST_ERR_ARG;
    }
    if (grid.N > 8192) { set_error("st_plan_create: N=%d too large", grid.N); return ST_ERR_ARG; }
    st_opts o = {ST_PREC_FP64, 1.0, 0, nullptr};
    if (opts) o = *opts;
    if (o.prec != ST_PREC_FP64 && o.prec != ST_PREC_FP32 && o.prec != ST_PREC_BF16X3 && o.prec != ST_PREC_BF16X6) {
        set_error("st_plan_create: unknown precision %d", (int)o.prec);
        return ST_ERR_ARG;
    }
    if (!(o.radius > 0) || !isfinite(o.radius)) { set_error("st_plan_create: radius must be > 0"); return ST_ERR_ARG; }
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) { set_error("st_plan_create: no CUDA device"); return ST_ERR_CUDA; }
    Plan* p = new Plan();
    memset((void*)p, 0, sizeof(Plan));
    p->T = T;
    p->nfld = nfld;
    p->grid = grid;
    p->opts = o;
    p->opts.tune_cache = nullptr;  // the path is only read during creation
    int rc = ST_OK;
    if ((o.flags & ST_FLAG_OTF) && o.prec != ST_PREC_FP64) {
        set_error("st_plan_create: ST_FLAG_OTF needs an FP64 plan");
        delete p;
        return ST_ERR_UNSUPPORTED;
    }
    if ((o.flags & ST_FLAG_DF64) && (o.prec != ST_PREC_FP64 || (o.flags & ST_FLAG_OTF))) {
        set_error("st_plan_create: ST_FLAG_DF64 needs an FP64 plan with a stored table (not ST_FLAG_OTF)");
        delete p;
        return ST_ERR_UNSUPPORTED;
    }
    p->tab = tables_acquire(T, grid.kind, grid.N, o.prec, (o.flags & ST_FLAG_OTF) != 0, &rc);
    if (!p->tab) { plan_free(p); return rc; }
    const Tables* t = p->tab;
    p->ncolp = (int)round_up(4L * nfld, 8);
    int eb = elt_bytes(o.prec);
    // four (inverse) and Gop (direct) alias; Aop (inverse) and Sop (direct) alias
    size_t four_b = (size_t)t->nfour_rows * p->ncolp * eb;
    size_t gop_rows = (size_t)t->ngop_rows;
    size_t gop_b = gop_rows * p->ncolp * (is_split(o.prec) ? 2 : eb);
    size_t op_b = (size_t)t->nops_rows * p->ncolp * (is_split(o.prec) ? 2 : eb);
    size_t sop_b = (size_t)t->nops_rows * p->ncolp * eb;
    size_t ws1 = std::max(four_b, gop_b), ws2 = std::max(op_b, sop_b);
    if (dev_malloc(&p->ws_four, ws1) != cudaSuccess || dev_malloc(&p->ws_op, ws2) != cudaSuccess ||
        dev_malloc((void**)&p->d_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("st_plan_create: out of device memory for workspaces (%.2f GB)", (ws1 + ws2) / 1e9);
        plan_free(p);
        return ST_ERR_NOMEM;
    }
    p->bytes = ws1 + ws2;
    p->ws_four_b = ws1;
    p->ws_op_b = ws2;
    if (is_split(o.prec)) {
        // planes p1 (and p2) of the split operands: the inverse operand and the
        // direct operand alias, as their plane p0 does
        size_t lo_b = std::max(gop_b, op_b);
        p->ws_lo_b = lo_b;
        // the r2c fold writes the direct operand in FP32 (one store per row
        // instead of one per plane); k_split_gop splits it into the planes
        const size_t g32_b = gop_rows * p->ncolp * sizeof(float);
        if (dev_malloc(&p->ws_op_lo, lo_b) != cudaSuccess ||
            (o.prec == ST_PREC_BF16X6 && dev_malloc(&p->ws_op_lo2, lo_b) != cudaSuccess) ||
            dev_malloc(&p->ws_gop32, g32_b) != cudaSuccess) {
            cudaGetLastError();
            set_error("st_plan_create: out of device memory for split operands");
            plan_free(p);
            return ST_ERR_NOMEM;
        }
        // rows and columns the fold never writes (row padding, unused
        // columns) are split as zeros
        if (cudaMemset(p->ws_gop32, 0, g32_b) != cudaSuccess) {
            set_error("st_plan_create: %s", cudaGetErrorString(cudaGetLastError()));
            plan_free(p);
            return ST_ERR_CUDA;
        }
        p->bytes += lo_b * (nsplit(o.prec) - 1) + g32_b;
        rc = tc_plan_maps(p, &p->amaps, &p->gmaps);
        if (rc != ST_OK) { plan_free(p); return rc; }
    }
    cudaMemset(p->d_status, 0, sizeof(int));
    if (o.flags & ST_FLAG_STAGE_TIMING) {
        p->ev = new cudaEvent_t[2 * ST_EV_POOL]();
        p->ev_stage = new int[ST_EV_POOL]();
        for (int i = 0; i < 2 * ST_EV_POOL; i++)
            if (cudaEventCreate(&p->ev[i]) != cudaSuccess) {
                set_error("st_plan_create: cudaEventCreate failed");
                plan_free(p);
                return ST_ERR_CUDA;
            }
    }
    p->wait_limit = ST_WAIT_LIMIT_DEFAULT;
    p->leg_bn[0] = p->leg_bn[1] = leg_bn_candidate(o.prec, 0);
    if (o.flags & ST_FLAG_AUTOTUNE) {
        rc = autotune_leg(p, o.tune_cache);
        if (rc != ST_OK) { set_error("st_plan_create: autotuning failed"); plan_free(p); return rc; }
    }
    rc = build_leg_worklists(p);
    if (rc != ST_OK) { set_error("st_plan_create: work lists"); plan_free(p); return rc; }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_error("st_plan_create: %s", cudaGetErrorString(cudaGetLastError()));
        plan_free(p);
        return ST_ERR_CUDA;
    }
    *out = (st_plan*)p;
    return ST_OK;
}

int st_plan_destroy(st_plan* pp)
{
    if (!pp) return ST_OK;
    cudaDeviceSynchronize();
    plan_free((Plan*)pp);
    return ST_OK;
}

int st_plan_info(const st_plan* pp, long* npts, long* ncoef, int* nlat, const int** nlon,
                 const long** ring_off)
{
    if (!pp) { set_error("st_plan_info: NULL plan"); return ST_ERR_ARG; }
    const Plan* p = (const Plan*)pp;
    if (npts) *npts = p->tab->npts;
    if (ncoef) *ncoef = (long)(p->T + 1) * (p->T + 2) / 2;
    if (nlat) *nlat = p->tab->nlat;
    if (nlon) *nlon = p->tab->nlon.data();
    if (ring_off) *ring_off = p->tab->roff.data();
    return ST_OK;
}

int st_plan_latitudes(const st_plan* pp, double* mu, double* w)
{
    if (!pp) { set_error("st_plan_latitudes: NULL plan"); return ST_ERR_ARG; }
    const Plan* p = (const Plan*)pp;
    if (mu) memcpy(mu, p->tab->mu.data(), sizeof(double) * p->tab->nlat);
    if (w) memcpy(w, p->tab->w.data(), sizeof(double) * p->tab->nlat);
    return ST_OK;
}

int st_plan_last_launches(const st_plan* pp) { return pp ? ((const Plan*)pp)->last_launches : 0; }

int st_plan_tuning(const st_plan* pp, int* bn_inv, int* bn_dir)
{
    if (!pp) { set_error("st_plan_tuning: NULL plan"); return ST_ERR_ARG; }
    const Plan* p = (const Plan*)pp;
    if (bn_inv) *bn_inv = p->leg_bn[0];
    if (bn_dir) *bn_dir = p->leg_bn[1];
    return ST_OK;
}

int st_debug_fail_alloc(int n)
{
    if (n < 0) {
        set_error("st_debug_fail_alloc: n=%d < 0", n);
        return ST_ERR_ARG;
    }
    g_fail_alloc.store(n);
    return ST_OK;
}

int st_debug_poison_workspaces(st_plan* pp, void* stream)
{
    if (!pp) {
        set_error("st_debug_poison_workspaces: NULL plan");
        return ST_ERR_ARG;
    }
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    // all-ones bytes: a NaN in FP64, FP32 and BF16 alike
    ST_CUDA_TRY(cudaMemsetAsync(p->ws_four, 0xFF, p->ws_four_b, s));
    ST_CUDA_TRY(cudaMemsetAsync(p->ws_op, 0xFF, p->ws_op_b, s));
    if (p->ws_op_lo) ST_CUDA_TRY(cudaMemsetAsync(p->ws_op_lo, 0xFF, p->ws_lo_b, s));
    if (p->ws_op_lo2) ST_CUDA_TRY(cudaMemsetAsync(p->ws_op_lo2, 0xFF, p->ws_lo_b, s));
    return ST_OK;
}

int st_debug_corrupt_worklist(st_plan* pp, int what)
{
    if (!pp || what < 0 || what > 2) {
        set_error("st_debug_corrupt_worklist: %s", pp ? "what must be 0, 1 or 2" : "NULL plan");
        return ST_ERR_ARG;
    }
    Plan* p = (Plan*)pp;
    ST_CUDA_TRY(cudaDeviceSynchronize());
    if (p->dbg_what == 1) ST_CUDA_TRY(cudaMemcpy(p->d_inv_tiles[0], &p->dbg_tile, sizeof(LegTile), cudaMemcpyHostToDevice));
    if (p->dbg_what == 2) ST_CUDA_TRY(cudaMemcpy(p->d_fft_items, &p->dbg_item, sizeof(int4), cudaMemcpyHostToDevice));
    p->dbg_what = 0;
    if (what == 1) {  // the first inverse Legendre tile gets a wavenumber above T
        ST_CUDA_TRY(cudaMemcpy(&p->dbg_tile, p->d_inv_tiles[0], sizeof(LegTile), cudaMemcpyDeviceToHost));
        LegTile bad = p->dbg_tile;
        bad.m = p->T + 7;
        ST_CUDA_TRY(cudaMemcpy(p->d_inv_tiles[0], &bad, sizeof(LegTile), cudaMemcpyHostToDevice));
    } else if (what == 2) {  // the first ring-FFT item gets a ring pair past the grid
        ST_CUDA_TRY(cudaMemcpy(&p->dbg_item, p->d_fft_items, sizeof(int4), cudaMemcpyDeviceToHost));
        int4 bad = p->dbg_item;
        bad.x = p->tab->nlat + 5;
        ST_CUDA_TRY(cudaMemcpy(p->d_fft_items, &bad, sizeof(int4), cudaMemcpyHostToDevice));
    }
    p->dbg_what = what;
    return ST_OK;
}

int st_plan_set_wait_limit(st_plan* pp, long long clocks)
{
    if (!pp || clocks < 0) {
        set_error("st_plan_set_wait_limit: %s", pp ? "negative limit" : "NULL plan");
        return ST_ERR_ARG;
    }
    ((Plan*)pp)->wait_limit = clocks ? clocks : ST_WAIT_LIMIT_DEFAULT;
    return ST_OK;
}

int st_plan_stage_times(st_plan* pp, double* ms, long* launches, int nstages)
{
    if (!pp || !ms || nstages < 1 || nstages > ST_NSTAGES) {
        set_error("st_plan_stage_times: bad argument");
        return ST_ERR_ARG;
    }
    Plan* p = (Plan*)pp;
    if (!p->ev) {
        set_error("st_plan_stage_times: plan created without ST_FLAG_STAGE_TIMING");
        return ST_ERR_ARG;
    }
    ST_CUDA_TRY(cudaDeviceSynchronize());
    for (int i = 0; i < p->ev_used; i++) {
        float t = 0.f;
        ST_CUDA_TRY(cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]));
        int sg = p->ev_stage[i];
        if (sg < nstages) {
            ms[sg] += t;
            if (launches) launches[sg] += 1;
        }
    }
    p->ev_used = 0;
    int ovf = p->ev_overflow;
    p->ev_overflow = 0;
    if (ovf) {
        set_error("st_plan_stage_times: event pool overflowed; some launches were not timed");
        return ST_ERR_UNSUPPORTED;
    }
    return ST_OK;
}

int st_sync_status(st_plan* pp)
{
    if (!pp) { set_error("st_sync_status: NULL plan"); return ST_ERR_ARG; }
    Plan* p = (Plan*)pp;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_error("st_sync_status: %s", cudaGetErrorString(e)); return ST_ERR_CUDA; }
    int h = 0;
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ST_ERR_CUDA;
    cudaMemset(p->d_status, 0, sizeof(int));
    if (h) set_error("device status word %d", h);
    return h;
}

}  // extern "C"
