/*
 * st_oracle.c -- plain FP64 CPU oracle of the spherical-harmonic transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA library.
 *
 * The paper (the ESCAPE spectral-transform dwarf, Sec. 3) names the transform
 * but never writes its mathematics, so every routine here is the plain
 * textbook definition, written out without any fast algorithm:
 *
 *   nodes      Gauss-Legendre nodes and weights by Newton iteration on P_NLAT
 *   P         orthonormal associated Legendre functions by the standard
 *              three-term recurrence, int P^2 dmu = 1, no Condon-Shortley phase
 *   inverse    F_m(mu_k) = sum_n a_n^m P_n^m(mu_k) for every latitude (no
 *              north/south folding), then a direct DFT along each ring
 *   direct     direct DFT along each ring, then the quadrature sum over all
 *              latitudes
 *   deriv, uv  derivatives of P evaluated pointwise (not the spectral shift
 *              recurrences a fast implementation uses)
 *   adjoints   the transposes of the two linear maps, written out
 *
 * Real-field convention: f = Re F_0 + 2 Re sum_{m>0} F_m e^{i m lambda}.
 * Ring k (0..NLAT-1) runs north -> south; its northern index is i = k+1
 * (k < N) or i = 2N-k (k >= N); it has nlon = 4i+16 points (octahedral) or
 * 4N (full Gaussian), lambda_j = 2 pi j / nlon, and carries the wavenumbers
 * m <= mmax = min(T, nlon/2 - 1) (both directions drop the Nyquist bin).
 *
 * Compile with -DORACLE_LONG_DOUBLE to carry every internal value in long
 * double (used at small T to bound this file's own FP64 rounding error).
 *
 * Parity: every function is pinned by the oracle tests (closed forms, library
 * routines, quadrature identities, Parseval, Laplacian, solid-body rotation,
 * adjoint identities, brute force on small sizes).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_LONG_DOUBLE
typedef long double real;
#define R(x) x##L
#define Rcos cosl
#define Rsin sinl
#define Rsqrt sqrtl
#define Rfabs fabsl
#define Rldexp ldexpl
#define Rfrexp frexpl
#define NEWTON_TOL 1e-18L
#else
typedef double real;
#define R(x) x
#define Rcos cos
#define Rsin sin
#define Rsqrt sqrt
#define Rfabs fabs
#define Rldexp ldexp
#define Rfrexp frexp
#define NEWTON_TOL 1e-15
#endif

static const real PI_R = R(3.14159265358979323846264338327950288);

/* ------------------------------------------------------------------ grid */

static int north_index(int N, int k) { return k < N ? k + 1 : 2 * N - k; }

static int ring_nlon(int kind, int N, int k)
{
    return kind == 0 ? 4 * north_index(N, k) + 16 : 4 * N;
}

static int ring_mmax(int T, int nlon)
{
    int a = nlon / 2 - 1;
    return a < T ? a : T;
}

static long coef_off(int T, int m) { return (long)m * (2 * T + 3 - m) / 2; }

/* nlon[k], mmax[k] for the NLAT = 2N rings; returns npts. */
long or_grid(int kind, int N, int T, int* nlon, int* mmax)
{
    long npts = 0;
    for (int k = 0; k < 2 * N; k++) {
        int n = ring_nlon(kind, N, k);
        if (nlon) nlon[k] = n;
        if (mmax) mmax[k] = ring_mmax(T, n);
        npts += n;
    }
    return npts;
}

/* -------------------------------------------------------- Gauss nodes */

/* Legendre polynomial P_n(x) and P_{n-1}(x) by (j+1)P_{j+1} = (2j+1)xP_j - jP_{j-1}. */
static void legendre_pn(int n, real x, real* pn, real* pn1)
{
    real p0 = 1, p1 = x;
    if (n == 0) { *pn = 1; *pn1 = 0; return; }
    for (int j = 1; j < n; j++) {
        real p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

static void gauss_nodes_real(int nlat, real* x, real* w)
{
    int half = (nlat + 1) / 2;
    for (int k = 0; k < half; k++) {
        real xk = Rcos(PI_R * ((k + 1) - R(0.25)) / (nlat + R(0.5)));
        int extra = 0;
        for (int it = 0; it < 100; it++) {
            real pn, pn1;
            legendre_pn(nlat, xk, &pn, &pn1);
            real dp = nlat * (xk * pn - pn1) / (xk * xk - 1);
            real dx = pn / dp;
            xk -= dx;
            if (extra) break;
            if (Rfabs(dx) < NEWTON_TOL) extra = 1;
        }
        if (2 * k + 1 == nlat) xk = 0; /* middle node of an odd count */
        real pn, pn1;
        legendre_pn(nlat, xk, &pn, &pn1);
        real dp = nlat * (xk * pn - pn1) / (xk * xk - 1);
        x[k] = xk;
        w[k] = 2 / ((1 - xk * xk) * dp * dp);
        x[nlat - 1 - k] = -xk;
        w[nlat - 1 - k] = w[k];
    }
}

int or_gauss(int nlat, double* x, double* w)
{
    if (nlat < 1) return 1;
    real* xr = malloc(sizeof(real) * nlat);
    real* wr = malloc(sizeof(real) * nlat);
    gauss_nodes_real(nlat, xr, wr);
    for (int k = 0; k < nlat; k++) { x[k] = (double)xr[k]; w[k] = (double)wr[k]; }
    free(xr);
    free(wr);
    return 0;
}

/* ------------------------------------------- associated Legendre functions */

static real eps_nm(int n, int m)
{
    if (n <= m) return 0;
    real nn = (real)n * n, mm = (real)m * m;
    return Rsqrt((nn - mm) / (4 * nn - 1));
}

/*
 * p[n-m] = P_n^m(x) for n = m..nmax (orthonormal, no Condon-Shortley phase):
 *   P_0^0 = 1/sqrt2,  P_m^m = sqrt((2m+1)/(2m)) sin(theta) P_{m-1}^{m-1},
 *   P_{m+1}^m = sqrt(2m+3) x P_m^m,
 *   P_n^m = (x P_{n-1}^m - eps_{n-1}^m P_{n-2}^m) / eps_n^m.
 * The values are carried as (mantissa, binary exponent) so that P_m^m, which
 * underflows near the poles at large m, keeps its range; results below the
 * FP64 range come out as 0.
 */
static void plm_column(int m, int nmax, real x, real* p)
{
    real s = Rsqrt((1 - x) * (1 + x));
    real v = 1 / Rsqrt(R(2.0));
    long e = 0;
    for (int k = 1; k <= m; k++) {
        int ee;
        v = v * Rsqrt((real)(2 * k + 1) / (real)(2 * k)) * s;
        if (v == 0) break;
        v = Rfrexp(v, &ee);
        e += ee;
    }
    if (nmax < m) return;
    real p2 = v, p1 = 0; /* scaled P_n and P_{n-1} */
    for (int n = m; n <= nmax; n++) {
        real pn;
        if (n == m) pn = v;
        else if (n == m + 1) pn = Rsqrt((real)(2 * m + 3)) * x * v;
        else pn = (x * p2 - eps_nm(n - 1, m) * p1) / eps_nm(n, m);
        if (n > m) { p1 = p2; p2 = pn; }
        /* keep the scaled pair in range */
        if (Rfabs(p2) > R(0x1p500)) { p2 = Rldexp(p2, -500); p1 = Rldexp(p1, -500); e += 500; }
        real out = (n == m) ? v : p2;
        long ex = e;
        if (ex < -20000) out = 0;
        else out = Rldexp(out, (int)ex);
        p[n - m] = out;
    }
}

/* H_n^m = (1 - x^2) dP_n^m/dx = -n eps_{n+1} P_{n+1} + (n+1) eps_n P_{n-1}, n = m..nmax-1. */
static void hlm_column(int m, int nmax, const real* p, real* h)
{
    for (int n = m; n < nmax; n++) {
        real pm1 = (n > m) ? p[n - 1 - m] : 0;
        h[n - m] = -n * eps_nm(n + 1, m) * p[n + 1 - m] + (n + 1) * eps_nm(n, m) * pm1;
    }
}

int or_plm(int m, int nmax, double x, double* out)
{
    if (m < 0 || nmax < m) return 1;
    real* p = malloc(sizeof(real) * (nmax - m + 1));
    plm_column(m, nmax, (real)x, p);
    for (int n = m; n <= nmax; n++) out[n - m] = (double)p[n - m];
    free(p);
    return 0;
}

/* out[n-m] = H_n^m(x) for n = m..nmax. */
int or_hlm(int m, int nmax, double x, double* out)
{
    if (m < 0 || nmax < m) return 1;
    real* p = malloc(sizeof(real) * (nmax - m + 2));
    real* h = malloc(sizeof(real) * (nmax - m + 1));
    plm_column(m, nmax + 1, (real)x, p);
    hlm_column(m, nmax + 1, p, h);
    for (int n = m; n <= nmax; n++) out[n - m] = (double)h[n - m];
    free(p);
    free(h);
    return 0;
}

/* ------------------------------------------------------------- helpers */

typedef struct {
    int T, kind, N, nlat;
    long npts, ncoef;
    real *x, *w;
    int *nlon, *mmax;
    long* roff;
} geom;

static int geom_init(geom* g, int T, int kind, int N)
{
    if (T < 0 || N < 1 || (kind != 0 && kind != 1)) return 1;
    g->T = T; g->kind = kind; g->N = N; g->nlat = 2 * N;
    g->x = malloc(sizeof(real) * g->nlat);
    g->w = malloc(sizeof(real) * g->nlat);
    g->nlon = malloc(sizeof(int) * g->nlat);
    g->mmax = malloc(sizeof(int) * g->nlat);
    g->roff = malloc(sizeof(long) * (g->nlat + 1));
    gauss_nodes_real(g->nlat, g->x, g->w);
    g->npts = or_grid(kind, N, T, g->nlon, g->mmax);
    g->roff[0] = 0;
    for (int k = 0; k < g->nlat; k++) g->roff[k + 1] = g->roff[k] + g->nlon[k];
    g->ncoef = (long)(T + 1) * (T + 2) / 2;
    return 0;
}

static void geom_free(geom* g)
{
    free(g->x); free(g->w); free(g->nlon); free(g->mmax); free(g->roff);
}

/* cos/sin(2 pi t / nlon), t = 0..nlon-1: the angle m*lambda_j is reduced to
 * t = (m*j) mod nlon exactly in integers before the lookup. */
static void ring_twiddles(int nlon, real* c, real* s)
{
    for (int t = 0; t < nlon; t++) {
        real a = 2 * PI_R * t / nlon;
        c[t] = Rcos(a);
        s[t] = Rsin(a);
    }
}

/* Synthesis on one ring: out_j = Re F_0 + 2 sum_{m=1}^{mmax} Re(F_m e^{i m lambda_j}). */
static void ring_synth(int nlon, int mmax, const real* Fre, const real* Fim,
                       const real* c, const real* s, real scale, double* out)
{
    for (int j = 0; j < nlon; j++) {
        real acc = Fre[0];
        for (int m = 1; m <= mmax; m++) {
            int t = (int)(((long)m * j) % nlon);
            acc += 2 * (Fre[m] * c[t] - Fim[m] * s[t]);
        }
        out[j] = (double)(acc * scale);
    }
}

/* Analysis on one ring: F_m = scale * sum_j f_j e^{-i m lambda_j}, m = 0..mmax
 * (only the m with msel[m] != 0 when msel is given). */
static void ring_analysis(int nlon, int mmax, const double* f, const real* c, const real* s,
                          real scale, real* Fre, real* Fim, const unsigned char* msel)
{
    for (int m = 0; m <= mmax; m++) {
        if (msel && !msel[m]) continue;
        real ar = 0, ai = 0;
        for (int j = 0; j < nlon; j++) {
            int t = (int)(((long)m * j) % nlon);
            ar += (real)f[j] * c[t];
            ai -= (real)f[j] * s[t];
        }
        Fre[m] = ar * scale;
        Fim[m] = ai * scale;
    }
}

/* ------------------------------------------------------------ inverse */

/*
 * Inverse transform of nfld fields: spec [nfld][ncoef][2] -> grid [nfld][npts].
 * dlam (d/dlambda) and dphi (d/dphi = cos(phi) d/dmu) are optional (NULL).
 */
static int inverse_impl(int T, int kind, int N, int nfld, const double* spec, double* grid,
                        double* dlam, double* dphi, const unsigned char* sel);

int or_inverse(int T, int kind, int N, int nfld, const double* spec, double* grid,
               double* dlam, double* dphi)
{
    return inverse_impl(T, kind, N, nfld, spec, grid, dlam, dphi, NULL);
}

/*
 * The same, for the rings k with sel[k] != 0 only (sel has 2N entries); the
 * other rings of the outputs are left untouched.  Used to check sampled rings
 * of the largest configurations in long double.
 */
int or_inverse_rings(int T, int kind, int N, int nfld, const double* spec, double* grid,
                     double* dlam, double* dphi, const unsigned char* sel)
{
    return inverse_impl(T, kind, N, nfld, spec, grid, dlam, dphi, sel);
}

static int inverse_impl(int T, int kind, int N, int nfld, const double* spec, double* grid,
                        double* dlam, double* dphi, const unsigned char* sel)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    int maxlon = 0;
    for (int k = 0; k < g.nlat; k++) if (g.nlon[k] > maxlon) maxlon = g.nlon[k];
    int fail = 0;
#pragma omp parallel
    {
        real* p = malloc(sizeof(real) * (T + 3));
        real* h = malloc(sizeof(real) * (T + 2));
        real* c = malloc(sizeof(real) * maxlon);
        real* s = malloc(sizeof(real) * maxlon);
        real* Fre = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Fim = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Gre = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Gim = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Dre = malloc(sizeof(real) * (T + 1));
        real* Dim = malloc(sizeof(real) * (T + 1));
        if (!p || !h || !c || !s || !Fre || !Fim || !Gre || !Gim || !Dre || !Dim) fail = 1;
#pragma omp for schedule(dynamic)
        for (int k = 0; k < g.nlat; k++) {
            if (fail || (sel && !sel[k])) continue;
            int nlon = g.nlon[k], mmax = g.mmax[k];
            real x = g.x[k];
            real coslat = Rsqrt((1 - x) * (1 + x));
            for (int m = 0; m <= mmax; m++) {
                plm_column(m, T + 1, x, p);
                if (dphi) hlm_column(m, T + 1, p, h);
                for (int f = 0; f < nfld; f++) {
                    const double* a = spec + ((size_t)f * g.ncoef + coef_off(T, m)) * 2;
                    real fr = 0, fi = 0, gr = 0, gi = 0;
                    for (int n = m; n <= T; n++) {
                        real ar = a[2 * (n - m)], ai = m ? a[2 * (n - m) + 1] : 0;
                        fr += ar * p[n - m];
                        fi += ai * p[n - m];
                        if (dphi) { gr += ar * h[n - m]; gi += ai * h[n - m]; }
                    }
                    Fre[(size_t)f * (T + 1) + m] = fr;
                    Fim[(size_t)f * (T + 1) + m] = fi;
                    Gre[(size_t)f * (T + 1) + m] = gr;
                    Gim[(size_t)f * (T + 1) + m] = gi;
                }
            }
            ring_twiddles(nlon, c, s);
            for (int f = 0; f < nfld; f++) {
                real* fr = Fre + (size_t)f * (T + 1);
                real* fi = Fim + (size_t)f * (T + 1);
                ring_synth(nlon, mmax, fr, fi, c, s, 1, grid + (size_t)f * g.npts + g.roff[k]);
                if (dlam) {
                    /* d/dlambda: F_m -> i m F_m */
                    for (int m = 0; m <= mmax; m++) { Dre[m] = -m * fi[m]; Dim[m] = m * fr[m]; }
                    ring_synth(nlon, mmax, Dre, Dim, c, s, 1, dlam + (size_t)f * g.npts + g.roff[k]);
                }
                if (dphi)
                    ring_synth(nlon, mmax, Gre + (size_t)f * (T + 1), Gim + (size_t)f * (T + 1), c, s,
                               1 / coslat, dphi + (size_t)f * g.npts + g.roff[k]);
            }
        }
        free(p); free(h); free(c); free(s); free(Fre); free(Fim); free(Gre); free(Gim);
        free(Dre); free(Dim);
    }
    geom_free(&g);
    return fail ? 3 : 0;
}

/* ------------------------------------------------------------- direct */

/* Fourier analysis of every ring: F[f][k][m] (stride T+1), F_m = scale_k sum_j y e^{-i m lambda_j}
 * (only the m with msel[m] != 0 when msel is given). */
static int analyse_all(const geom* g, int nfld, const double* grid, int mode, real* Fre, real* Fim,
                       const unsigned char* msel)
{
    int maxlon = 0, T = g->T, fail = 0;
    for (int k = 0; k < g->nlat; k++) if (g->nlon[k] > maxlon) maxlon = g->nlon[k];
#pragma omp parallel
    {
        real* c = malloc(sizeof(real) * maxlon);
        real* s = malloc(sizeof(real) * maxlon);
        if (!c || !s) fail = 1;
#pragma omp for schedule(dynamic)
        for (int k = 0; k < g->nlat; k++) {
            if (fail) continue;
            int nlon = g->nlon[k];
            ring_twiddles(nlon, c, s);
            /* mode 0: 1/nlon (direct transform); mode 1: 1 (adjoint of the inverse) */
            real scale = mode == 0 ? (real)1 / nlon : 1;
            for (int f = 0; f < nfld; f++) {
                size_t o = ((size_t)f * g->nlat + k) * (T + 1);
                ring_analysis(nlon, g->mmax[k], grid + (size_t)f * g->npts + g->roff[k], c, s, scale,
                              Fre + o, Fim + o, msel);
            }
        }
        free(c);
        free(s);
    }
    return fail;
}

/*
 * Direct transform: grid [nfld][npts] -> spec [nfld][ncoef][2],
 * a_n^m = sum_{k: m <= mmax_k} w_k F_m(k) P_n^m(mu_k).
 */
static int direct_impl(int T, int kind, int N, int nfld, const double* grid, double* spec,
                       const unsigned char* msel);

int or_direct(int T, int kind, int N, int nfld, const double* grid, double* spec)
{
    return direct_impl(T, kind, N, nfld, grid, spec, NULL);
}

/*
 * The same, for the wavenumbers m with msel[m] != 0 only (msel has T+1
 * entries); the coefficients of the other m are left untouched.  Used to check
 * sampled wavenumbers of the largest configurations.
 */
int or_direct_m(int T, int kind, int N, int nfld, const double* grid, double* spec, const unsigned char* msel)
{
    return direct_impl(T, kind, N, nfld, grid, spec, msel);
}

static int direct_impl(int T, int kind, int N, int nfld, const double* grid, double* spec,
                       const unsigned char* msel)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    size_t nf = (size_t)nfld * g.nlat * (T + 1);
    real* Fre = malloc(sizeof(real) * (nf ? nf : 1));
    real* Fim = malloc(sizeof(real) * (nf ? nf : 1));
    int fail = (!Fre || !Fim) || analyse_all(&g, nfld, grid, 0, Fre, Fim, msel);
    if (!fail) {
#pragma omp parallel
        {
            real* p = malloc(sizeof(real) * (T + 2));
            real* acc = malloc(sizeof(real) * (size_t)nfld * (T + 1) * 2);
#pragma omp for schedule(dynamic)
            for (int m = 0; m <= T; m++) {
                if (msel && !msel[m]) continue;
                int K = T - m + 1;
                memset(acc, 0, sizeof(real) * (size_t)nfld * K * 2);
                for (int k = 0; k < g.nlat; k++) {
                    if (m > g.mmax[k]) continue;
                    plm_column(m, T, g.x[k], p);
                    for (int f = 0; f < nfld; f++) {
                        size_t o = ((size_t)f * g.nlat + k) * (T + 1) + m;
                        real fr = g.w[k] * Fre[o], fi = g.w[k] * Fim[o];
                        real* a = acc + (size_t)f * K * 2;
                        for (int n = m; n <= T; n++) {
                            a[2 * (n - m)] += fr * p[n - m];
                            a[2 * (n - m) + 1] += fi * p[n - m];
                        }
                    }
                }
                for (int f = 0; f < nfld; f++)
                    for (int n = m; n <= T; n++) {
                        double* o = spec + ((size_t)f * g.ncoef + coef_off(T, m) + (n - m)) * 2;
                        o[0] = (double)acc[((size_t)f * K + (n - m)) * 2];
                        o[1] = m ? (double)acc[((size_t)f * K + (n - m)) * 2 + 1] : 0.0;
                    }
            }
            free(p);
            free(acc);
        }
    }
    free(Fre);
    free(Fim);
    geom_free(&g);
    return fail ? 3 : 0;
}

/* ----------------------------------------------------------------- uv */

/*
 * Vorticity/divergence -> wind on the sphere of radius a.
 *   psi = -a^2 zeta / (n(n+1)),  chi = -a^2 D / (n(n+1))  (n >= 1; the n = 0 term is 0)
 *   u = (1/a) (-d psi/d phi + (1/cos phi) d chi/d lambda)
 *   v = (1/a) ((1/cos phi) d psi/d lambda + d chi/d phi)
 * evaluated pointwise with d/d phi = H / cos(phi), H = (1 - mu^2) dP/dmu.
 */
static int inverse_uv_impl(int T, int kind, int N, int nfld, double radius, const double* vor,
                           const double* div, double* u, double* v, const unsigned char* sel);

int or_inverse_uv(int T, int kind, int N, int nfld, double radius, const double* vor,
                  const double* div, double* u, double* v)
{
    return inverse_uv_impl(T, kind, N, nfld, radius, vor, div, u, v, NULL);
}

/* The same, for the rings k with sel[k] != 0 only (as or_inverse_rings). */
int or_inverse_uv_rings(int T, int kind, int N, int nfld, double radius, const double* vor,
                        const double* div, double* u, double* v, const unsigned char* sel)
{
    return inverse_uv_impl(T, kind, N, nfld, radius, vor, div, u, v, sel);
}

static int inverse_uv_impl(int T, int kind, int N, int nfld, double radius, const double* vor,
                           const double* div, double* u, double* v, const unsigned char* sel)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    int maxlon = 0, fail = 0;
    for (int k = 0; k < g.nlat; k++) if (g.nlon[k] > maxlon) maxlon = g.nlon[k];
    real a = radius;
#pragma omp parallel
    {
        real* p = malloc(sizeof(real) * (T + 3));
        real* h = malloc(sizeof(real) * (T + 2));
        real* c = malloc(sizeof(real) * maxlon);
        real* s = malloc(sizeof(real) * maxlon);
        real* Ure = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Uim = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Vre = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        real* Vim = malloc(sizeof(real) * (size_t)nfld * (T + 1));
        if (!p || !h || !c || !s || !Ure || !Uim || !Vre || !Vim) fail = 1;
#pragma omp for schedule(dynamic)
        for (int k = 0; k < g.nlat; k++) {
            if (fail || (sel && !sel[k])) continue;
            int nlon = g.nlon[k], mmax = g.mmax[k];
            real x = g.x[k];
            real coslat = Rsqrt((1 - x) * (1 + x));
            for (int m = 0; m <= mmax; m++) {
                plm_column(m, T + 1, x, p);
                hlm_column(m, T + 1, p, h);
                for (int f = 0; f < nfld; f++) {
                    const double* z = vor + ((size_t)f * g.ncoef + coef_off(T, m)) * 2;
                    const double* d = div + ((size_t)f * g.ncoef + coef_off(T, m)) * 2;
                    real ur = 0, ui = 0, vr = 0, vi = 0;
                    for (int n = (m ? m : 1); n <= T; n++) {
                        real fac = -a * a / ((real)n * (n + 1));
                        real pr = fac * z[2 * (n - m)], pi = m ? fac * z[2 * (n - m) + 1] : 0;
                        real cr = fac * d[2 * (n - m)], ci = m ? fac * d[2 * (n - m) + 1] : 0;
                        real P = p[n - m], H = h[n - m];
                        /* U = -psi H + i m chi P,  V = i m psi P + chi H */
                        ur += -pr * H - m * ci * P;
                        ui += -pi * H + m * cr * P;
                        vr += -m * pi * P + cr * H;
                        vi += m * pr * P + ci * H;
                    }
                    Ure[(size_t)f * (T + 1) + m] = ur;
                    Uim[(size_t)f * (T + 1) + m] = ui;
                    Vre[(size_t)f * (T + 1) + m] = vr;
                    Vim[(size_t)f * (T + 1) + m] = vi;
                }
            }
            ring_twiddles(nlon, c, s);
            real sc = 1 / (a * coslat);
            for (int f = 0; f < nfld; f++) {
                ring_synth(nlon, mmax, Ure + (size_t)f * (T + 1), Uim + (size_t)f * (T + 1), c, s, sc,
                           u + (size_t)f * g.npts + g.roff[k]);
                ring_synth(nlon, mmax, Vre + (size_t)f * (T + 1), Vim + (size_t)f * (T + 1), c, s, sc,
                           v + (size_t)f * g.npts + g.roff[k]);
            }
        }
        free(p); free(h); free(c); free(s); free(Ure); free(Uim); free(Vre); free(Vim);
    }
    geom_free(&g);
    return fail ? 3 : 0;
}

/*
 * Wind -> vorticity/divergence (direct):
 *   U = u cos(phi), V = v cos(phi), Fourier analysed with 1/nlon,
 *   zeta_n^m = (1/a) sum_k w_k [i m V_m P_n + U_m H_n] / (1 - mu_k^2)
 *   D_n^m    = (1/a) sum_k w_k [i m U_m P_n - V_m H_n] / (1 - mu_k^2)
 * (the d/dmu term integrated by parts; U vanishes at the poles).
 */
static int direct_uv_impl(int T, int kind, int N, int nfld, double radius, const double* u,
                          const double* v, double* vor, double* div, const unsigned char* msel);

int or_direct_uv(int T, int kind, int N, int nfld, double radius, const double* u, const double* v,
                 double* vor, double* div)
{
    return direct_uv_impl(T, kind, N, nfld, radius, u, v, vor, div, NULL);
}

/* The same, for the wavenumbers m with msel[m] != 0 only (as or_direct_m). */
int or_direct_uv_m(int T, int kind, int N, int nfld, double radius, const double* u, const double* v,
                   double* vor, double* div, const unsigned char* msel)
{
    return direct_uv_impl(T, kind, N, nfld, radius, u, v, vor, div, msel);
}

static int direct_uv_impl(int T, int kind, int N, int nfld, double radius, const double* u,
                          const double* v, double* vor, double* div, const unsigned char* msel)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    size_t nf = (size_t)nfld * g.nlat * (T + 1);
    real* Ure = malloc(sizeof(real) * (nf ? nf : 1));
    real* Uim = malloc(sizeof(real) * (nf ? nf : 1));
    real* Vre = malloc(sizeof(real) * (nf ? nf : 1));
    real* Vim = malloc(sizeof(real) * (nf ? nf : 1));
    /* the grid values times cos(phi) */
    double* Ug = malloc(sizeof(double) * ((size_t)nfld * g.npts + 1));
    double* Vg = malloc(sizeof(double) * ((size_t)nfld * g.npts + 1));
    int fail = !Ure || !Uim || !Vre || !Vim || !Ug || !Vg;
    if (!fail) {
        for (int f = 0; f < nfld; f++)
            for (int k = 0; k < g.nlat; k++) {
                real coslat = Rsqrt((1 - g.x[k]) * (1 + g.x[k]));
                for (long j = g.roff[k]; j < g.roff[k + 1]; j++) {
                    Ug[(size_t)f * g.npts + j] = (double)(u[(size_t)f * g.npts + j] * coslat);
                    Vg[(size_t)f * g.npts + j] = (double)(v[(size_t)f * g.npts + j] * coslat);
                }
            }
        fail = analyse_all(&g, nfld, Ug, 0, Ure, Uim, msel) || analyse_all(&g, nfld, Vg, 0, Vre, Vim, msel);
    }
    real ainv = 1 / (real)radius;
    if (!fail) {
#pragma omp parallel
        {
            real* p = malloc(sizeof(real) * (T + 3));
            real* h = malloc(sizeof(real) * (T + 2));
            real* acc = malloc(sizeof(real) * (size_t)nfld * (T + 1) * 4);
#pragma omp for schedule(dynamic)
            for (int m = 0; m <= T; m++) {
                if (msel && !msel[m]) continue;
                int K = T - m + 1;
                memset(acc, 0, sizeof(real) * (size_t)nfld * K * 4);
                for (int k = 0; k < g.nlat; k++) {
                    if (m > g.mmax[k]) continue;
                    real x = g.x[k];
                    plm_column(m, T + 1, x, p);
                    hlm_column(m, T + 1, p, h);
                    real wk = g.w[k] / ((1 - x) * (1 + x));
                    for (int f = 0; f < nfld; f++) {
                        size_t o = ((size_t)f * g.nlat + k) * (T + 1) + m;
                        real ur = Ure[o], ui = Uim[o], vr = Vre[o], vi = Vim[o];
                        real* A = acc + (size_t)f * K * 4;
                        for (int n = m; n <= T; n++) {
                            real P = p[n - m], H = h[n - m];
                            /* zeta: i m V P + U H;  D: i m U P - V H */
                            A[4 * (n - m) + 0] += wk * (-m * vi * P + ur * H);
                            A[4 * (n - m) + 1] += wk * (m * vr * P + ui * H);
                            A[4 * (n - m) + 2] += wk * (-m * ui * P - vr * H);
                            A[4 * (n - m) + 3] += wk * (m * ur * P - vi * H);
                        }
                    }
                }
                for (int f = 0; f < nfld; f++)
                    for (int n = m; n <= T; n++) {
                        size_t io = ((size_t)f * g.ncoef + coef_off(T, m) + (n - m)) * 2;
                        const real* A = acc + ((size_t)f * K + (n - m)) * 4;
                        vor[io] = (double)(ainv * A[0]);
                        vor[io + 1] = m ? (double)(ainv * A[1]) : 0.0;
                        div[io] = (double)(ainv * A[2]);
                        div[io + 1] = m ? (double)(ainv * A[3]) : 0.0;
                    }
            }
            free(p);
            free(h);
            free(acc);
        }
    }
    free(Ure); free(Uim); free(Vre); free(Vim); free(Ug); free(Vg);
    geom_free(&g);
    return fail ? 3 : 0;
}

/* ------------------------------------------------------------ adjoints */

/*
 * Adjoint (transpose) of the inverse transform under the real Euclidean inner
 * products on the grid and on the (Re, Im) spectral pairs (Im a_n^0 excluded):
 *   g_n^m = c_m sum_k P_n^m(mu_k) sum_j y_kj e^{-i m lambda_j},  c_0 = 1, c_{m>0} = 2.
 */
int or_inverse_adjoint(int T, int kind, int N, int nfld, const double* grid_cot, double* spec_cot)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    size_t nf = (size_t)nfld * g.nlat * (T + 1);
    real* Fre = malloc(sizeof(real) * (nf ? nf : 1));
    real* Fim = malloc(sizeof(real) * (nf ? nf : 1));
    int fail = (!Fre || !Fim) || analyse_all(&g, nfld, grid_cot, 1, Fre, Fim, NULL);
    if (!fail) {
#pragma omp parallel
        {
            real* p = malloc(sizeof(real) * (T + 2));
            real* acc = malloc(sizeof(real) * (size_t)nfld * (T + 1) * 2);
#pragma omp for schedule(dynamic)
            for (int m = 0; m <= T; m++) {
                int K = T - m + 1;
                real cm = m ? 2 : 1;
                memset(acc, 0, sizeof(real) * (size_t)nfld * K * 2);
                for (int k = 0; k < g.nlat; k++) {
                    if (m > g.mmax[k]) continue;
                    plm_column(m, T, g.x[k], p);
                    for (int f = 0; f < nfld; f++) {
                        size_t o = ((size_t)f * g.nlat + k) * (T + 1) + m;
                        real* a = acc + (size_t)f * K * 2;
                        for (int n = m; n <= T; n++) {
                            a[2 * (n - m)] += cm * Fre[o] * p[n - m];
                            a[2 * (n - m) + 1] += cm * Fim[o] * p[n - m];
                        }
                    }
                }
                for (int f = 0; f < nfld; f++)
                    for (int n = m; n <= T; n++) {
                        double* o = spec_cot + ((size_t)f * g.ncoef + coef_off(T, m) + (n - m)) * 2;
                        o[0] = (double)acc[((size_t)f * K + (n - m)) * 2];
                        o[1] = m ? (double)acc[((size_t)f * K + (n - m)) * 2 + 1] : 0.0;
                    }
            }
            free(p);
            free(acc);
        }
    }
    free(Fre);
    free(Fim);
    geom_free(&g);
    return fail ? 3 : 0;
}

/*
 * Adjoint (transpose) of the direct transform:
 *   y_kj = (w_k / nlon_k) sum_{m <= mmax_k} Re(S_m(k) e^{i m lambda_j}),
 *   S_m(k) = sum_n s_n^m P_n^m(mu_k)   (no factor 2 for m > 0; Im s_n^0 unused).
 */
int or_direct_adjoint(int T, int kind, int N, int nfld, const double* spec_cot, double* grid_cot)
{
    geom g;
    if (nfld < 0 || geom_init(&g, T, kind, N)) return 1;
    int maxlon = 0, fail = 0;
    for (int k = 0; k < g.nlat; k++) if (g.nlon[k] > maxlon) maxlon = g.nlon[k];
#pragma omp parallel
    {
        real* p = malloc(sizeof(real) * (T + 2));
        real* c = malloc(sizeof(real) * maxlon);
        real* s = malloc(sizeof(real) * maxlon);
        real* Sre = malloc(sizeof(real) * (T + 1));
        real* Sim = malloc(sizeof(real) * (T + 1));
        if (!p || !c || !s || !Sre || !Sim) fail = 1;
#pragma omp for schedule(dynamic)
        for (int k = 0; k < g.nlat; k++) {
            if (fail) continue;
            int nlon = g.nlon[k], mmax = g.mmax[k];
            ring_twiddles(nlon, c, s);
            real sc = g.w[k] / nlon;
            for (int f = 0; f < nfld; f++) {
                double* out = grid_cot + (size_t)f * g.npts + g.roff[k];
                for (int m = 0; m <= mmax; m++) {
                    plm_column(m, T, g.x[k], p);
                    const double* a = spec_cot + ((size_t)f * g.ncoef + coef_off(T, m)) * 2;
                    real sr = 0, si = 0;
                    for (int n = m; n <= T; n++) {
                        sr += a[2 * (n - m)] * p[n - m];
                        si += (m ? a[2 * (n - m) + 1] : 0) * p[n - m];
                    }
                    Sre[m] = sr;
                    Sim[m] = si;
                }
                for (int j = 0; j < nlon; j++) {
                    real acc = Sre[0];
                    for (int m = 1; m <= mmax; m++) {
                        int t = (int)(((long)m * j) % nlon);
                        acc += Sre[m] * c[t] - Sim[m] * s[t];
                    }
                    out[j] = (double)(acc * sc);
                }
            }
        }
        free(p); free(c); free(s); free(Sre); free(Sim);
    }
    geom_free(&g);
    return fail ? 3 : 0;
}

/* --------------------------------------------------------- diagnostics */

/*
 * Quadrature defect of the rings a wavenumber does not reach:
 *   E_m = max_{n, n'} | sum_{k: m > mmax_k} w_k P_n^m(mu_k) P_n'^m(mu_k) |.
 * On the octahedral grid inverse-then-direct returns a_n^m exactly up to
 * this defect (times sum |a|); it is 0 on the full Gaussian grid.
 * Em has T+1 entries; returns max_m E_m.
 */
double or_roundtrip_defect(int T, int kind, int N, double* Em)
{
    geom g;
    if (geom_init(&g, T, kind, N)) return -1;
    double emax = 0;
    real* p = malloc(sizeof(real) * (T + 2));
    real* M = malloc(sizeof(real) * (size_t)(T + 1) * (T + 1));
    for (int m = 0; m <= T; m++) {
        int K = T - m + 1;
        memset(M, 0, sizeof(real) * (size_t)K * K);
        for (int k = 0; k < g.nlat; k++) {
            if (m <= g.mmax[k]) continue;
            plm_column(m, T, g.x[k], p);
            for (int a = 0; a < K; a++)
                for (int b = 0; b < K; b++) M[(size_t)a * K + b] += g.w[k] * p[a] * p[b];
        }
        real e = 0;
        for (size_t q = 0; q < (size_t)K * K; q++) if (Rfabs(M[q]) > e) e = Rfabs(M[q]);
        if (Em) Em[m] = (double)e;
        if ((double)e > emax) emax = (double)e;
    }
    free(p);
    free(M);
    geom_free(&g);
    return emax;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
