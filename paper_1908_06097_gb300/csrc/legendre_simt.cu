// Legendre step on the CUDA cores (FP64 and FP32 paths) and the table build.
//
// For each zonal wavenumber m the Legendre transform is a dense contraction,
// split by the parity of n - m.  The split uses P_n^m(-mu) = (-1)^{n-m} P_n^m(mu),
// so only the northern rings are stored:
//   inverse  S/A[l][c] = sum_k P_{m,p}[k][l] A_{m,p}[k][c]        (p = 0: S, 1: A)
//            north ring = S + A, south ring = S - A
//   direct   a_{m,p}[k][c] = sum_l P_{m,p}[k][l] G_{m,p}[l][c]
// Every (m, tile) pair is one CTA of a single grouped launch.  The work list
// is ordered longest-first.  The inverse epilogue writes both hemispheres
// straight into the ring-major Fourier buffer.  That write is the transposition.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "st_internal.cuh"

namespace st {

// ---------------------------------------------------------- Legendre tables
// One thread per (m, northern ring).  P_m^m = Q_m sin^m(theta) / sqrt(2), with
// Q_m = prod_{k<=m} sqrt((2k+1)/(2k)) given as (mantissa, exponent).  The
// mantissa and exponent are carried through the n recurrence, so the range
// never underflows, and values below FP64 range are written as 0.
__device__ __forceinline__ double norm2(double v, int* e)
{
    int t;
    double r = frexp(v, &t);
    *e += t;
    return r;
}

// P_m^m at a latitude with sin(colatitude) s, as pmm 2^e (pmm of order 1):
// s^m by binary powering with separate exponents, times Q_m / sqrt(2).
__device__ double pmm_start(int m, double s, double2 Qm, long* e_out)
{
    int er = 0, eb = 0;
    double r = 1.0, bm = norm2(s, &eb);
    for (int mm = m; mm; mm >>= 1) {
        if (mm & 1) {
            r *= bm;
            er += eb;
            r = norm2(r, &er);
        }
        bm *= bm;
        eb *= 2;
        bm = norm2(bm, &eb);
    }
    *e_out = (long)Qm.y + er;
    return Qm.x * r * 0.70710678118654752440;
}

__global__ void k_table_gen(LegGeom lg, const double* __restrict__ mu, const double* __restrict__ coslat,
                            const double2* __restrict__ Q, int prec, double* P64, float* P32, __nv_bfloat16* Phi,
                            __nv_bfloat16* Plo, __nv_bfloat16* Plo2)
{
    const int m = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= lg.L[m]) return;
    const int kN = lg.k0[m] + l, Lp = lg.Lp[m], nmax = lg.T + 1;
    const double x = mu[kN], s = coslat[kN];
    long e;
    const double pmm = pmm_start(m, s, Q[m], &e);
    double cur = 0.0, prev = 0.0;  // P_{n-1}, P_{n-2} (scaled by 2^-e)
    for (int n = m; n <= nmax; n++) {
        double pn;
        if (n == m) {
            pn = pmm;
        } else if (n == m + 1) {
            pn = sqrt((double)(2 * m + 3)) * x * cur;
        } else {
            double e1 = sqrt((double)((n - 1 - m) * (n - 1 + m)) / (double)(4 * (n - 1) * (n - 1) - 1));
            double e2 = sqrt((double)((n - m) * (n + m)) / (double)(4 * n * n - 1));
            pn = (x * cur - e1 * prev) / e2;
        }
        prev = cur;
        cur = pn;
        if (fabs(cur) > 0x1p400) {
            cur = ldexp(cur, -400);
            prev = ldexp(prev, -400);
            e += 400;
        }
        const double v = (e < -1200) ? 0.0 : ldexp(cur, (int)e);
        const int p = (n - m) & 1, kk = (n - m) >> 1;
        const long idx = lg.toff[2 * m + p] + (long)kk * Lp + l;
        if (prec == ST_PREC_FP64) {
            P64[idx] = v;
        } else if (prec == ST_PREC_FP32) {
            P32[idx] = (float)v;
        } else {
            put_split<float>((float*)Phi, Plo, Plo2, idx, v, 3);
        }
    }
}

// Free the table arrays of one precision (after a failed build, so that no
// plan ever finds a table that was allocated but not computed).
static void table_drop(Tables* t, st_prec prec)
{
    void** arrs[] = {(void**)&t->P64, (void**)&t->P32, (void**)&t->Phi, (void**)&t->Plo, (void**)&t->Plo2, &t->tmaps};
    for (int i = 0; i < 6; i++) {
        const bool mine = prec == ST_PREC_FP64 ? i == 0 : (prec == ST_PREC_FP32 ? i == 1 : i >= 2);
        if (mine && *arrs[i]) {
            cudaFree(*arrs[i]);
            *arrs[i] = nullptr;
        }
    }
}

static int table_build(Tables* t, st_prec prec)
{
    const size_t n = (size_t)t->ntab;
    const double gb = n * (prec == ST_PREC_FP64 ? 8.0 : (prec == ST_PREC_FP32 ? 4.0 : 6.0)) / 1e9;
    bool ok;
    if (prec == ST_PREC_FP64) {
        ok = dev_malloc((void**)&t->P64, n * 8) == cudaSuccess;
    } else if (prec == ST_PREC_FP32) {
        ok = dev_malloc((void**)&t->P32, n * 4) == cudaSuccess;
    } else {
        // three bf16 planes serve both split precisions
        ok = dev_malloc((void**)&t->Phi, n * 2) == cudaSuccess && dev_malloc((void**)&t->Plo, n * 2) == cudaSuccess &&
             dev_malloc((void**)&t->Plo2, n * 2) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        set_error("out of device memory for the Legendre table (%.2f GB)", gb);
        return ST_ERR_NOMEM;
    }
    if (prec == ST_PREC_FP64) {
        ST_CUDA_TRY(cudaMemset(t->P64, 0, n * 8));
    } else if (prec == ST_PREC_FP32) {
        ST_CUDA_TRY(cudaMemset(t->P32, 0, n * 4));
    } else {
        ST_CUDA_TRY(cudaMemset(t->Phi, 0, n * 2));
        ST_CUDA_TRY(cudaMemset(t->Plo, 0, n * 2));
        ST_CUDA_TRY(cudaMemset(t->Plo2, 0, n * 2));
        int rc = tc_table_maps(t, &t->tmaps);
        if (rc) return rc;
    }
    // Q_m = prod_{k=1}^m sqrt((2k+1)/(2k)) as (mantissa, exponent), long double
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
    double2* dQ = nullptr;
    if (dev_malloc((void**)&dQ, Q.size() * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        set_error("out of device memory for the Legendre table build");
        return ST_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpy(dQ, Q.data(), Q.size() * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        dim3 grid((t->N + 127) / 128, t->T + 1);
        k_table_gen<<<grid, 128>>>(t->leg(), t->d_mu, t->d_coslat, dQ, is_split(prec) ? (int)ST_PREC_BF16X3 : (int)prec,
                                   t->P64, t->P32, t->Phi, t->Plo, t->Plo2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dQ);
    if (e != cudaSuccess) {
        set_error("Legendre table build: %s", cudaGetErrorString(e));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}

int launch_table_gen(Tables* t, st_prec prec)
{
    const int rc = table_build(t, prec);
    if (rc != ST_OK) table_drop(t, prec);
    return rc;
}

// ------------------------------------------------------------- SIMT GEMMs
// Tiles of 256 threads: BM x BN outputs, TM x TN per thread (TN = BN/16).
// The tile width BN is the autotuned choice (see st_plan_create).
template <typename R, int BN_> struct SimtCfg;
template <int BN_> struct SimtCfg<double, BN_> { enum { BM = 64, BN = BN_, BK = 16, TM = 4, TN = BN_ / 16 }; };
template <int BN_> struct SimtCfg<float, BN_> { enum { BM = 128, BN = BN_, BK = 16, TM = 8, TN = BN_ / 16 }; };

// Candidate tile widths per precision (variant 0 is the default).
int leg_bn_candidate(st_prec prec, int variant)
{
    if (prec == ST_PREC_FP64) return variant ? 32 : 64;
    if (prec == ST_PREC_FP32) return variant ? 64 : 128;
    return variant ? 64 : 128;  // tensor-core tiles (legendre_tc.cu)
}

int leg_bm(st_prec prec) { return prec == ST_PREC_FP64 ? 64 : 128; }

__device__ __forceinline__ int kcount(int nmax, int m, int p) { return nmax - m - p >= 0 ? (nmax - m - p) / 2 + 1 : 0; }

template <typename R, int BNT>
__device__ __forceinline__ void leg_inv_simt_item(const LegArgs& Ag, int item)
{
    const LegTile tl = Ag.tiles[item];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const RingGeom& rg = D.rg;
    const R* __restrict__ P = (const R*)D.P;
    const R* __restrict__ Aop = (const R*)D.X;
    R* __restrict__ four = (R*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    typedef SimtCfg<R, BNT> SC;
    enum { BM = SC::BM, BN = SC::BN, BK = SC::BK, TM = SC::TM, TN = SC::TN };
    enum { NTX = BN / TN, NT = (BM / TM) * (BN / TN) };
    __shared__ __align__(16) R As[BK][BM];
    __shared__ __align__(16) R Bs[BK][BN];
    const int m = tl.m, l0 = tl.r0, c0 = tl.c0;
    const int L = lg.L[m], Lp = lg.Lp[m];
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    R acc[2][TM][TN];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) acc[p][i][j] = 0;
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int K = kcount(nmax, m, p);
        const R* Pb = P + lg.toff[2 * m + p];
        const R* Ab = Aop + lg.aoff[2 * m + p] * (long)ncolp;
        for (int k0 = 0; k0 < K; k0 += BK) {
            for (int e = threadIdx.x; e < BK * BM; e += NT) {
                const int kk = e / BM, i = e % BM;
                As[kk][i] = (k0 + kk < K && l0 + i < L) ? Pb[(long)(k0 + kk) * Lp + l0 + i] : (R)0;
            }
            for (int e = threadIdx.x; e < BK * BN; e += NT) {
                const int kk = e / BN, j = e % BN;
                Bs[kk][j] = (k0 + kk < K && c0 + j < ncol) ? Ab[(long)(k0 + kk) * ncolp + c0 + j] : (R)0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                R a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; i++) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; j++) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; i++)
#pragma unroll
                    for (int j = 0; j < TN; j++) acc[p][i][j] = fma(a[i], b[j], acc[p][i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int l = l0 + ty * TM + i;
        if (l >= L) continue;
        const int kN = lg.k0[m] + l, kS = lg.nlat - 1 - kN;
        R* on = four + (rg.foff[kN] + m) * (long)ncolp;
        R* os = four + (rg.foff[kS] + m) * (long)ncolp;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = c0 + tx * TN + j;
            if (c < ncol) {
                on[c] = acc[0][i][j] + acc[1][i][j];
                os[c] = acc[0][i][j] - acc[1][i][j];
            }
        }
    }
}

template <typename R, int BNT>
__device__ __forceinline__ void leg_dir_simt_item(const LegArgs& Ag, int item)
{
    const LegTile tl = Ag.tiles[item];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const R* __restrict__ P = (const R*)D.P;
    const R* __restrict__ Gop = (const R*)D.X;
    R* __restrict__ Sop = (R*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    typedef SimtCfg<R, BNT> SC;
    enum { BM = SC::BM, BN = SC::BN, BK = SC::BK, TM = SC::TM, TN = SC::TN };
    enum { NTX = BN / TN, NT = (BM / TM) * (BN / TN) };
    __shared__ __align__(16) R As[BK][BM + 1];
    __shared__ __align__(16) R Bs[BK][BN];
    const int m = tl.m, p = tl.p, r0 = tl.r0, c0 = tl.c0;
    const int K = kcount(nmax, m, p);
    if (r0 >= K) return;
    const int L = lg.L[m], Lp = lg.Lp[m];
    const R* Pb = P + lg.toff[2 * m + p];
    const R* Gb = Gop + lg.goff[2 * m + p] * (long)ncolp;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = 0;
    for (int l0 = 0; l0 < L; l0 += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += NT) {
            const int kk = e % BK, i = e / BK;
            As[kk][i] = (r0 + i < K && l0 + kk < L) ? Pb[(long)(r0 + i) * Lp + l0 + kk] : (R)0;
        }
        for (int e = threadIdx.x; e < BK * BN; e += NT) {
            const int kk = e / BN, j = e % BN;
            Bs[kk][j] = (l0 + kk < L && c0 + j < ncol) ? Gb[(long)(l0 + kk) * ncolp + c0 + j] : (R)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            R a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; i++) a[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; j++) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    R* Sb = Sop + lg.aoff[2 * m + p] * (long)ncolp;
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int k = r0 + ty * TM + i;
        if (k >= K) continue;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = c0 + tx * TN + j;
            if (c < ncol) Sb[(long)k * ncolp + c] = acc[i][j];
        }
    }
}

// ---------------------------------------- double-float Legendre (ST_FLAG_DF64)
// FP64 plans whose Legendre contractions run on the FP32 pipes, which GB300
// issues 64 times faster than FP64.  Table and operands stay FP64 in memory;
// each value is split as it is staged in shared memory into hi = fp32(x) and
// lo = fp32(x - hi), about 48 significant bits between them, and each output
// accumulates in a pair (sh, sl):
//   - the product of two pairs a, b: the leading product exactly by an FMA
//     (p + e = a.h b.h, Dekker's two-product), the cross terms a.h b.l and
//     a.l b.h added into e (a.l b.l, below 2^-47 of the product, is dropped);
//   - the sum: sh + p exactly by Knuth's two-sum, its error and e into sl;
//   - every DF_NORM products sl is folded back into sh (fast two-sum), so
//     that it stays a few units of 2^-24 of sh and its own rounding is near
//     2^-48 of the partial sums.
// Outputs leave as FP64 sh + sl.  The _rn intrinsics keep the compiler from
// contracting these steps.  Values beyond the FP32 range (about 3.4e38) are
// not representable on this path; values below about 1e-38 lose their low
// part (their share of any output is below that).
constexpr int DF_NORM = 4;
struct DfPair {
    float h, l;
};
// hi = fp32(x) by the integer conversion dbl2flt_rn, and lo = fp32(x - hi)
// from the significand bits that hi drops, also with integer operations: the
// split then keeps GB300's narrow FP64 pipe free (two FP64 conversions and a
// subtraction per staged value kept it as busy as the FP32 pipe).  With
// M = the 53-bit significand of x and Mh = M >> 29 rounded to nearest even
// (hi's significand), x - hi = (M - Mh 2^29) 2^(e - 1075), an integer R with
// |R| <= 2^28; lo = fp32(R) 2^(e - 1075).  |x| < 2^-100 (and zero) keep no low
// part; values out of the FP32 range are not supported on this path.
__device__ __forceinline__ DfPair df_split(double x)
{
    const float h = dbl2flt_rn(x);
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const int e = (int)((hw >> 20) & 0x7FFu);
    if (e < 1023 - 100 || e > 1023 + 127) return {h, 0.f};
    const unsigned long long m = ((unsigned long long)(hw & 0xFFFFFu) << 32) | lw;
    const unsigned long long M = m | (1ull << 52);
    const unsigned long long Mh = (M + 0x0FFFFFFFull + ((M >> 29) & 1ull)) >> 29;
    const int R = (int)((long long)M - (long long)(Mh << 29));
    // 2^(e - 1075) as a float: e - 1075 + 127 = e - 948 lies in [-25, 202] here;
    // below 1 the scale goes through two steps so that it stays a normal float
    float lo = (float)R;
    const int sc = e - 948;
    if (sc >= 1) lo *= __int_as_float(sc << 23);
    else lo = (lo * __int_as_float((sc + 64) << 23)) * 5.421010862427522e-20f;  // 2^-64
    return {h, (hw >> 31) ? -lo : lo};  // R is the residual of |x|
}
__device__ __forceinline__ void df_mac(float& sh, float& sl, DfPair a, DfPair b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float s = __fadd_rn(sh, p), v = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}
__device__ __forceinline__ void df_norm(float& sh, float& sl)
{
    const float s = __fadd_rn(sh, sl);
    sl = __fsub_rn(sl, __fsub_rn(s, sh));
    sh = s;
}
__device__ __forceinline__ double df_value(float sh, float sl) { return (double)sh + (double)sl; }

// 64 x BN tiles of 256 threads, 4 x (BN/16) outputs per thread, 16-deep slabs
template <int BNT>
__device__ __forceinline__ void leg_inv_df_item(const LegArgs& Ag, int item)
{
    const LegTile tl = Ag.tiles[item];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const RingGeom& rg = D.rg;
    const double* __restrict__ P = (const double*)D.P;
    const double* __restrict__ Aop = (const double*)D.X;
    double* __restrict__ four = (double*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    enum { BM = 64, BN = BNT, BK = 16, TM = 4, TN = BNT / 16, NTX = BN / TN, NT = (BM / TM) * NTX };
    __shared__ __align__(16) DfPair As[BK][BM];
    __shared__ __align__(16) DfPair Bs[BK][BN];
    const int m = tl.m, l0 = tl.r0, c0 = tl.c0;
    const int L = lg.L[m], Lp = lg.Lp[m];
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    float ah[2][TM][TN], al[2][TM][TN];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) ah[p][i][j] = al[p][i][j] = 0.f;
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int K = kcount(nmax, m, p);
        const double* Pb = P + lg.toff[2 * m + p];
        const double* Ab = Aop + lg.aoff[2 * m + p] * (long)ncolp;
        // the next slab's values are loaded into registers while this slab
        // is multiplied (its loads were the top stall)
        double ra[BK * BM / NT], rb[BK * BN / NT];
        auto fetch = [&](int k0) {
#pragma unroll
            for (int q = 0; q < BK * BM / NT; q++) {
                const int e = threadIdx.x + q * NT, kk = e / BM, i = e % BM;
                ra[q] = (k0 + kk < K && l0 + i < L) ? Pb[(long)(k0 + kk) * Lp + l0 + i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < BK * BN / NT; q++) {
                const int e = threadIdx.x + q * NT, kk = e / BN, j = e % BN;
                rb[q] = (k0 + kk < K && c0 + j < ncol) ? Ab[(long)(k0 + kk) * ncolp + c0 + j] : 0.0;
            }
        };
        if (K > 0) fetch(0);
        for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
            for (int q = 0; q < BK * BM / NT; q++) {
                const int e = threadIdx.x + q * NT;
                As[e / BM][e % BM] = df_split(ra[q]);
            }
#pragma unroll
            for (int q = 0; q < BK * BN / NT; q++) {
                const int e = threadIdx.x + q * NT;
                Bs[e / BN][e % BN] = df_split(rb[q]);
            }
            __syncthreads();
            if (k0 + BK < K) fetch(k0 + BK);
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                DfPair a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; i++) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; j++) b[j] = Bs[kk][j * NTX + tx];
#pragma unroll
                for (int i = 0; i < TM; i++)
#pragma unroll
                    for (int j = 0; j < TN; j++) {
                        df_mac(ah[p][i][j], al[p][i][j], a[i], b[j]);
                        if (kk % DF_NORM == DF_NORM - 1) df_norm(ah[p][i][j], al[p][i][j]);
                    }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int l = l0 + ty * TM + i;
        if (l >= L) continue;
        const int kN = lg.k0[m] + l, kS = lg.nlat - 1 - kN;
        double* on = four + (rg.foff[kN] + m) * (long)ncolp;
        double* os = four + (rg.foff[kS] + m) * (long)ncolp;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = c0 + j * NTX + tx;
            if (c < ncol) {
                const double S = df_value(ah[0][i][j], al[0][i][j]), A = df_value(ah[1][i][j], al[1][i][j]);
                on[c] = S + A;
                os[c] = S - A;
            }
        }
    }
}

template <int BNT>
__device__ __forceinline__ void leg_dir_df_item(const LegArgs& Ag, int item)
{
    const LegTile tl = Ag.tiles[item];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const double* __restrict__ P = (const double*)D.P;
    const double* __restrict__ Gop = (const double*)D.X;
    double* __restrict__ Sop = (double*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    enum { BM = 64, BN = BNT, BK = 16, TM = 4, TN = BNT / 16, NTX = BN / TN, NT = (BM / TM) * NTX };
    __shared__ __align__(16) DfPair As[BK][BM + 1];
    __shared__ __align__(16) DfPair Bs[BK][BN];
    const int m = tl.m, p = tl.p, r0 = tl.r0, c0 = tl.c0;
    const int K = kcount(nmax, m, p);
    if (r0 >= K) return;
    const int L = lg.L[m], Lp = lg.Lp[m];
    const double* Pb = P + lg.toff[2 * m + p];
    const double* Gb = Gop + lg.goff[2 * m + p] * (long)ncolp;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    float ah[TM][TN], al[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) ah[i][j] = al[i][j] = 0.f;
    // the next slab's values are loaded into registers while this slab is
    // multiplied (its loads were the top stall)
    double ra[BK * BM / NT], rb[BK * BN / NT];
    auto fetch = [&](int l0) {
#pragma unroll
        for (int q = 0; q < BK * BM / NT; q++) {
            const int e = threadIdx.x + q * NT, kk = e % BK, i = e / BK;
            ra[q] = (r0 + i < K && l0 + kk < L) ? Pb[(long)(r0 + i) * Lp + l0 + kk] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < BK * BN / NT; q++) {
            const int e = threadIdx.x + q * NT, kk = e / BN, j = e % BN;
            rb[q] = (l0 + kk < L && c0 + j < ncol) ? Gb[(long)(l0 + kk) * ncolp + c0 + j] : 0.0;
        }
    };
    if (L > 0) fetch(0);
    for (int l0 = 0; l0 < L; l0 += BK) {
#pragma unroll
        for (int q = 0; q < BK * BM / NT; q++) {
            const int e = threadIdx.x + q * NT;
            As[e % BK][e / BK] = df_split(ra[q]);
        }
#pragma unroll
        for (int q = 0; q < BK * BN / NT; q++) {
            const int e = threadIdx.x + q * NT;
            Bs[e / BN][e % BN] = df_split(rb[q]);
        }
        __syncthreads();
        if (l0 + BK < L) fetch(l0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            DfPair a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; i++) a[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; j++) b[j] = Bs[kk][j * NTX + tx];
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) {
                    df_mac(ah[i][j], al[i][j], a[i], b[j]);
                    if (kk % DF_NORM == DF_NORM - 1) df_norm(ah[i][j], al[i][j]);
                }
        }
        __syncthreads();
    }
    double* Sb = Sop + lg.aoff[2 * m + p] * (long)ncolp;
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int k = r0 + ty * TM + i;
        if (k >= K) continue;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = c0 + j * NTX + tx;
            if (c < ncol) Sb[(long)k * ncolp + c] = df_value(ah[i][j], al[i][j]);
        }
    }
}

// Tiles of m <= 1 run the FP64 body (same 64 x BN tiling): there the two
// terms of the direct winds cancel by about 1e3 near the poles, which would
// make the double-float rounding visible; these are 2 of T+1 wavenumbers.
template <int BNT>
__global__ void __launch_bounds__(256, 1) k_leg_inv_df(const __grid_constant__ LegArgs Ag)
{
    run_items(Ag.q, [&](int w) {
        if (Ag.tiles[w].m <= 1) leg_inv_simt_item<double, BNT>(Ag, w);
        else leg_inv_df_item<BNT>(Ag, w);
    });
}
template <int BNT>
__global__ void __launch_bounds__(256, 1) k_leg_dir_df(const __grid_constant__ LegArgs Ag)
{
    run_items(Ag.q, [&](int w) {
        if (Ag.tiles[w].m <= 1) leg_dir_simt_item<double, BNT>(Ag, w);
        else leg_dir_df_item<BNT>(Ag, w);
    });
}

// ------------------------------------------- on-the-fly Legendre functions
// FP64 plans created with ST_FLAG_OTF store no table of P_n^m: the kernels
// below regenerate it inside the contraction by the same three-term
// recurrence in n that the table generator runs, in the scaled
// representation P = cur 2^e (so that the polar values that FP64 cannot hold
// are carried, and written as 0 below 2^-1200 as in the table):
//   P_{m+1} = sqrt(2m+3) mu P_m,   P_n = (mu P_{n-1} - eps_{n-1} P_{n-2}) / eps_n.
// The division is a multiplication by 1/eps_n from a table.  Every step uses
// explicit round-to-nearest operations, so the checkpoint builder and both
// kernels produce the same values bit for bit.  The inverse kernel walks n
// upwards from m for its latitudes (n is its contraction index).  The direct
// kernel needs P_n for one block of 128 degrees (64 rows of each parity) at
// every latitude: it restarts the recurrence from a checkpoint, the state
// (P_{n-2}, P_{n-1}) stored before each block, so the stored data per (m,
// latitude) is 1/64 of the table.
struct OtfState {
    double prev, cur;  // P_{n-2}, P_{n-1} times 2^-e
    long e;
};

__device__ __forceinline__ double otf_value(const OtfState& st)
{
    return st.e < -1200 ? 0.0 : ldexp(st.cur, (int)st.e);
}

// advance to degree n > m and return P_n
__device__ __forceinline__ double otf_step(int n, int m, double x, double s2m3, const double* eps_m,
                                           const double* reps_m, OtfState& st)
{
    double pn;
    if (n == m + 1) pn = __dmul_rn(__dmul_rn(s2m3, x), st.cur);
    else pn = __dmul_rn(__fma_rn(x, st.cur, -__dmul_rn(eps_m[n - 1], st.prev)), reps_m[n]);
    st.prev = st.cur;
    st.cur = pn;
    if (fabs(st.cur) > 0x1p400) {
        st.cur = __dmul_rn(st.cur, 0x1p-400);
        st.prev = __dmul_rn(st.prev, 0x1p-400);
        st.e += 400;
    }
    return otf_value(st);
}

// the state after degree m at latitude (x, s)
__device__ __forceinline__ OtfState otf_start(int m, double s, double2 Qm)
{
    OtfState st;
    st.prev = 0.0;
    st.cur = pmm_start(m, s, Qm, &st.e);
    return st;
}

// checkpoints: one thread per (m, northern latitude); the state before
// degree m + 128 b is stored at ck[ckoff[m] + (b - 1) L_m + l], b >= 1
__global__ void k_otf_ckpt(LegGeom lg, const double* __restrict__ mu, const double* __restrict__ coslat,
                           const double2* __restrict__ Q, const double* __restrict__ reps, const long* __restrict__ ckoff,
                           OtfState* __restrict__ ck)
{
    const int m = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int L = lg.L[m];
    if (l >= L) return;
    const int kN = lg.k0[m] + l, nmax = lg.T + 1;
    const double x = mu[kN], s2m3 = sqrt((double)(2 * m + 3));
    const double* eps_m = lg.eps + eps_off(lg.T, m) - m;
    const double* reps_m = reps + eps_off(lg.T, m) - m;
    OtfState st = otf_start(m, coslat[kN], Q[m]);
    for (int n = m + 1; n <= nmax; n++) {
        if (((n - m) & 127) == 0) ck[ckoff[m] + (long)((n - m) / 128 - 1) * L + l] = st;
        otf_step(n, m, x, s2m3, eps_m, reps_m, st);
    }
}

template <int BNT>
__global__ void __launch_bounds__(256) k_leg_inv_otf(const __grid_constant__ LegArgs Ag)
{
    const LegTile tl = Ag.tiles[blockIdx.x];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const RingGeom& rg = D.rg;
    const double* __restrict__ Aop = (const double*)D.X;
    double* __restrict__ four = (double*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    typedef SimtCfg<double, BNT> SC;
    enum { BM = SC::BM, BN = SC::BN, BK = SC::BK, TM = SC::TM, TN = SC::TN };
    enum { NTX = BN / TN, NT = (BM / TM) * (BN / TN) };
    __shared__ __align__(16) double As[2][BK][BM];
    __shared__ __align__(16) double Bs[2][BK][BN];
    const int m = tl.m, l0 = tl.r0, c0 = tl.c0;
    const int L = lg.L[m];
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const int Ks = kcount(nmax, m, 0), Ka = kcount(nmax, m, 1);
    // the first BM threads each run the recurrence of one latitude
    const bool gen = threadIdx.x < BM, glive = gen && l0 + (int)threadIdx.x < L;
    const double* eps_m = lg.eps + eps_off(lg.T, m) - m;
    const double* reps_m = D.reps + eps_off(lg.T, m) - m;
    const double s2m3 = sqrt((double)(2 * m + 3));
    double x = 0.0;
    OtfState st = {0.0, 0.0, 0};
    if (glive) {
        const int kN = lg.k0[m] + l0 + threadIdx.x;
        x = D.mu[kN];
        st = otf_start(m, rg.coslat[kN], D.Qm[m]);
    }
    double acc[2][TM][TN];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) acc[p][i][j] = 0.0;
    // each step covers 2 BK consecutive degrees: BK rows of each parity
    for (int n0 = m; n0 <= nmax; n0 += 2 * BK) {
        const int k0 = (n0 - m) >> 1;
        if (gen) {
#pragma unroll 4
            for (int j = 0; j < 2 * BK; j++) {
                const int n = n0 + j;
                double v = 0.0;
                if (glive && n <= nmax) v = n == m ? otf_value(st) : otf_step(n, m, x, s2m3, eps_m, reps_m, st);
                As[j & 1][j >> 1][threadIdx.x] = v;
            }
        }
        for (int e = threadIdx.x; e < 2 * BK * BN; e += NT) {
            const int p = e / (BK * BN), r = e % (BK * BN), kk = r / BN, j = r % BN;
            const int K = p ? Ka : Ks;
            Bs[p][kk][j] = (k0 + kk < K && c0 + j < ncol) ? Aop[(lg.aoff[2 * m + p] + k0 + kk) * (long)ncolp + c0 + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 2; p++) {
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                double a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; i++) a[i] = As[p][kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; j++) b[j] = Bs[p][kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; i++)
#pragma unroll
                    for (int j = 0; j < TN; j++) acc[p][i][j] = fma(a[i], b[j], acc[p][i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int l = l0 + ty * TM + i;
        if (l >= L) continue;
        const int kN = lg.k0[m] + l, kS = lg.nlat - 1 - kN;
        double* on = four + (rg.foff[kN] + m) * (long)ncolp;
        double* os = four + (rg.foff[kS] + m) * (long)ncolp;
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int c = c0 + tx * TN + j;
            if (c < ncol) {
                on[c] = acc[0][i][j] + acc[1][i][j];
                os[c] = acc[0][i][j] - acc[1][i][j];
            }
        }
    }
}

// direct: a tile is one block of BM rows of BOTH parities (degrees n0 .. n0 +
// 2 BM - 1, n0 = m + 2 r0) and BN columns; the contraction runs over the
// latitudes, BK at a time, whose recurrences restart from the checkpoint of
// the block
template <int BNT>
__global__ void __launch_bounds__(256) k_leg_dir_otf(const __grid_constant__ LegArgs Ag)
{
    const LegTile tl = Ag.tiles[blockIdx.x];
    if (!leg_tile_ok(Ag, tl)) return;
    const LegDesc& D = Ag.desc ? Ag.desc[tl.mb] : Ag.d0;
    const LegGeom& lg = D.lg;
    const RingGeom& rg = D.rg;
    const double* __restrict__ Gop = (const double*)D.X;
    double* __restrict__ Sop = (double*)D.Y;
    const int ncolp = D.ncolp, ncol = D.ncol, nmax = D.nmax;
    typedef SimtCfg<double, BNT> SC;
    enum { BM = SC::BM, BN = SC::BN, BK = SC::BK, TM = SC::TM, TN = SC::TN };
    enum { NTX = BN / TN, NT = (BM / TM) * (BN / TN) };
    static_assert(2 * BM == 128, "a direct tile covers one checkpoint block of 128 degrees");
    __shared__ __align__(16) double As[2][BK][BM + 1];
    __shared__ __align__(16) double Bs[2][BK][BN];
    const int m = tl.m, r0 = tl.r0, c0 = tl.c0;
    const int Ks = kcount(nmax, m, 0), Ka = kcount(nmax, m, 1);
    if (r0 >= Ks || (r0 & (BM - 1))) return;  // whole CTA (Ks >= Ka); r0 starts a block
    const int L = lg.L[m], blk = r0 / BM, n0 = m + 2 * r0;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const double* eps_m = lg.eps + eps_off(lg.T, m) - m;
    const double* reps_m = D.reps + eps_off(lg.T, m) - m;
    const double s2m3 = sqrt((double)(2 * m + 3));
    // the checkpoints of this block (blocks after the first; the first starts at n = m)
    const OtfState* ck = blk > 0 ? (const OtfState*)D.ckpt + D.ckoff[m] + (long)(blk - 1) * L : nullptr;
    double acc[2][TM][TN];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) acc[p][i][j] = 0.0;
    for (int l0 = 0; l0 < L; l0 += BK) {
        if (threadIdx.x < BK) {
            const int l = l0 + threadIdx.x;
            if (l < L) {
                const int kN = lg.k0[m] + l;
                const double x = D.mu[kN];
                OtfState st = blk == 0 ? otf_start(m, rg.coslat[kN], D.Qm[m]) : ck[l];
                for (int j = 0; j < 2 * BM; j++) {
                    const int n = n0 + j;
                    double v = 0.0;
                    if (n <= nmax) v = n == m ? otf_value(st) : otf_step(n, m, x, s2m3, eps_m, reps_m, st);
                    As[j & 1][threadIdx.x][j >> 1] = v;
                }
            } else {
                for (int j = 0; j < 2 * BM; j++) As[j & 1][threadIdx.x][j >> 1] = 0.0;
            }
        }
        for (int e = threadIdx.x; e < 2 * BK * BN; e += NT) {
            const int p = e / (BK * BN), r = e % (BK * BN), kk = r / BN, j = r % BN;
            Bs[p][kk][j] = (l0 + kk < L && c0 + j < ncol) ? Gop[(lg.goff[2 * m + p] + l0 + kk) * (long)ncolp + c0 + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 2; p++) {
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                double a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; i++) a[i] = As[p][kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; j++) b[j] = Bs[p][kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; i++)
#pragma unroll
                    for (int j = 0; j < TN; j++) acc[p][i][j] = fma(a[i], b[j], acc[p][i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int K = p ? Ka : Ks;
        double* Sb = Sop + lg.aoff[2 * m + p] * (long)ncolp;
#pragma unroll
        for (int i = 0; i < TM; i++) {
            const int k = r0 + ty * TM + i;
            if (k >= K) continue;
#pragma unroll
            for (int j = 0; j < TN; j++) {
                const int c = c0 + tx * TN + j;
                if (c < ncol) Sb[(long)k * ncolp + c] = acc[p][i][j];
            }
        }
    }
}

int launch_otf_ckpt(Tables* t)
{
    // checkpoint offsets: blocks b = 1 .. (T+1-m)/128 of every m
    std::vector<long> ckoff(t->T + 2, 0);
    for (int m = 0; m <= t->T; m++) ckoff[m + 1] = ckoff[m] + (long)((t->T + 1 - m) / 128) * t->L[m];
    const long n = std::max(ckoff[t->T + 1], 1L);
    if (dev_malloc((void**)&t->d_ckoff, ckoff.size() * sizeof(long)) != cudaSuccess) {
        cudaGetLastError();
        set_error("out of device memory for the Legendre checkpoints");
        return ST_ERR_NOMEM;
    }
    if (dev_malloc(&t->ckpt, n * sizeof(OtfState)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(t->d_ckoff);
        t->d_ckoff = nullptr;
        set_error("out of device memory for the Legendre checkpoints (%.2f GB)", n * sizeof(OtfState) / 1e9);
        return ST_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpy(t->d_ckoff, ckoff.data(), ckoff.size() * sizeof(long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        dim3 grid((t->N + 127) / 128, t->T + 1);
        k_otf_ckpt<<<grid, 128>>>(t->leg(), t->d_mu, t->d_coslat, t->d_Q, t->d_reps, t->d_ckoff, (OtfState*)t->ckpt);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(t->d_ckoff);
        cudaFree(t->ckpt);
        t->d_ckoff = nullptr;
        t->ckpt = nullptr;
        set_error("Legendre checkpoint build: %s", cudaGetErrorString(e));
        return ST_ERR_CUDA;
    }
    t->nckpt = n;
    return ST_OK;
}

template <typename R, int BNT>
__global__ void __launch_bounds__(256) k_leg_inv_simt(const __grid_constant__ LegArgs Ag)
{
    run_items(Ag.q, [&](int w) { leg_inv_simt_item<R, BNT>(Ag, w); });
}
template <typename R, int BNT>
__global__ void __launch_bounds__(256) k_leg_dir_simt(const __grid_constant__ LegArgs Ag)
{
    run_items(Ag.q, [&](int w) { leg_dir_simt_item<R, BNT>(Ag, w); });
}

int persistent_grid(const void* kernel, int threads, int smem, int nwork)
{
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1)
        occ = 1, nsm = nsm > 0 ? nsm : 1;
    const long g = (long)occ * nsm;
    return (int)(g < nwork ? g : nwork);
}

int launch_leg_tc(bool inverse, st_prec prec, const LegArgs& A, int ntiles, int bn, cudaStream_t s);

LegDesc leg_desc(const Plan* p, bool inverse, int nleg, int nmax)
{
    const Tables* t = p->tab;
    LegDesc d;
    memset(&d, 0, sizeof d);
    d.lg = t->leg();
    d.rg = t->ring();
    d.P = p->opts.prec == ST_PREC_FP64 ? (const void*)t->P64 : (const void*)t->P32;
    d.otf = (p->opts.flags & ST_FLAG_OTF) ? 1 : 0;
    d.df = (p->opts.flags & ST_FLAG_DF64) ? 1 : 0;
    d.mu = t->d_mu;
    d.Qm = t->d_Q;
    d.reps = t->d_reps;
    d.ckpt = t->ckpt;
    d.ckoff = t->d_ckoff;
    d.X = inverse ? p->ws_op : p->ws_four;
    d.Y = inverse ? p->ws_four : p->ws_op;
    d.tmP = t->tmaps;
    d.tmX = inverse ? p->amaps : p->gmaps;
    d.status = p->d_status;
    d.wait_limit = p->wait_limit > 0 ? p->wait_limit : ST_WAIT_LIMIT_DEFAULT;
    d.nb = 2 * (t->T + 1);
    d.ncolp = p->ncolp;
    d.ncol = 2 * nleg;
    d.nmax = nmax;
    return d;
}

template <typename R, int BN>
static void simt(bool inverse, const LegArgs& A, int ntiles, cudaStream_t s)
{
    const void* k = inverse ? (const void*)k_leg_inv_simt<R, BN> : (const void*)k_leg_dir_simt<R, BN>;
    const int grid = A.q.ctr ? persistent_grid(k, 256, 0, ntiles) : ntiles;
    if (inverse) k_leg_inv_simt<R, BN><<<grid, 256, 0, s>>>(A);
    else k_leg_dir_simt<R, BN><<<grid, 256, 0, s>>>(A);
}

int launch_leg(bool inverse, st_prec prec, const LegArgs& A, int ntiles, int bn, cudaStream_t s)
{
    if (ntiles <= 0) return ST_OK;
    if (is_split(prec)) return launch_leg_tc(inverse, prec, A, ntiles, bn, s);
    if (A.d0.otf) {  // FP64 plans without a stored table (group launches never take this path)
        if (inverse) {
            if (bn == 32) k_leg_inv_otf<32><<<ntiles, 256, 0, s>>>(A);
            else k_leg_inv_otf<64><<<ntiles, 256, 0, s>>>(A);
        } else {
            if (bn == 32) k_leg_dir_otf<32><<<ntiles, 256, 0, s>>>(A);
            else k_leg_dir_otf<64><<<ntiles, 256, 0, s>>>(A);
        }
        ST_CUDA_TRY(cudaGetLastError());
        return ST_OK;
    }
    if (prec == ST_PREC_FP64 && A.d0.df) {  // double-float contractions (group launches never take this path)
        if (inverse) {
            if (bn == 32) k_leg_inv_df<32><<<ntiles, 256, 0, s>>>(A);
            else k_leg_inv_df<64><<<ntiles, 256, 0, s>>>(A);
        } else {
            if (bn == 32) k_leg_dir_df<32><<<ntiles, 256, 0, s>>>(A);
            else k_leg_dir_df<64><<<ntiles, 256, 0, s>>>(A);
        }
    } else if (prec == ST_PREC_FP64) {
        if (bn == 32) simt<double, 32>(inverse, A, ntiles, s);
        else simt<double, 64>(inverse, A, ntiles, s);
    } else {
        if (bn == 64) simt<float, 64>(inverse, A, ntiles, s);
        else simt<float, 128>(inverse, A, ntiles, s);
    }
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}

float time_leg(bool inverse, st_prec prec, const LegArgs& A, int ntiles, int bn, int reps)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.f;
    float best = 1e30f;
    for (int r = 0; r <= reps; r++) {  // the first run warms up
        cudaEventRecord(e0, 0);
        if (launch_leg(inverse, prec, A, ntiles, bn, 0) != ST_OK) best = -1.f;
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) best = -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && best >= 0.f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

int launch_leg_inv(Plan* p, int nleg, cudaStream_t s)
{
    const int cls = nleg > p->nfld ? 1 : 0;
    LegArgs A;
    memset(&A, 0, sizeof A);
    A.d0 = leg_desc(p, true, nleg, cls ? p->T + 1 : p->T);
    A.tiles = p->d_inv_tiles[cls];
    stage_begin(p, ST_STAGE_LEG_INV, s);
    int rc = launch_leg(true, p->opts.prec, A, p->n_inv_tiles[cls], p->leg_bn[0], s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    stage_end(p, ST_STAGE_LEG_INV, s);
    p->last_launches++;
    return ST_OK;
}

int launch_leg_dir(Plan* p, int nleg, int nmax, cudaStream_t s)
{
    const int cls = nleg > p->nfld ? 1 : 0;
    LegArgs A;
    memset(&A, 0, sizeof A);
    A.d0 = leg_desc(p, false, nleg, nmax);
    A.tiles = p->d_dir_tiles[cls];
    stage_begin(p, ST_STAGE_LEG_DIR, s);
    int rc = launch_leg(false, p->opts.prec, A, p->n_dir_tiles[cls], p->leg_bn[1], s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    stage_end(p, ST_STAGE_LEG_DIR, s);
    p->last_launches++;
    return ST_OK;
}

}  // namespace st
