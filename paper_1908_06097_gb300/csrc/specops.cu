// Spectral-side steps: building the inverse Legendre operand from the
// spectral fields, and scattering the direct Legendre result back to them.
//
// Recurrences used (orthonormal P_n^m, eps_n^m = sqrt((n^2-m^2)/(4n^2-1))):
//   (1-mu^2) dP_n/dmu = -n eps_{n+1} P_{n+1} + (n+1) eps_n P_{n-1}
// so for f = sum_n s_n P_n:
//   (1-mu^2) df/dmu = sum_k b_k P_k,   b_k = (k+2) eps_{k+1} s_{k+1} - (k-1) eps_k s_{k-1},
// with k running to T+1.  Then d f/d phi = b-synthesis / cos(phi).
//   winds   psi = -a zeta/(n(n+1)), chi = -a D/(n(n+1))   (one factor a; the grid
//           scale 1/cos(phi) completes u = (1/a)(...) with the other a^2/a)
//           U = -b[psi] + i m chi,  V = i m psi + b[chi]   (u cos(phi), v cos(phi) / a)
//   direct  zeta = (1/a)(i m c_n[V] + h_n[U]),  D = (1/a)(i m c_n[U] - h_n[V]),
//           h_n[X] = -n eps_{n+1} c_{n+1}[X] + (n+1) eps_n c_{n-1}[X],
//           c_n[X] = sum_k w_k X_m(k) P_n(mu_k) / (1 - mu_k^2)  (degree T+1 rows)
// Each CTA handles 32 consecutive degrees n of one m and 32 fields.  It keeps
// one halo degree on each side in shared memory, so both the strided spectral
// layout and the m-major operand layout are accessed in coalesced runs.
#include <math.h>
#include <string.h>

#include <type_traits>

#include "st_internal.cuh"

namespace st {


__device__ __forceinline__ long coef_off(int T, int m) { return (long)m * (2 * T + 3 - m) / 2; }

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };
template <typename R> __device__ __forceinline__ typename V2<R>::T mk2(R x, R y)
{
    typename V2<R>::T v;
    v.x = x;
    v.y = y;
    return v;
}


template <typename CT> __device__ __forceinline__ CT cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return dbl2flt_rn(x); }
__device__ __forceinline__ void bcoef(const LegGeom& lg, long i, double* cp, double* cm)
{
    const double2 c = lg.bc[i];
    *cp = c.x;
    *cm = c.y;
}
__device__ __forceinline__ void bcoef(const LegGeom& lg, long i, float* cp, float* cm)
{
    const float2 c = lg.bc32[i];
    *cp = c.x;
    *cm = c.y;
}

// (re, im) at columns i, i+1 (i even) of an operand row: one vector store
// per plane (the split of put_split)
template <typename R, typename V>
__device__ __forceinline__ void put_split_pair(R* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long i, V x, V y, int ns)
{
    if (ns == 0) {
        *(typename V2<R>::T*)(p0 + i) = mk2<R>((R)x, (R)y);
        return;
    }
    const float xf = to_flt(x), yf = to_flt(y);
    __nv_bfloat162 a, b, c;
    a.x = __float2bfloat16_rn(xf);
    a.y = __float2bfloat16_rn(yf);
    const float rx = xf - __bfloat162float(a.x), ry = yf - __bfloat162float(a.y);
    b.x = __float2bfloat16_rn(rx);
    b.y = __float2bfloat16_rn(ry);
    *(__nv_bfloat162*)((__nv_bfloat16*)p0 + i) = a;
    *(__nv_bfloat162*)(p1 + i) = b;
    if (ns == 3) {
        c.x = __float2bfloat16_rn(rx - __bfloat162float(b.x));
        c.y = __float2bfloat16_rn(ry - __bfloat162float(b.y));
        *(__nv_bfloat162*)(p2 + i) = c;
    }
}

// mode: PRE_PLAIN (nleg = nf), PRE_HALF (nleg = nf, m > 0 halved),
//       PRE_DERIV (fields nf..2nf-1 = b[a]), PRE_UV (U from (a,b) at 0.., V at nf..)
template <typename R>
__device__ __forceinline__ void pre_item(const SpecArgs& A, int item)
{
    int mb = 0, ci = item, f0 = blockIdx.y * 32;
    if (A.work) {  // group launch: (member, chunk, first field)
        const int4 w = A.work[item];
        mb = w.x;
        ci = w.y;
        f0 = w.z;
    }
    const SpecDesc& D = A.desc ? A.desc[mb] : A.d0;
    const int mode = A.mode, nf = D.nf, T = D.T, nmax = T + A.nmax_extra, ncolp = D.ncolp, split = D.split;
    const double* a = A.pa[mb];
    const double* b = A.pb[mb];
    const double radius = D.radius;
    const LegGeom& lg = D.lg;
    R* aop = (R*)D.op;
    __nv_bfloat16* aop_lo = D.lo;
    __nv_bfloat16* aop_lo2 = D.lo2;
    // the recurrences run in the plan's precision: the rows of the polar rings,
    // where the 1/cos(phi) synthesis scale would amplify their rounding, are
    // recomputed in FP64 by k_polar
    typedef R CT;
    typedef typename V2<CT>::T R2;
    __shared__ R2 sa[32][35];
    __shared__ R2 sb[32][35];
    __shared__ CT fac_n[34];
    const int2 ch = D.chunks[ci];
    const int m = ch.x, n0 = ch.y;
    const long ncoef = (long)(T + 1) * (T + 2) / 2;
    const long off = coef_off(T, m);
    const int nsrc = mode == PRE_UV ? 2 : 1;
    if (mode == PRE_UV && threadIdx.x < 34) {
        // psi, chi = -a x / (n (n+1)) for the 34 degrees of this chunk
        const int n = n0 - 1 + threadIdx.x;
        fac_n[threadIdx.x] = (CT)(n > 0 ? -radius / (double)((long)n * (n + 1)) : 0.0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 34 * nsrc; e += blockDim.x) {
        const int which = e / (32 * 34), r = e % (32 * 34);
        const int fi = r / 34, j = r % 34;
        const int n = n0 - 1 + j, f = f0 + fi;
        const double* src = which ? b : a;
        R2 v = mk2<CT>(0, 0);
        if (f < nf && n >= m && n <= T) {
            const double2 d = *(const double2*)(src + 2 * ((long)f * ncoef + off + (n - m)));
            // ST_FLAG_CHECKS: a non-finite coefficient (Im a_n^0 is not used)
            if (D.checks && !(isfinite(d.x) && (m == 0 || isfinite(d.y)))) atomicMax(D.status, (int)ST_ERR_CHECK);
            v = mk2<CT>(cvt<CT>(d.x), m == 0 ? (CT)0 : cvt<CT>(d.y));
        }
        if (mode == PRE_UV) {
            v.x *= fac_n[j];
            v.y *= fac_n[j];
        }
        (which ? sb : sa)[fi][j] = v;
    }
    __syncthreads();
    const int nout = mode == PRE_DERIV || mode == PRE_UV ? 2 : 1;
    // every operand row up to n = T+1 is written (zeros above nmax), so a
    // kernel that reads whole 64-row slabs never sees a previous call's data
    const int nn_hi = min(n0 + 32, T + 2);
    for (int e = threadIdx.x; e < 32 * 32 * nout; e += blockDim.x) {
        const int cls = e / 1024, r = e % 1024;
        const int fi = r % 32, nn = r / 32;
        const int n = n0 + nn, f = f0 + fi;
        if (n >= nn_hi || f >= nf) continue;
        const int j = nn + 1;  // shared-memory index of degree n
        R2 v;
        if (n > nmax) {
            v = mk2<CT>(0, 0);
        } else if (mode == PRE_PLAIN || mode == PRE_HALF || (mode == PRE_DERIV && cls == 0)) {
            v = sa[fi][j];
            if (mode == PRE_HALF && m > 0) {
                v.x *= (CT)0.5;
                v.y *= (CT)0.5;
            }
        } else {
            CT cp, cm;  // (n+2) eps_{n+1}, (n-1) eps_n
            bcoef(lg, eps_off(T, m) + n - m, &cp, &cm);
            if (mode == PRE_DERIV) {
                v.x = cp * sa[fi][j + 1].x - cm * sa[fi][j - 1].x;
                v.y = cp * sa[fi][j + 1].y - cm * sa[fi][j - 1].y;
            } else {
                const R2 *X = cls == 0 ? sa[fi] : sb[fi], *Y = cls == 0 ? sb[fi] : sa[fi];
                // cls 0: U = -b[psi] + i m chi   (X = psi, Y = chi)
                // cls 1: V =  b[chi] + i m psi   (X = chi, Y = psi)
                const CT sg = cls == 0 ? (CT)-1 : (CT)1, fm = (CT)m;
                const CT bx = cp * X[j + 1].x - cm * X[j - 1].x;
                const CT by = cp * X[j + 1].y - cm * X[j - 1].y;
                v.x = sg * bx - fm * Y[j].y;
                v.y = sg * by + fm * Y[j].x;
            }
        }
        const int fo = f + (cls ? nf : 0);
        const int p = (n - m) & 1, k = (n - m) >> 1;
        const long i = (lg.aoff[2 * m + p] + k) * (long)ncolp + 2 * fo;
        put_split_pair<R>(aop, aop_lo, aop_lo2, i, v.x, v.y, split);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_pre(const __grid_constant__ SpecArgs A)
{
    run_items(A.q, [&](int w) { pre_item<R>(A, w); });
}

// One wind-recombination value before the 1/a factor:
//   v = sg h_n[H] + i m C,  h_n[H] = -n eps_{n+1} H_{n+1} + (n+1) eps_n H_{n-1},
// from the operands Hp = H_{n+1}, Hm = H_{n-1}, C = C_n.  The h recurrence
// cancels, so its products must not be rounded to the operands' precision.
// FP64 operands: in FP64.  FP32 operands: in double-float arithmetic on the
// FP32 ALUs (GB300 issues 64 FP32 operations per FP64 one): every product of
// an FP32 operand with a coefficient hi + lo (hi, lo FP32; from the FP64
// value) is split exactly into p + e by an FMA (Dekker's two-product), sums
// are exact by Knuth's two-sum, and the result is rounded once to FP64.
// the h-recurrence coefficient of degree n: FP64, or hi/lo FP32 pairs
__device__ __forceinline__ double2 hcoef(const LegGeom& lg, long i, double) { return lg.hc[i]; }
__device__ __forceinline__ float4 hcoef(const LegGeom& lg, long i, float) { return lg.hc32[i]; }

__device__ __forceinline__ void wind_recombine(double2 hc, int m, int sg, double2 Hp, double2 Hm,
                                               double2 C, double* vx, double* vy)
{
    // hc: -n eps_{n+1}, (n+1) eps_n
    const double hx = hc.x * Hp.x + hc.y * Hm.x, hy = hc.x * Hp.y + hc.y * Hm.y;
    *vx = -(double)m * C.y + sg * hx;
    *vy = (double)m * C.x + sg * hy;
}
// a * (hi + lo) + b * (hi2 + lo2) + c * d as an unevaluated FP32 pair, then
// to FP64.  The products and sums that must be exact use the _rn intrinsics,
// which the compiler never contracts into FMAs (a contraction would break the
// error-free transformations).
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float z = __fsub_rn(s, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
__device__ __forceinline__ double df_dot3(float a, float hi, float lo, float b, float hi2, float lo2, float c, float d)
{
    const float p1 = __fmul_rn(a, hi), e1 = __fadd_rn(fmaf(a, hi, -p1), __fmul_rn(a, lo));
    const float p2 = __fmul_rn(b, hi2), e2 = __fadd_rn(fmaf(b, hi2, -p2), __fmul_rn(b, lo2));
    const float p3 = __fmul_rn(c, d), e3 = fmaf(c, d, -p3);
    const float s1 = __fadd_rn(p1, p2), t1 = two_sum_err(p1, p2, s1);
    const float s2 = __fadd_rn(s1, p3), t2 = two_sum_err(s1, p3, s2);
    const float lo_sum = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), e3), __fadd_rn(t1, t2));
    return to_dbl(s2) + to_dbl(lo_sum);
}
__device__ __forceinline__ void wind_recombine(float4 h, int m, int sg, float2 Hp, float2 Hm,
                                               float2 C, double* vx, double* vy)
{
    // h: hi/lo of -n eps_{n+1}, (n+1) eps_n
    const float fs = (float)sg, fm = (float)m;  // exact
    // sg h = (sg hp_hi + sg hp_lo) Hp + (sg hm_hi + sg hm_lo) Hm (negation exact)
    *vx = df_dot3(Hp.x, fs * h.x, fs * h.y, Hm.x, fs * h.z, fs * h.w, -fm, C.y);
    *vy = df_dot3(Hp.y, fs * h.x, fs * h.y, Hm.y, fs * h.z, fs * h.w, fm, C.x);
}

// mode: POST_PLAIN, POST_CM (times c_m), POST_UV (a <- zeta, b <- D from U at 0.., V at nf..)
template <typename R>
__device__ __forceinline__ void post_item(const SpecArgs& A, int item)
{
    int mb = 0, ci = item, f0 = blockIdx.y * 32;
    if (A.work) {  // group launch: (member, chunk, first field)
        const int4 w = A.work[item];
        mb = w.x;
        ci = w.y;
        f0 = w.z;
    }
    const SpecDesc& D = A.desc ? A.desc[mb] : A.d0;
    const int mode = A.mode, nf = D.nf, T = D.T, nmax = T + A.nmax_extra, ncolp = D.ncolp;
    double* a = A.pa[mb];
    double* b = A.pb[mb];
    const double inv_radius = 1.0 / D.radius;
    const LegGeom& lg = D.lg;
    const R* sop = (const R*)D.op;
    typedef typename V2<R>::T R2;
    __shared__ R2 su[32][35];
    __shared__ R2 sv[32][35];
    const int2 ch = D.chunks[ci];
    const int m = ch.x, n0 = ch.y;
    if (n0 > T) return;
    const long ncoef = (long)(T + 1) * (T + 2) / 2;
    const long off = coef_off(T, m);
    const int nsrc = mode == POST_UV ? 2 : 1;
    // all loads of the chunk in flight before the first is used (latency:
    // 9 per thread at most)
    constexpr int NLD = (32 * 34 * 2 + 255) / 256;
    const int nload = 32 * 34 * nsrc;
    R2 ld[NLD];
#pragma unroll
    for (int q = 0; q < NLD; q++) {
        const int e = threadIdx.x + q * 256;
        const int which = e / (32 * 34), r = e % (32 * 34);
        const int fi = r % 32, j = r / 32;
        const int n = n0 - 1 + j, f = f0 + fi;
        ld[q] = mk2<R>(0, 0);
        if (e < nload && f < nf && n >= m && n <= nmax) {
            const int p = (n - m) & 1, k = (n - m) >> 1;
            // columns 2 (f + which nf), +1: 8- or 16-byte aligned (ncolp is a multiple of 8)
            ld[q] = *(const R2*)(sop + (lg.aoff[2 * m + p] + k) * (long)ncolp + 2 * (f + which * nf));
        }
    }
#pragma unroll
    for (int q = 0; q < NLD; q++) {
        const int e = threadIdx.x + q * 256;
        if (e >= nload) break;
        const int which = e / (32 * 34), r = e % (32 * 34);
        const int fi = r % 32, j = r / 32;
        (which ? sv : su)[fi][j] = ld[q];
    }
    __syncthreads();
    // the outputs are FP64: the recombination runs in FP64 on the exact
    // FP64 images of the operands (the h recurrence cancels, and rounding
    // its products in FP32 would add to the operands' own rounding)
    const double cmf = (mode == POST_CM && m > 0) ? 2.0 : 1.0;
    const int nout = mode == POST_UV ? 2 : 1;
    for (int e = threadIdx.x; e < 32 * 32 * nout; e += blockDim.x) {
        const int cls = e / 1024, r = e % 1024;
        const int nn = r % 32, fi = r / 32;
        const int n = n0 + nn, f = f0 + fi;
        if (n > T || f >= nf) continue;
        const int j = nn + 1;
        double vx, vy;
        if (mode != POST_UV) {
            vx = to_dbl(su[fi][j].x);
            vy = to_dbl(su[fi][j].y);
            if (cmf != 1.0) {
                vx *= cmf;
                vy *= cmf;
            }
        } else {
            // cls 0: zeta = i m c[V] + h[U];  cls 1: D = i m c[U] - h[V]
            const R2 *H = cls == 0 ? su[fi] : sv[fi], *C = cls == 0 ? sv[fi] : su[fi];
            wind_recombine(hcoef(lg, eps_off(T, m) + n - m, R(0)), m, cls == 0 ? 1 : -1, H[j + 1], H[j - 1], C[j], &vx,
                           &vy);
            if (inv_radius != 1.0) {
                vx *= inv_radius;
                vy *= inv_radius;
            }
        }
        if (m == 0) vy = 0;
        double* dst = cls ? b : a;
        *(double2*)(dst + 2 * ((long)f * ncoef + off + (n - m))) = make_double2(vx, vy);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_post(const __grid_constant__ SpecArgs A)
{
    run_items(A.q, [&](int w) { post_item<R>(A, w); });
}

// ------------------------------------------------- direct winds at m = 1
// FP32 and split plans.  The wind recombination h_n = (n+1) eps_n c_{n-1} -
// n eps_{n+1} c_{n+1} differences neighbouring degrees of the Legendre sums
// c_n; at m = 1 the direct operand of U and V grows like 1/cos(phi) towards
// the poles, its sums vary slowly with n, and h_n keeps about 1e-3 of its
// terms, so rounding errors that are independent from one n to the next
// (those of an FP32 sum and of an FP32 table) come back about 1e3 times
// larger; perturbations of the operand itself do not, being smooth in n.
// This kernel redoes the m = 1 sums from the same FP32 operand in
// double-float: the table P_n^1 as FP32 (hi, lo) pairs from long double, each
// product x (hi + lo) formed exactly up to the x lo term (FMA for the error
// of x hi), each sum by Knuth's two-sum into an FP32 (sum, compensation)
// pair, and the recombination in FP64, overwriting what k_post wrote at
// m = 1.  One CTA: W1R consecutive degrees (the W1O outputs and one
// neighbour on each side) by W1F fields (their U and V columns); thread
// (ty, tx) holds degrees 2ty, 2ty + 1 of the tile (one of each parity) and
// four columns.
constexpr int W1R = 32, W1O = W1R - 2, W1F = 16, W1C = 4 * W1F, W1K = 32;
static_assert(W1O % 2 == 0, "row parity is fixed by the row index only when W1O is even");

struct WindM1Args {
    const float* gop;   // FP32 direct operand: row (row0[p] + l), column 2 (f or nf + f) + re/im
    const float2* pw;   // P_n^1 (hi, lo) at pw[l (T+2) + n]
    const double2* hc;  // (-n eps_{n+1}, (n+1) eps_n) of m = 1 at hc[n - 1]
    double* vor;
    double* div;
    long row0[2];       // first operand row of m = 1: symmetric (even n - 1), antisymmetric
    int nl, ncolp, nf, T;
    double inv_radius;
};

// (s, c) += x (ph + pl): the error of x ph by an FMA, x pl added to it, the
// sum by Knuth's two-sum (the _rn intrinsics are never contracted)
__device__ __forceinline__ void w1_mac(float& s, float& c, float x, float ph, float pl)
{
    const float p = __fmul_rn(x, ph);
    const float e = fmaf(x, pl, fmaf(x, ph, -p));
    const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

__global__ void __launch_bounds__(256) k_wind_m1(const __grid_constant__ WindM1Args A)
{
    __shared__ __align__(16) float2 sp[W1K][W1R];
    __shared__ __align__(16) float sx[2][W1K][W1C];  // [parity][ring][tile column]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int n0 = 1 + blockIdx.x * W1O;  // tile row r holds degree n0 - 1 + r
    const int f0 = blockIdx.y * W1F, NP = A.T + 2;
    // row 2ty: n - 1 odd (antisymmetric rows); row 2ty + 1: n - 1 even
    float sh[2][4], sl[2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) sh[i][j] = sl[i][j] = 0.f;
    for (int lb = 0; lb < A.nl; lb += W1K) {
        for (int e = tid; e < W1K * W1R; e += 256) {
            const int kk = e / W1R, r = e % W1R, l = lb + kk, n = n0 - 1 + r;
            sp[kk][r] = (l < A.nl && n >= 1 && n <= A.T + 1) ? A.pw[(long)l * NP + n] : make_float2(0.f, 0.f);
        }
        // tile column c: U of fields f0 + c/2 (c < 2 W1F), then V; re/im = c & 1
        for (int e = tid; e < 2 * W1K * W1C; e += 256) {
            const int par = e / (W1K * W1C), rem = e % (W1K * W1C), kk = rem / W1C, c = rem % W1C;
            const int l = lb + kk, f = f0 + (c % (2 * W1F)) / 2;
            float v = 0.f;
            if (l < A.nl && f < A.nf)
                v = A.gop[(A.row0[par] + l) * (long)A.ncolp + 2 * ((c < 2 * W1F ? 0 : A.nf) + f) + (c & 1)];
            sx[par][kk][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < W1K; kk++) {
            const float4 pp = *(const float4*)&sp[kk][2 * ty];
            const float4 xa = *(const float4*)&sx[1][kk][4 * tx];
            const float4 xs = *(const float4*)&sx[0][kk][4 * tx];
            w1_mac(sh[0][0], sl[0][0], xa.x, pp.x, pp.y);
            w1_mac(sh[0][1], sl[0][1], xa.y, pp.x, pp.y);
            w1_mac(sh[0][2], sl[0][2], xa.z, pp.x, pp.y);
            w1_mac(sh[0][3], sl[0][3], xa.w, pp.x, pp.y);
            w1_mac(sh[1][0], sl[1][0], xs.x, pp.z, pp.w);
            w1_mac(sh[1][1], sl[1][1], xs.y, pp.z, pp.w);
            w1_mac(sh[1][2], sl[1][2], xs.z, pp.z, pp.w);
            w1_mac(sh[1][3], sl[1][3], xs.w, pp.z, pp.w);
        }
        __syncthreads();
    }
    // the sums c_n as FP64, [row][tile column], in the staging area
    double(*cs)[W1C] = reinterpret_cast<double(*)[W1C]>(&sx[0][0][0]);
    static_assert(sizeof(sx) == W1R * W1C * sizeof(double), "the sums fill the operand staging area");
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) cs[2 * ty + i][4 * tx + j] = (double)sh[i][j] + (double)sl[i][j];
    __syncthreads();
    // zeta = i c_n[V] + h_n[U], D = i c_n[U] - h_n[V] (m = 1)
    const long ncoef = (long)(A.T + 1) * (A.T + 2) / 2, off = coef_off(A.T, 1);
    for (int e = tid; e < 2 * W1F * W1O; e += 256) {
        const int cls = e / (W1F * W1O), rem = e % (W1F * W1O), fi = rem / W1O, j = rem % W1O;
        const int n = n0 + j, f = f0 + fi, r = j + 1;
        if (n > A.T || f >= A.nf) continue;
        const int hcol = (cls == 0 ? 0 : 2 * W1F) + 2 * fi, ccol = (cls == 0 ? 2 * W1F : 0) + 2 * fi;
        const double2 h = A.hc[n - 1];
        const double sg = cls == 0 ? 1.0 : -1.0;
        const double hx = h.x * cs[r + 1][hcol] + h.y * cs[r - 1][hcol];
        const double hy = h.x * cs[r + 1][hcol + 1] + h.y * cs[r - 1][hcol + 1];
        double vx = -cs[r][ccol + 1] + sg * hx, vy = cs[r][ccol] + sg * hy;
        if (A.inv_radius != 1.0) {
            vx *= A.inv_radius;
            vy *= A.inv_radius;
        }
        double* dst = cls ? A.div : A.vor;
        *(double2*)(dst + 2 * ((long)f * ncoef + off + (n - 1))) = make_double2(vx, vy);
    }
}

// ------------------------------------------------------------- polar rings
// The syntheses that end in a 1/cos(phi) factor (d/dphi, the winds) lose
// accuracy on the polar rings when they are formed as the Legendre kernels
// form them: the recurrence (n+2) eps_{n+1} X_{n+1} - (n-1) eps_n X_{n-1} of
// the operand has terms about 5000 times the synthesised value on the first
// O1280 ring, which is O(cos(phi)) before the 1/cos(phi) (about 1600) scales
// it, so the operand's rounding comes back amplified.  For the rings with
// cos(phi) < ST_POLAR_COS, this kernel recomputes the Fourier rows of those
// classes from the FP64 spectral input and overwrites what the Legendre
// kernel wrote.  It sums the terms X_n G_n^m instead, G_n^m = (n+1) eps_n
// P_{n-1}^m - n eps_{n+1} P_{n+1}^m = cos(phi) dP_n^m/dphi, from a table formed
// in long double on the host (beside the table of P_n^m, both at the
// long-double Gauss nodes), so that no term exceeds the sum by that factor.
// FP64 plans go further, so that the polar rings reach what long-double
// evaluation of the definition gives: the degree sums are accumulated in
// double-double (every product exact by an FMA, every sum exact by Knuth's
// two-sum, one rounding at the end), and the plain field's rows (grid and
// d/dlambda) are recomputed too, from the long-double table instead of the
// FP64 recurrence table.  FP32 and split plans sum in FP32 from FP32 copies of
// the tables.  One thread per (field, group of up to PG polar rings) of one m.
// Partitioned plans (mown set) recompute only the rows of their own m.
constexpr int PG = 4;
// The degree loop of one (m, field, ring group) is split into PCH chunks run
// by PCH threads (threadIdx.y), whose partial sums are added in shared
// memory: the loop is a few thousand dependent FP64 operations, and one
// thread per (field, group) would leave most SMs with a handful of warps.
constexpr int PCH = 4, PNT = 64;

// s + c += x * y exactly up to the final rounding of s + c (double-double)
__device__ __forceinline__ void dd_fma(double& s, double& c, double x, double y)
{
    const double p = __dmul_rn(x, y), pe = __fma_rn(x, y, -p);
    const double t = __dadd_rn(s, p), z = __dsub_rn(t, s);
    const double te = __dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(p, z));
    s = t;
    c = __dadd_rn(c, __dadd_rn(te, pe));
}
__device__ __forceinline__ void dd_add(double& s, double& c, double s2, double c2)
{
    const double t = __dadd_rn(s, s2), z = __dsub_rn(t, s);
    const double te = __dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(s2, z));
    s = t;
    c = __dadd_rn(c, __dadd_rn(te, c2));
}

// Outputs per mode: PRE_PLAIN: the field (column 2f); PRE_DERIV: d/dphi
// (column 2(nf+f)) and, with plain, the field; PRE_UV: U (2f) and V (2(nf+f)).
// Accumulator k (0..3): e1 re, e1 im, o1 re, o1 im of output 1, then 4..7 of
// output 2 (e: even n - m, o: odd; north = e + o, south = e - o).
// (FP64 plans: one block per SM, the double-double sums need the registers)
template <typename R>
__global__ void __launch_bounds__(PNT * PCH, sizeof(R) == 8 ? 1 : 2) k_polar(int mode, int plain, const double* __restrict__ a,
                                                     const double* __restrict__ b, int nf, int T, double radius,
                                                     LegGeom lg, RingGeom rg, PolarGeom pg, R* __restrict__ four,
                                                     int ncolp, const unsigned char* __restrict__ mown)
{
    constexpr bool DD = sizeof(R) == 8;  // FP64 plans: double-double sums
    constexpr int NS = DD ? 16 : 8;      // partial sums per ring (with DD their compensations)
    // partial sums of chunks 1..PCH-1: [chunk-1][thread][ring][NS] (dynamic: 96 KB with DD)
    extern __shared__ double part_raw[];
    auto part = [&](int cc, int th, int r) { return part_raw + (((long)cc * PNT + th) * PG + r) * NS; };
    const int m = blockIdx.x;
    if (mown && !mown[m]) return;
    int k0 = 0;  // the polar rings carrying m: mmax grows towards the equator
    while (k0 < pg.np && rg.mmax[k0] < m) k0++;
    const int nk = pg.np - k0, ng = (nk + PG - 1) / PG;
    if (nk <= 0) return;
    const long ncoef = (long)(T + 1) * (T + 2) / 2;
    const long off = coef_off(T, m);
    const double fm = (double)m;
    const bool uv = mode == PRE_UV, deriv = mode == PRE_DERIV;
    const bool two = uv || (deriv && plain);  // a second output
    // degrees n = m .. T+1 in PCH contiguous chunks
    const int nlen = T + 2 - m, clen = (nlen + PCH - 1) / PCH;
    const int c = threadIdx.y, nb = m + c * clen, ne = min(nb + clen, T + 2);
    const int nwork = nf * ng, nslab = (nwork + PNT - 1) / PNT;
    // every thread of the block runs the same slab iterations (the barriers)
    for (int sl = blockIdx.y; sl < nslab; sl += gridDim.y) {
        const int idx = sl * PNT + threadIdx.x;
        const bool live = idx < nwork;
        const int f = live ? idx % nf : 0, kb = k0 + (live ? idx / nf : 0) * PG, nr = min(PG, pg.np - kb);
        const double* P[PG];
        const double* G[PG];  // DD: G_n^m of the same rings
#pragma unroll
        for (int r = 0; r < PG; r++) {
            const long o = pg.poff[(long)(kb + min(r, nr - 1)) * (T + 1) + m] - m;
            P[r] = pg.pt + o;
            G[r] = pg.gt + o;
        }
        const double2* sa = (const double2*)(a + 2 * ((long)f * ncoef + off)) - m;  // sa[n]
        const double2* sb = uv ? (const double2*)(b + 2 * ((long)f * ncoef + off)) - m : nullptr;
        // X_n (Y_n for the winds), zero outside [m, T]; Im of m = 0 ignored;
        // psi, chi = -a X / (n (n+1)) for the winds
        auto ld = [&](const double2* src, int n) {
            if (n < m || n > T) return make_double2(0.0, 0.0);
            double2 v = src[n];
            if (m == 0) v.y = 0.0;
            if (uv) {
                const double fac = radius * pg.fac[n];
                v.x *= fac;
                v.y *= fac;
            }
            return v;
        };
        double acc[PG][8], cmp[PG][8];  // sums and (DD) their compensations
#pragma unroll
        for (int r = 0; r < PG; r++)
#pragma unroll
            for (int q = 0; q < 8; q++) acc[r][q] = cmp[r][q] = 0.0;
        if (live && DD) {
            double2 x0 = ld(sa, nb), y0 = uv ? ld(sb, nb) : make_double2(0, 0);
            for (int n = nb; n < ne; n++) {
                // x_n P_n and x_n G_n terms.  G_n^m has the parity of n - m + 1
                // in mu, so its products go to the other (even, odd) sums than
                // the P products of the same n.
                auto add = [&](auto O) {
                    constexpr int o = decltype(O)::value, og = 2 - o;
#pragma unroll
                    for (int r = 0; r < PG; r++) {
                        const double pn = P[r][n];
                        if (mode == PRE_PLAIN) {
                            dd_fma(acc[r][o], cmp[r][o], x0.x, pn);
                            dd_fma(acc[r][o + 1], cmp[r][o + 1], x0.y, pn);
                        } else if (!uv) {  // d/dphi: x G; with plain, the field: x P
                            const double gn = G[r][n];
                            dd_fma(acc[r][og], cmp[r][og], x0.x, gn);
                            dd_fma(acc[r][og + 1], cmp[r][og + 1], x0.y, gn);
                            if (two) {
                                dd_fma(acc[r][4 + o], cmp[r][4 + o], x0.x, pn);
                                dd_fma(acc[r][5 + o], cmp[r][5 + o], x0.y, pn);
                            }
                        } else {  // U = -psi G + i m chi P, V = chi G + i m psi P
                            const double gn = G[r][n];
                            dd_fma(acc[r][og], cmp[r][og], -x0.x, gn);
                            dd_fma(acc[r][og + 1], cmp[r][og + 1], -x0.y, gn);
                            dd_fma(acc[r][o], cmp[r][o], -fm * y0.y, pn);
                            dd_fma(acc[r][o + 1], cmp[r][o + 1], fm * y0.x, pn);
                            dd_fma(acc[r][4 + og], cmp[r][4 + og], y0.x, gn);
                            dd_fma(acc[r][5 + og], cmp[r][5 + og], y0.y, gn);
                            dd_fma(acc[r][4 + o], cmp[r][4 + o], -fm * x0.y, pn);
                            dd_fma(acc[r][5 + o], cmp[r][5 + o], fm * x0.x, pn);
                        }
                    }
                };
                if ((n - m) & 1) add(std::integral_constant<int, 2>());
                else add(std::integral_constant<int, 0>());
                x0 = ld(sa, n + 1);
                if (uv) y0 = ld(sb, n + 1);
            }
        }
        if (live && !DD) {
            // FP32 and split plans: the same x P and x G terms in FP32.  With G
            // taking the derivative, no term exceeds the sum by the 1/cos(phi)
            // factor, so FP32 products and sums keep the rows near 1e-6 of the
            // result; the FP32 tables are copies of the long-double ones.
            const float* P32[PG];
            const float* G32[PG];
#pragma unroll
            for (int r = 0; r < PG; r++) {
                const long o = pg.poff[(long)(kb + min(r, nr - 1)) * (T + 1) + m] - m;
                P32[r] = pg.pt32 + o;
                G32[r] = pg.gt32 + o;
            }
            const float rad = (float)radius, fmf = (float)m;
            // X_n as FP32 (integer conversion), times -a / (n (n+1)) for the winds
            auto ldf = [&](const double2* src, int n) {
                if (n < m || n > T) return make_float2(0.f, 0.f);
                const double2 v = src[n];
                float2 r = make_float2(dbl2flt_rn(v.x), m == 0 ? 0.f : dbl2flt_rn(v.y));
                if (uv) {
                    const float fac = rad * pg.fac32[n];
                    r.x *= fac;
                    r.y *= fac;
                }
                return r;
            };
            float fa[PG][8];
#pragma unroll
            for (int r = 0; r < PG; r++)
#pragma unroll
                for (int q = 0; q < 8; q++) fa[r][q] = 0.f;
            for (int n = nb; n < ne; n++) {
                const float2 x = ldf(sa, n), y = uv ? ldf(sb, n) : make_float2(0.f, 0.f);
                auto add = [&](auto O) {
                    constexpr int o = decltype(O)::value, og = 2 - o;
#pragma unroll
                    for (int r = 0; r < PG; r++) {
                        const float pn = P32[r][n], gn = G32[r][n];
                        if (!uv) {  // d/dphi: x G; with plain, the field: x P
                            fa[r][og] = fmaf(x.x, gn, fa[r][og]);
                            fa[r][og + 1] = fmaf(x.y, gn, fa[r][og + 1]);
                            if (two) {
                                fa[r][4 + o] = fmaf(x.x, pn, fa[r][4 + o]);
                                fa[r][5 + o] = fmaf(x.y, pn, fa[r][5 + o]);
                            }
                        } else {  // U = -psi G + i m chi P, V = chi G + i m psi P
                            fa[r][og] = fmaf(-x.x, gn, fa[r][og]);
                            fa[r][og + 1] = fmaf(-x.y, gn, fa[r][og + 1]);
                            fa[r][o] = fmaf(-fmf * y.y, pn, fa[r][o]);
                            fa[r][o + 1] = fmaf(fmf * y.x, pn, fa[r][o + 1]);
                            fa[r][4 + og] = fmaf(y.x, gn, fa[r][4 + og]);
                            fa[r][5 + og] = fmaf(y.y, gn, fa[r][5 + og]);
                            fa[r][4 + o] = fmaf(-fmf * x.y, pn, fa[r][4 + o]);
                            fa[r][5 + o] = fmaf(fmf * x.x, pn, fa[r][5 + o]);
                        }
                    }
                };
                if ((n - m) & 1) add(std::integral_constant<int, 2>());
                else add(std::integral_constant<int, 0>());
            }
#pragma unroll
            for (int r = 0; r < PG; r++)
#pragma unroll
                for (int q = 0; q < 8; q++) acc[r][q] = (double)fa[r][q];
        }
        if (c > 0) {
#pragma unroll
            for (int r = 0; r < PG; r++) {
                double* q = part(c - 1, threadIdx.x, r);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    q[k] = acc[r][k];
                    if (DD) q[8 + k] = cmp[r][k];
                }
            }
        }
        __syncthreads();
        if (c == 0 && live) {
            // chunk sums in chunk order
            for (int cc = 0; cc < PCH - 1; cc++) {
#pragma unroll
                for (int r = 0; r < PG; r++) {
                    const double* q = part(cc, threadIdx.x, r);
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        if (DD) dd_add(acc[r][k], cmp[r][k], q[k], q[8 + k]);
                        else acc[r][k] += q[k];
                    }
                }
            }
            // output columns: output 1 (u) and output 2 (v)
            const int c1 = mode == PRE_DERIV ? 2 * (nf + f) : 2 * f;
            const int c2 = uv ? 2 * (nf + f) : 2 * f;
#pragma unroll
            for (int r = 0; r < PG; r++) {
                if (r >= nr) break;
                const int k = kb + r, kS = lg.nlat - 1 - k;
                R* rn = four + (rg.foff[k] + m) * (long)ncolp;
                R* rs = four + (rg.foff[kS] + m) * (long)ncolp;
                double e[8];  // (north, south) from the (even, odd) sums, rounded once
#pragma unroll
                for (int q = 0; q < 8; q += 4) {
                    double sr = acc[r][q], sr_c = cmp[r][q], si = acc[r][q + 1], si_c = cmp[r][q + 1];
                    double ar = acc[r][q + 2], ar_c = cmp[r][q + 2], ai = acc[r][q + 3], ai_c = cmp[r][q + 3];
                    if (DD) {
                        double nr_s = sr, nr_c = sr_c, sr2 = sr, sr2_c = sr_c;
                        dd_add(nr_s, nr_c, ar, ar_c);
                        dd_add(sr2, sr2_c, -ar, -ar_c);
                        double ni_s = si, ni_c = si_c, si2 = si, si2_c = si_c;
                        dd_add(ni_s, ni_c, ai, ai_c);
                        dd_add(si2, si2_c, -ai, -ai_c);
                        e[q] = nr_s + nr_c;
                        e[q + 1] = ni_s + ni_c;
                        e[q + 2] = sr2 + sr2_c;
                        e[q + 3] = si2 + si2_c;
                    } else {
                        e[q] = sr + ar;
                        e[q + 1] = si + ai;
                        e[q + 2] = sr - ar;
                        e[q + 3] = si - ai;
                    }
                }
                rn[c1] = (R)e[0];
                rn[c1 + 1] = (R)e[1];
                rs[c1] = (R)e[2];
                rs[c1 + 1] = (R)e[3];
                if (two) {
                    rn[c2] = (R)e[4];
                    rn[c2 + 1] = (R)e[5];
                    rs[c2] = (R)e[6];
                    rs[c2 + 1] = (R)e[7];
                }
            }
        }
        __syncthreads();  // part is reused by the next slab
    }
}

int launch_polar(Plan* p, PreMode mode, const double* a, const double* b, cudaStream_t s)
{
    const Tables* t = p->tab;
    if (t->npolar <= 0) return ST_OK;
    const bool f64 = p->opts.prec == ST_PREC_FP64;
    if (mode == PRE_PLAIN && !f64) return ST_OK;  // the plain rows need no recomputation below FP64
    const int mmax_p = t->mmax[t->npolar - 1];
    // small blocks: the work is a few hundred thousand long FP64 loops, spread
    // over every SM
    const int ng = (t->npolar + PG - 1) / PG;
    dim3 grid(mmax_p + 1, (p->nfld * ng + PNT - 1) / PNT), block(PNT, PCH);
    const int smem = (PCH - 1) * PNT * PG * (f64 ? 16 : 8) * (int)sizeof(double);
    static bool ready = false;
    if (!ready) {
        ST_CUDA_TRY(cudaFuncSetAttribute(k_polar<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (PCH - 1) * PNT * PG * 16 * (int)sizeof(double)));
        ready = true;
    }
    stage_begin(p, ST_STAGE_LEG_INV, s);
    const unsigned char* mown = p->part ? p->part->d_mown : nullptr;
    if (f64)
        k_polar<double><<<grid, block, smem, s>>>((int)mode, 1, a, b, p->nfld, p->T, p->opts.radius, t->leg(),
                                                   t->ring(), t->polar(), (double*)p->ws_four, p->ncolp, mown);
    else
        k_polar<float><<<grid, block, smem, s>>>((int)mode, 0, a, b, p->nfld, p->T, p->opts.radius, t->leg(),
                                                  t->ring(), t->polar(), (float*)p->ws_four, p->ncolp, mown);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        stage_fail(p);
        set_error("k_polar launch: %s", cudaGetErrorString(e));
        return ST_ERR_CUDA;
    }
    stage_end(p, ST_STAGE_LEG_INV, s);
    p->last_launches++;
    return ST_OK;
}

SpecDesc spec_desc(const Plan* p)
{
    SpecDesc d;
    memset(&d, 0, sizeof d);
    d.lg = p->tab->leg();
    d.chunks = p->d_spec_chunks;
    d.op = p->ws_op;
    d.lo = (__nv_bfloat16*)p->ws_op_lo;
    d.lo2 = (__nv_bfloat16*)p->ws_op_lo2;
    d.radius = p->opts.radius;
    d.status = p->d_status;
    d.checks = (p->opts.flags & ST_FLAG_CHECKS) ? 1 : 0;
    d.T = p->T;
    d.ncolp = p->ncolp;
    d.split = nsplit(p->opts.prec);
    d.nf = p->nfld;
    return d;
}

int launch_spec(bool pre, st_prec prec, const SpecArgs& A, dim3 grid, cudaStream_t s)
{
    if (A.q.ctr) {  // persistent (group launches): grid.x items
        const void* k = pre ? (prec == ST_PREC_FP64 ? (const void*)k_pre<double> : (const void*)k_pre<float>)
                            : (prec == ST_PREC_FP64 ? (const void*)k_post<double> : (const void*)k_post<float>);
        grid = dim3(persistent_grid(k, 256, 0, (int)grid.x), 1);
    }
    if (pre) {
        if (prec == ST_PREC_FP64) k_pre<double><<<grid, 256, 0, s>>>(A);
        else k_pre<float><<<grid, 256, 0, s>>>(A);
    } else {
        if (prec == ST_PREC_FP64) k_post<double><<<grid, 256, 0, s>>>(A);
        else k_post<float><<<grid, 256, 0, s>>>(A);
    }
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}

int launch_pre(Plan* p, PreMode mode, const double* a, const double* b, int nf, cudaStream_t s)
{
    if (p->n_spec_chunks <= 0) return ST_OK;  // a partition that owns no wavenumber
    SpecArgs A;
    memset(&A, 0, sizeof A);
    A.d0 = spec_desc(p);
    A.d0.nf = nf;
    A.mode = (int)mode;
    A.nmax_extra = (mode == PRE_DERIV || mode == PRE_UV) ? 1 : 0;
    A.pa[0] = const_cast<double*>(a);
    A.pb[0] = const_cast<double*>(b);
    stage_begin(p, ST_STAGE_PRE, s);
    int rc = launch_spec(true, p->opts.prec, A, dim3(p->n_spec_chunks, (nf + 31) / 32), s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    stage_end(p, ST_STAGE_PRE, s);
    p->last_launches++;
    return ST_OK;
}

int launch_post(Plan* p, PostMode mode, double* a, double* b, int nf, cudaStream_t s)
{
    if (p->n_spec_chunks <= 0) return ST_OK;
    SpecArgs A;
    memset(&A, 0, sizeof A);
    A.d0 = spec_desc(p);
    A.d0.nf = nf;
    A.mode = (int)mode;
    A.nmax_extra = mode == POST_UV ? 1 : 0;
    A.pa[0] = a;
    A.pb[0] = b;
    stage_begin(p, ST_STAGE_POST, s);
    int rc = launch_spec(false, p->opts.prec, A, dim3(p->n_spec_chunks, (nf + 31) / 32), s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    stage_end(p, ST_STAGE_POST, s);
    p->last_launches++;
    return ST_OK;
}

int launch_wind_m1(Plan* p, double* vor, double* div, cudaStream_t s)
{
    const Tables* t = p->tab;
    // FP64 plans meet their gate at m = 1 as they are; partitioned plans
    // transform only their halves
    if (p->opts.prec == ST_PREC_FP64 || p->T < 1 || p->part || p->nfld <= 0) return ST_OK;
    if (!t->d_pw1) {
        set_error("launch_wind_m1: the m = 1 table of T=%d was not built", p->T);
        return ST_ERR_UNSUPPORTED;
    }
    WindM1Args A;
    memset(&A, 0, sizeof A);
    A.gop = (const float*)(is_split(p->opts.prec) ? p->ws_gop32 : p->ws_four);
    A.pw = t->d_pw1;
    A.hc = t->d_hc + eps_off(p->T, 1);
    A.vor = vor;
    A.div = div;
    A.row0[0] = t->goff[2];
    A.row0[1] = t->goff[3];
    A.nl = t->L[1];
    A.ncolp = p->ncolp;
    A.nf = p->nfld;
    A.T = p->T;
    A.inv_radius = 1.0 / p->opts.radius;
    const dim3 grid((p->T + W1O - 1) / W1O, (p->nfld + W1F - 1) / W1F);
    stage_begin(p, ST_STAGE_POST, s);
    k_wind_m1<<<grid, 256, 0, s>>>(A);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        stage_fail(p);
        set_error("k_wind_m1 launch: %s", cudaGetErrorString(e));
        return ST_ERR_CUDA;
    }
    stage_end(p, ST_STAGE_POST, s);
    p->last_launches++;
    return ST_OK;
}

}  // namespace st
