// Ring-FFT device code of the spectral transform (latitude rings of uneven
// length), included by one translation unit per kernel and precision.
//
// A north ring and its southern mirror have the same length n = nlon (even)
// and carry the same wavenumbers m < K = mmax + 1.  One CTA slot transforms
// the pair as ONE complex sequence, and only the 2K - 1 wavenumbers
// -(K-1) .. K-1 of the pair are touched.  With the chirp
// c_t = exp(i pi t^2 / n) (period n in t because n is even):
//   direct   z_j = f_N(j) + i f_S(j),  j < n,
//            Z_m = conj(c_m) sum_j (z_j conj(c_j)) c_{m-j},           |m| < K,
//            F_N(m) = (Z_m + conj Z_{-m}) / 2,  F_S(m) = (Z_m - conj Z_{-m}) / 2i;
//   inverse  Y_m = H_N(m) + i H_S(m), H(m) = F_m, H(-m) = conj F_m,  |m| < K,
//            g_j = c_j sum_m (Y_m c_m) conj(c_{j-m}),  f_N = Re g, f_S = Im g.
// Both sums are circular convolutions of length M = 2^a >= n + 2K - 2, which
// holds every index difference j - m without wrap-around (chirp-z, Bluestein).
// The direct kernel b_t = c_t, t in [-(n+K-2), K-1], has the precomputed
// transform B = FFT_M(b)/M; the inverse kernel is conj(b_{-t}), whose
// transform is conj(B), so one table serves both directions.
//
// The length-M FFTs run in registers: every thread holds P points (P = 32 in
// FP32, 16 in FP64) and a transform uses M/P threads.  The length is split into
// NST stages of radix <= P (13 = 5+4+4 bits in FP32).  Forward stages are
// decimation in frequency (natural order in, digit-reversed out), inverse
// stages decimation in time (digit-reversed in, natural out), so no
// permutation is ever done and the filter is stored in the digit-reversed
// order.  The last forward stage, the filter product and the first inverse
// stage share registers.  Stages exchange data through shared memory, padded
// by one element every 16, which keeps every exchange of the long transforms
// free of bank conflicts.  A CTA covers 8192 points: one transform of length
// 8192, or 8192/M shorter ones (consecutive fields of a ring pair).
//
// Fusions (the transposition of the paper's all-to-all, Sec. 3.1.3, done as a
// change of layout):
//   c2r  reads the ring-major Fourier buffer four[ring][m][col] that the
//        Legendre epilogue wrote; applies i*m for d/dlambda and a per-ring
//        scale (1/cos(phi), or w/nlon for the adjoint); writes both rings of
//        the grid.
//   r2c  reads both rings of the grid, separates the two spectra and folds
//        them, G_s = s (F_N + F_S) and G_a = s (F_N - F_S), with the per-ring
//        scale s (w/nlon, w/(nlon cos(phi)) or 1).  It writes the m-major
//        direct Legendre operand; on the split paths in FP32, which
//        k_split_gop then splits into bf16 planes with coalesced accesses
//        (the rows of one transform are far apart, so one FP32 store per row
//        costs a third of one store per plane).
#pragma once
#include "st_internal.cuh"

namespace st {
namespace fft {

template <typename R> struct Cx;
template <> struct Cx<double> { typedef double2 T; };
template <> struct Cx<float> { typedef float2 T; };
template <typename C> struct ReT;
template <> struct ReT<double2> { typedef double T; };
template <> struct ReT<float2> { typedef float T; };

template <typename C> __device__ __forceinline__ C cx(typename ReT<C>::T a, typename ReT<C>::T b)
{
    C r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cx<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return cx<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C conjg(C a) { return cx<C>(a.x, -a.y); }

// cos(2 pi k / 32) for k = 0..8 (the first quadrant), then by symmetry
__host__ __device__ constexpr double cos32q(int k)
{
    return k == 0 ? 1.0
         : k == 1 ? 0.98078528040323044913
         : k == 2 ? 0.92387953251128675613
         : k == 3 ? 0.83146961230254523708
         : k == 4 ? 0.70710678118654752440
         : k == 5 ? 0.55557023301960222474
         : k == 6 ? 0.38268343236508977173
         : k == 7 ? 0.19509032201612826785
                  : 0.0;
}
__host__ __device__ constexpr double cos32(int k)
{
    return (k & 31) <= 8 ? cos32q(k & 31)
         : (k & 31) <= 16 ? -cos32q(16 - (k & 31))
         : (k & 31) <= 24 ? -cos32q((k & 31) - 16)
                          : cos32q(32 - (k & 31));
}
__host__ __device__ constexpr double sin32(int k) { return cos32(k - 8); }

// x * exp(SIGN 2 pi i e / 32).  e is a constant after unrolling, so the
// branches fold and the trivial rotations cost no multiplication.
template <int SIGN, typename C> __device__ __forceinline__ C rot(C x, int e)
{
    typedef typename ReT<C>::T R;
    e &= 31;
    if (e == 0) return x;
    if (e == 16) return cx<C>(-x.x, -x.y);
    if (e == 8) return SIGN > 0 ? cx<C>(-x.y, x.x) : cx<C>(x.y, -x.x);
    if (e == 24) return SIGN > 0 ? cx<C>(x.y, -x.x) : cx<C>(-x.y, x.x);
    const double c = cos32(e), s = SIGN * sin32(e);
    if ((e & 7) == 4) {
        const R h = (R)0.70710678118654752440;
        const R re = (c > 0 ? x.x : -x.x) - (s > 0 ? x.y : -x.y);
        const R im = (s > 0 ? x.x : -x.x) + (c > 0 ? x.y : -x.y);
        return cx<C>(re * h, im * h);
    }
    return cx<C>(x.x * (R)c - x.y * (R)s, x.x * (R)s + x.y * (R)c);
}

// In-register N-point DFTs (N = 1..32, power of two), in place, kernel
// exp(SIGN 2 pi i r k / N), as iterative radix-2 networks:
//   dft_dif  natural order in, X[k] left in register brev(k);
//   dft_dit  input r taken from register brev(r), natural order out.
// The bit reversal is a relabelling of registers, fixed at compile time.
__host__ __device__ constexpr int brev(int k, int N)
{
    int r = 0;
    for (int b = 1; b < N; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

template <int N, int SIGN, typename C>
__device__ __forceinline__ void dft_dif(C* v)
{
#pragma unroll
    for (int s = N; s >= 2; s >>= 1) {
#pragma unroll
        for (int b = 0; b < N; b += s) {
#pragma unroll
            for (int j = 0; j < s / 2; j++) {
                const C a = v[b + j], c = v[b + j + s / 2];
                v[b + j] = cx<C>(a.x + c.x, a.y + c.y);
                v[b + j + s / 2] = rot<SIGN>(cx<C>(a.x - c.x, a.y - c.y), j * (32 / s));
            }
        }
    }
}

template <int N, int SIGN, typename C>
__device__ __forceinline__ void dft_dit(C* v)
{
#pragma unroll
    for (int s = 2; s <= N; s <<= 1) {
#pragma unroll
        for (int b = 0; b < N; b += s) {
#pragma unroll
            for (int j = 0; j < s / 2; j++) {
                const C a = v[b + j], c = rot<SIGN>(v[b + j + s / 2], j * (32 / s));
                v[b + j] = cx<C>(a.x + c.x, a.y + c.y);
                v[b + j + s / 2] = cx<C>(a.x - c.x, a.y - c.y);
            }
        }
    }
}

// Twiddles of a stage of span L = 2^logL and radix R = 2^lr (lr <= 5) are
// stored [k][j] = exp(-2 pi i j k / L), j < L/R, so a warp reads them
// contiguously.  Block (logL, lr) starts at 5 (2^logL - 2) + (lr - 1) 2^logL.
__host__ __device__ inline long tw_off(int logL, int lr) { return 5L * ((1L << logL) - 2) + (long)(lr - 1) * (1L << logL); }

// shared-memory position with one pad element every 16
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
// (a CTA's point count depends on the precision, see KC below)

// Stage plan of a length-2^LOGM transform with 2^LOGP points per thread.
template <int LOGM, int LOGP>
struct Geo {
    static constexpr int M = 1 << LOGM, P = 1 << LOGP, T = M / P;
    static constexpr int NST = (LOGM + LOGP - 1) / LOGP;
    static constexpr int lr(int s) { return LOGM / NST + (s < LOGM % NST ? 1 : 0); }
    static constexpr int logL(int s)
    {
        int l = LOGM;
        for (int i = 0; i < s; i++) l -= lr(i);
        return l;
    }
};

// Butterflies of stage S handled by thread t: b = t + T i, i < P/R.  Butterfly
// b of span L covers the positions base + q r, r < R, q = L/R, with
// base = (b / q) L + (b mod q) and twiddle index j = b mod q.
#define ST_STAGE_CONSTS(S)                                              \
    typedef Geo<LOGM, LOGP> G;                                          \
    constexpr int lr = G::lr(S), R = 1 << lr, logL = G::logL(S);        \
    constexpr int logq = logL - lr, q = 1 << logq, PER = G::P / R;

// An integer zero that the compiler cannot see through, computed from x: an
// address offset by it waits for x, so table loads are not hoisted above the
// arithmetic that produces x (which would hold them all in registers at once).
__device__ __forceinline__ int after(float x)
{
    int z = 0;
    asm volatile("" : "+r"(z) : "f"(x));
    return z;
}
__device__ __forceinline__ int after(double x)
{
    int z = 0;
    asm volatile("" : "+r"(z) : "d"(x));
    return z;
}

// Two-level twiddles of one butterfly: W^{j k} = W^{4 j a} W^{j b} for
// k = 4a + b, from the table entries k = 1, 2, 3 and k = 4, 8, ..., R-4 of
// its column j (R/4 + 2 loads instead of R - 1, one extra rounding).  Fewer
// live table values leave the registers to the data.
template <int R, typename C>
struct Twiddles {
    C lo[4], hi[R / 4 > 1 ? R / 4 : 1];
    __device__ __forceinline__ void load(const C* __restrict__ w, int q)
    {
#pragma unroll
        for (int b = 1; b < 4 && b < R; b++) lo[b] = w[b * q];
#pragma unroll
        for (int a = 1; a < R / 4; a++) hi[a] = w[4 * a * q];
    }
    // W^{j k}, k = 1 .. R-1
    __device__ __forceinline__ C get(int k) const
    {
        const int a = k >> 2, b = k & 3;
        if (a == 0) return lo[b];
        if (b == 0) return hi[a];
        return cmul(hi[a], lo[b]);
    }
};

// forward (DIF) stage S: load, R-point DFT, twiddle.  Output k of butterfly
// i is left in register i R + brev(k).
template <typename C, int LOGM, int LOGP, int S, typename Ld>
__device__ __forceinline__ void dif(C* v, int t, const C* __restrict__ tw, const Ld& ld)
{
    ST_STAGE_CONSTS(S)
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int b = t + G::T * i;
        const int j = b & (q - 1), base = ((b >> logq) << logL) + j;
#pragma unroll
        for (int r = 0; r < R; r++) v[i * R + r] = ld(base + r * q);
        dft_dif<R, -1>(v + i * R);
        if (q > 1) {
            Twiddles<R, C> tw2;
            tw2.load(tw + tw_off(logL, lr) + j + after(v[i * R + R - 1].x), q);
#pragma unroll
            for (int k = 1; k < R; k++) v[i * R + brev(k, R)] = cmul(v[i * R + brev(k, R)], tw2.get(k));
        }
    }
}

// inverse (DIT) stage S: load, conjugate twiddle, R-point inverse DFT.  The
// loads go to register brev(r), so the outputs come out in natural order.
template <typename C, int LOGM, int LOGP, int S, typename Ld>
__device__ __forceinline__ void dit(C* v, int t, const C* __restrict__ tw, const Ld& ld)
{
    ST_STAGE_CONSTS(S)
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int b = t + G::T * i;
        const int j = b & (q - 1), base = ((b >> logq) << logL) + j;
#pragma unroll
        for (int r = 0; r < R; r++) v[i * R + brev(r, R)] = ld(base + r * q);
        if (q > 1) {
            Twiddles<R, C> tw2;
            tw2.load(tw + tw_off(logL, lr) + j + after(v[i * R + brev(R - 1, R)].x), q);
#pragma unroll
            for (int r = 1; r < R; r++) v[i * R + brev(r, R)] = cmulc(v[i * R + brev(r, R)], tw2.get(r));
        }
        dft_dit<R, 1>(v + i * R);
    }
}

// write the thread's points of stage S (same positions as its loads); BR:
// the registers hold the stage outputs in bit-reversed order (after dif)
template <bool BR, typename C, int LOGM, int LOGP, int S, typename St>
__device__ __forceinline__ void put(const C* v, int t, const St& st)
{
    ST_STAGE_CONSTS(S)
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int b = t + G::T * i;
        const int j = b & (q - 1), base = ((b >> logq) << logL) + j;
#pragma unroll
        for (int r = 0; r < R; r++) st(base + r * q, v[i * R + (BR ? brev(r, R) : r)]);
    }
}

// Storage position of filter entry p (p = ((t + T i) << logL) + k in the
// digit-reversed order of the last forward stage, k < R): the entries are
// kept in the order the threads of that stage use them, [i][k][t], so that
// the 32 threads of a warp read 32 consecutive entries per load.
template <int LOGM, int LOGP>
__host__ __device__ constexpr int filt_pos(int p)
{
    typedef Geo<LOGM, LOGP> G;
    constexpr int logR = G::lr(G::NST - 1), R = 1 << logR;
    const int b = p >> logR, k = p & (R - 1);
    return ((b / G::T) * R + k) * G::T + b % G::T;
}

// the last forward stage (q = 1, no twiddles), the filter product and the
// first inverse stage, on the same registers (outputs in natural order)
template <typename C, int LOGM, int LOGP, typename Ld>
__device__ __forceinline__ void middle(C* v, int t, const Ld& ld, const C* __restrict__ filt, bool conj_filt)
{
    constexpr int S = Geo<LOGM, LOGP>::NST - 1;
    ST_STAGE_CONSTS(S)
    static_assert(q == 1, "the last stage spans its radix");
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int base = (t + G::T * i) << logL;
#pragma unroll
        for (int r = 0; r < R; r++) v[i * R + r] = ld(base + r);
        dft_dif<R, -1>(v + i * R);
#pragma unroll
        for (int k = 0; k < R; k++) {
            const C f = filt[(i * R + k) * G::T + t];  // filt_pos(base + k)
            v[i * R + brev(k, R)] = cmul(v[i * R + brev(k, R)], conj_filt ? conjg(f) : f);
        }
        dft_dit<R, 1>(v + i * R);
    }
}

// Circular convolution of the M = 2^LOGM points given by in(p) with the
// filter, out(p, y_p) in natural order.  buf is this transform's padded
// shared-memory slot; every thread of the CTA must call (barriers inside).
template <typename C, int LOGM, int LOGP, typename In, typename Out>
__device__ __forceinline__ void convolve(C* buf, int t, const C* __restrict__ tw, const C* __restrict__ filt,
                                         bool conj_filt, const In& in, const Out& out)
{
    typedef Geo<LOGM, LOGP> G;
    C v[G::P];
    auto lds = [buf](int p) { return buf[pad(p)]; };
    auto sts = [buf](int p, C x) { buf[pad(p)] = x; };
    if constexpr (G::NST == 1) {
        middle<C, LOGM, LOGP>(v, t, in, filt, conj_filt);
        put<false, C, LOGM, LOGP, 0>(v, t, out);
    } else {
        dif<C, LOGM, LOGP, 0>(v, t, tw, in);
        put<true, C, LOGM, LOGP, 0>(v, t, sts);
        __syncthreads();
        if constexpr (G::NST >= 3) {
            dif<C, LOGM, LOGP, 1>(v, t, tw, lds);
            put<true, C, LOGM, LOGP, 1>(v, t, sts);
            __syncthreads();
        }
        if constexpr (G::NST >= 4) {
            dif<C, LOGM, LOGP, 2>(v, t, tw, lds);
            put<true, C, LOGM, LOGP, 2>(v, t, sts);
            __syncthreads();
        }
        static_assert(G::NST <= 4, "at most four stages");
        middle<C, LOGM, LOGP>(v, t, lds, filt, conj_filt);
        put<false, C, LOGM, LOGP, G::NST - 1>(v, t, sts);
        __syncthreads();
        if constexpr (G::NST >= 4) {
            dit<C, LOGM, LOGP, 2>(v, t, tw, lds);
            put<false, C, LOGM, LOGP, 2>(v, t, sts);
            __syncthreads();
        }
        if constexpr (G::NST >= 3) {
            dit<C, LOGM, LOGP, 1>(v, t, tw, lds);
            put<false, C, LOGM, LOGP, 1>(v, t, sts);
            __syncthreads();
        }
        dit<C, LOGM, LOGP, 0>(v, t, tw, lds);
        put<false, C, LOGM, LOGP, 0>(v, t, out);
    }
}

// Forward transform only (filter build): out(p, X) in the digit-reversed order.
template <typename C, int LOGM, int LOGP, typename In, typename Out>
__device__ __forceinline__ void forward(C* buf, int t, const C* __restrict__ tw, const In& in, const Out& out)
{
    typedef Geo<LOGM, LOGP> G;
    C v[G::P];
    auto lds = [buf](int p) { return buf[pad(p)]; };
    auto sts = [buf](int p, C x) { buf[pad(p)] = x; };
    dif<C, LOGM, LOGP, 0>(v, t, tw, in);
    if constexpr (G::NST >= 2) {
        put<true, C, LOGM, LOGP, 0>(v, t, sts);
        __syncthreads();
        dif<C, LOGM, LOGP, 1>(v, t, tw, lds);
    }
    if constexpr (G::NST >= 3) {
        put<true, C, LOGM, LOGP, 1>(v, t, sts);
        __syncthreads();
        dif<C, LOGM, LOGP, 2>(v, t, tw, lds);
    }
    if constexpr (G::NST >= 4) {
        put<true, C, LOGM, LOGP, 2>(v, t, sts);
        __syncthreads();
        dif<C, LOGM, LOGP, 3>(v, t, tw, lds);
    }
    put<true, C, LOGM, LOGP, G::NST - 1>(v, t, out);
}

// double -> float without the FP64 pipe (which is narrow on this GPU):
// integer bit operations on the IEEE encodings, branch free (dbl2flt_rn,
// st_internal.cuh); the r2c input measured faster with it than with the
// hardware conversion.
template <typename R> __device__ __forceinline__ R from_dbl(double d);
template <> __device__ __forceinline__ double from_dbl<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_dbl<float>(double d) { return dbl2flt_rn(d); }

// per-ring scale factor in the kernel's precision (tables, no FP64 arithmetic)
template <typename R> __device__ __forceinline__ R scale_of(const RingGeom& g, int k, int which);
template <> __device__ __forceinline__ double scale_of<double>(const RingGeom& g, int k, int which) { return g.sc64[4 * k + which]; }
template <> __device__ __forceinline__ float scale_of<float>(const RingGeom& g, int k, int which) { return g.sc32[4 * k + which]; }

// chirp c_u, u in [0, n): the table holds u = 0..n/2 (c_{n-u} = c_u)
template <typename C> __device__ __forceinline__ C chirp_at(const C* __restrict__ ch, int u, int n)
{
    return ch[u <= (n >> 1) ? u : n - u];
}

// ------------------------------------------------------------ precisions
template <typename R> struct KC;
// FP32: 32 points per thread, 256 threads, two CTAs per SM (8192 points: one
// transform of the largest length, or 8192/M shorter ones); FP64: 16 points,
// 512 threads (8192 points).  Two independent CTAs per SM hide the global
// memory phases of one behind the stages of the other, which measured faster
// than one 512-thread CTA holding two paired transforms.  The filter build
// (FP64 arithmetic with each precision's stage plan) runs FILT_NT threads
// over 8192 points.
template <> struct KC<float> { enum { LOGP = 5, NT = 256, MINB = 2, FILT_NT = 256 }; };
template <> struct KC<double> { enum { LOGP = 4, NT = 512, MINB = 1, FILT_NT = 512 }; };

template <typename R> __host__ __device__ constexpr int cta_points() { return KC<R>::NT << KC<R>::LOGP; }
template <typename R> __host__ __device__ constexpr int smem_bytes()
{
    return (cta_points<R>() + cta_points<R>() / 16) * (int)sizeof(typename Cx<R>::T);
}
constexpr int FILT_POINTS = 8192;
__host__ __device__ constexpr int filt_smem_bytes() { return (FILT_POINTS + FILT_POINTS / 16) * (int)sizeof(double2); }

// Slots x and x+1 of a CTA form a pair when they hold fields f and f+1 of the
// same ring pair and member, and the first Legendre field col0 + f is even:
// then their Fourier-side accesses (the c2r gather, the r2c fold stores) are
// shared, 4 columns at a time.  The even field makes column 2 (col0 + f) a
// multiple of 4, which the 16-byte (FP32) and 8-byte (split planes) vector
// accesses need (rows are multiples of 8 columns).
// (Both items must also lie inside the plan d: a pair is never formed from an
// item that the work-list check rejects.)
__device__ __forceinline__ bool paired(const FftIO& io, int4 cta, int x, int col0, const FftDesc& d)
{
    const int xe = x & ~1;
    if (xe + 1 >= cta.y) return false;
    const int4 a = io.items[cta.x + xe], b = io.items[cta.x + xe + 1];
    return a.x == b.x && a.z == b.z && ((col0 + a.y) & 1) == 0 && b.y == a.y + 1 && a.x >= 0 && a.x < d.nlat / 2 &&
           a.y >= 0 && b.y < d.nfld;
}

// 4 consecutive Fourier-buffer values from a 16-byte aligned address
__device__ __forceinline__ void ld4(const float* p, float* v)
{
    const float4 q = *(const float4*)p;
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v)
{
    const double2 q0 = *(const double2*)p, q1 = *(const double2*)(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

template <typename R> __device__ __forceinline__ const typename Cx<R>::T* chirp_of(const FftDesc& d);
template <> __device__ __forceinline__ const double2* chirp_of<double>(const FftDesc& d) { return d.chirp64; }
template <> __device__ __forceinline__ const float2* chirp_of<float>(const FftDesc& d) { return d.chirp32; }
template <typename R> __device__ __forceinline__ const typename Cx<R>::T* filt_of(const FftDesc& d);
template <> __device__ __forceinline__ const double2* filt_of<double>(const FftDesc& d) { return d.filt64; }
template <> __device__ __forceinline__ const float2* filt_of<float>(const FftDesc& d) { return d.filt32; }
template <typename R> __device__ __forceinline__ const typename Cx<R>::T* tw_of(const FftDesc& d);
template <> __device__ __forceinline__ const double2* tw_of<double>(const FftDesc& d) { return d.tw64; }
template <> __device__ __forceinline__ const float2* tw_of<float>(const FftDesc& d) { return d.tw32; }

// Work-list check of the ring-FFT kernels (always on): an item whose member,
// ring pair or field lies outside the plan is reported as ST_ERR_CHECK and
// replaced by a harmless one (ring pair 0, field 0) whose slot is not live,
// before any table is indexed with it.
__device__ __forceinline__ int4 fft_item(const FftIO& io, int4 cta, int x, bool& live)
{
    int4 it = io.items[cta.x + (live ? x : 0)];
    const bool mb_ok = io.desc ? (it.z >= 0 && it.z < io.nmemb) : it.z == 0;
    const FftDesc& d = io.desc ? io.desc[mb_ok ? it.z : 0] : io.d0;
    const bool ok = mb_ok && it.x >= 0 && it.x < d.nlat / 2 && it.y >= 0 && it.y < d.nfld;
    if (!ok) {
        if (live) atomicMax(d.status, (int)ST_ERR_CHECK);
        it = make_int4(0, 0, mb_ok ? it.z : 0, 0);
        live = false;
    }
    return it;
}

// ------------------------------------------------------------------ c2r
// The inputs are gathered into the transform's shared-memory slot first and
// the outputs leave it after the last stage, in loops of their own: the FFT
// stages then only read shared memory, and the global loads and stores do not
// compete with the stage registers.
template <typename R, int LOGM>
__device__ __forceinline__ void c2r_body(const FftIO& io, int4 cta, unsigned char* smem)
{
    typedef typename Cx<R>::T C;
    typedef Geo<LOGM, KC<R>::LOGP> G;
    const int x = threadIdx.x / G::T, t = threadIdx.x % G::T;
    bool live = x < cta.y;
    const int4 it = fft_item(io, cta, x, live);
    const int kN = it.x, f = it.y, mb = it.z, a = blockIdx.y;
    const FftDesc& d = io.desc ? io.desc[mb] : io.d0;
    const int slot = mb * io.narr + a;
    const int kS = d.nlat - 1 - kN, n = d.g.nlon[kN], K = d.g.mmax[kN] + 1;
    const long ncolp = d.ncolp;
    const int col = 2 * (io.col[slot] + f);
    const R* four = (const R*)d.four;
    const C* ch = chirp_of<R>(d) + d.f.choff[kN];
    C* buf = (C*)smem + x * (G::M + G::M / 16);
    // Y_m = H_N(m) + i H_S(m) for m and -m, times c_m, at positions m and M - m
    auto gather = [&](C* bf, int m, C A, C B) {
        if (m == 0) A.y = B.y = 0;
        if (io.dlam[slot]) {  // i m F_m
            const R fm = (R)m;
            A = cx<C>(-fm * A.y, fm * A.x);
            B = cx<C>(-fm * B.y, fm * B.x);
        }
        const C cm = ch[m];
        bf[pad(m)] = cmul(cx<C>(A.x - B.y, A.y + B.x), cm);
        if (m) bf[pad(G::M - m)] = cmul(cx<C>(A.x + B.y, B.x - A.y), cm);  // conj H_N + i conj H_S
    };
    if (paired(io, cta, x, io.col[slot], d)) {
        // both slots of the pair gather fields f, f+1 with one 4-column load
        const int xe = x & ~1, tt = (x - xe) * G::T + t;
        C* be = (C*)smem + xe * (G::M + G::M / 16);
        C* bo = be + (G::M + G::M / 16);
        const int ce = 2 * (io.col[slot] + io.items[cta.x + xe].y);
        const R* xn = four + d.g.foff[kN] * ncolp + ce;
        const R* xs = four + d.g.foff[kS] * ncolp + ce;
#pragma unroll 2
        for (int m = tt; m < K; m += 2 * G::T) {
            R vn[4], vs[4];
            ld4(xn + m * ncolp, vn);
            ld4(xs + m * ncolp, vs);
            gather(be, m, cx<C>(vn[0], vn[1]), cx<C>(vs[0], vs[1]));
            gather(bo, m, cx<C>(vn[2], vn[3]), cx<C>(vs[2], vs[3]));
        }
    } else if (live) {
        const R* xn = four + d.g.foff[kN] * ncolp + col;
        const R* xs = four + d.g.foff[kS] * ncolp + col;
#pragma unroll 4
        for (int m = t; m < K; m += G::T) gather(buf, m, *(const C*)(xn + m * ncolp), *(const C*)(xs + m * ncolp));
    }
    __syncthreads();
    auto in0 = [buf, K](int p) { return (p < K || p > G::M - K) ? buf[pad(p)] : cx<C>(0, 0); };
    auto sts = [buf](int p, C v) { buf[pad(p)] = v; };
    convolve<C, LOGM, KC<R>::LOGP>(buf, t, tw_of<R>(d), filt_of<R>(d) + d.f.floff[kN], true, in0, sts);
    __syncthreads();
    if (live) {
        // 0: none, 1: 1/cos(phi), 2: w/nlon
        const int sm = io.scale[slot] == 1 ? SC_INVCOS : (io.scale[slot] == 2 ? SC_WN : SC_ONE);
        const R scr = scale_of<R>(d.g, kN, sm);
        double* gb = io.out[slot] + (long)f * d.npts;
        double* gn = gb + d.g.roff[kN];
        double* gs = gb + d.g.roff[kS];
        // f_N + i f_S = c_p y_p; two adjacent points per thread (nlon is a
        // multiple of 4 and the rings start 32-byte aligned): 16-byte stores.
        // float -> double by the hardware conversion here: measured 2 % faster
        // than the integer one on the 8192-point transforms (the r2c input
        // keeps the integer double -> float, which measured faster there)
#pragma unroll 4
        for (int p = 2 * t; p < n; p += 2 * G::T) {
            const C g0 = cmul(buf[pad(p)], chirp_at(ch, p, n));
            const C g1 = cmul(buf[pad(p + 1)], chirp_at(ch, p + 1, n));
            // streaming stores: the grid is not read again by this step, so it
            // should not push the scattered Fourier rows out of L2
            __stcs((double2*)(gn + p), make_double2((double)(g0.x * scr), (double)(g1.x * scr)));
            __stcs((double2*)(gs + p), make_double2((double)(g0.y * scr), (double)(g1.y * scr)));
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(KC<R>::NT, KC<R>::MINB) k_c2r(const __grid_constant__ FftIO io)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 cta = io.ctas[blockIdx.x];
    switch (cta.z) {
        case 5: c2r_body<R, 5>(io, cta, smem_raw); break;
        case 6: c2r_body<R, 6>(io, cta, smem_raw); break;
        case 7: c2r_body<R, 7>(io, cta, smem_raw); break;
        case 8: c2r_body<R, 8>(io, cta, smem_raw); break;
        case 9: c2r_body<R, 9>(io, cta, smem_raw); break;
        case 10: c2r_body<R, 10>(io, cta, smem_raw); break;
        case 11: c2r_body<R, 11>(io, cta, smem_raw); break;
        case 12: c2r_body<R, 12>(io, cta, smem_raw); break;
        case 13: c2r_body<R, 13>(io, cta, smem_raw); break;
        default: break;
    }
}

// store (re, im) at columns i, i+1 of a direct-operand row: one vector store
// per plane (split planes as in put_split)
template <typename R>
__device__ __forceinline__ void put_pair(R* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long i, R re, R im, int ns)
{
    typedef typename Cx<R>::T C;
    if (ns == 0) {
        *(C*)(p0 + i) = cx<C>(re, im);
        return;
    }
    const float xr = (float)re, xi = (float)im;
    __nv_bfloat162 a, b, c;
    a.x = __float2bfloat16_rn(xr);
    a.y = __float2bfloat16_rn(xi);
    const float rr = xr - __bfloat162float(a.x), ri = xi - __bfloat162float(a.y);
    b.x = __float2bfloat16_rn(rr);
    b.y = __float2bfloat16_rn(ri);
    *(__nv_bfloat162*)((__nv_bfloat16*)p0 + i) = a;
    *(__nv_bfloat162*)(p1 + i) = b;
    if (ns == 3) {
        c.x = __float2bfloat16_rn(rr - __bfloat162float(b.x));
        c.y = __float2bfloat16_rn(ri - __bfloat162float(b.y));
        *(__nv_bfloat162*)(p2 + i) = c;
    }
}

// store 4 consecutive columns of a direct-operand row (two fields' re, im):
// one 16-byte store (FP32), two (FP64), or one 8-byte store per split plane
__device__ __forceinline__ void put_quad(double* p0, __nv_bfloat16*, __nv_bfloat16*, long i, const double* v, int)
{
    *(double2*)(p0 + i) = make_double2(v[0], v[1]);
    *(double2*)(p0 + i + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void put_quad(float* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long i, const float* v, int ns)
{
    if (ns == 0) {
        *(float4*)(p0 + i) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
    __nv_bfloat162 a[2], b[2], c[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const float x0 = v[2 * h], x1 = v[2 * h + 1];
        a[h].x = __float2bfloat16_rn(x0);
        a[h].y = __float2bfloat16_rn(x1);
        const float r0 = x0 - __bfloat162float(a[h].x), r1 = x1 - __bfloat162float(a[h].y);
        b[h].x = __float2bfloat16_rn(r0);
        b[h].y = __float2bfloat16_rn(r1);
        c[h].x = __float2bfloat16_rn(r0 - __bfloat162float(b[h].x));
        c[h].y = __float2bfloat16_rn(r1 - __bfloat162float(b[h].y));
    }
    *(uint2*)((__nv_bfloat16*)p0 + i) = make_uint2(*(unsigned*)&a[0], *(unsigned*)&a[1]);
    *(uint2*)(p1 + i) = make_uint2(*(unsigned*)&b[0], *(unsigned*)&b[1]);
    if (ns == 3) *(uint2*)(p2 + i) = make_uint2(*(unsigned*)&c[0], *(unsigned*)&c[1]);
}

// ------------------------------------------------------------------ r2c
template <typename R, int LOGM>
__device__ __forceinline__ void r2c_body(const FftIO& io, int4 cta, unsigned char* smem)
{
    typedef typename Cx<R>::T C;
    typedef Geo<LOGM, KC<R>::LOGP> G;
    const int x = threadIdx.x / G::T, t = threadIdx.x % G::T;
    bool live = x < cta.y;
    const int4 it = fft_item(io, cta, x, live);
    const int kN = it.x, f = it.y, mb = it.z, a = blockIdx.y;
    const FftDesc& d = io.desc ? io.desc[mb] : io.d0;
    const int slot = mb * io.narr + a;
    const int kS = d.nlat - 1 - kN, n = d.g.nlon[kN], K = d.g.mmax[kN] + 1;
    const C* ch = chirp_of<R>(d) + d.f.choff[kN];
    C* buf = (C*)smem + x * (G::M + G::M / 16);
    if (live) {
        // z_j conj(c_j), z = f_N + i f_S
        const double* gb = io.in[slot] + (long)f * d.npts;
        const double* fn = gb + d.g.roff[kN];
        const double* fs = gb + d.g.roff[kS];
        // two adjacent points per thread: 16-byte loads (see the c2r output)
#pragma unroll 4
        for (int p = 2 * t; p < n; p += 2 * G::T) {
            const double2 u = *(const double2*)(fn + p), w = *(const double2*)(fs + p);
            if (d.checks && !(isfinite(u.x) && isfinite(u.y) && isfinite(w.x) && isfinite(w.y)))
                atomicMax(d.status, (int)ST_ERR_CHECK);
            buf[pad(p)] = cmulc(cx<C>(from_dbl<R>(u.x), from_dbl<R>(w.x)), chirp_at(ch, p, n));
            buf[pad(p + 1)] = cmulc(cx<C>(from_dbl<R>(u.y), from_dbl<R>(w.y)), chirp_at(ch, p + 1, n));
        }
    }
    __syncthreads();
    auto in0 = [buf, n](int p) { return p < n ? buf[pad(p)] : cx<C>(0, 0); };
    auto sts = [buf](int p, C v) { buf[pad(p)] = v; };
    convolve<C, LOGM, KC<R>::LOGP>(buf, t, tw_of<R>(d), filt_of<R>(d) + d.f.floff[kN], false, in0, sts);
    __syncthreads();
    // separate the two rings, fold, write the m-major operand rows:
    // 2 F_N = Zp + conj Zn, 2 F_S = -i (Zp - conj Zn), G_s/a = s (F_N +- F_S)
    const int smode = io.scale[slot] == 1 ? SC_WNCOS : (io.scale[slot] == 2 ? SC_ONE : SC_WN);
    const R s = (R)0.5 * scale_of<R>(d.g, kN, smode);  // 0: w/nlon, 1: w/(nlon cos), 2: none; x 1/2
    // split paths write the FP32 operand (split into the planes by
    // k_split_gop); the FP32 and FP64 paths write the operand itself
    R* gop = d.g32 ? (R*)d.g32 : (R*)d.four;
    const int ns = d.g32 ? 0 : d.split;
    auto fold = [&](const C* bf, int m, C cm, R* gs, R* ga) {
        const C Zp = cmulc(bf[pad(m)], cm);
        const C Zn = cmulc(bf[pad(m ? G::M - m : 0)], cm);
        const C fN = cx<C>(Zp.x + Zn.x, Zp.y - Zn.y);
        const C dd = cx<C>(Zp.x - Zn.x, Zp.y + Zn.y);
        const C fS = cx<C>(dd.y, -dd.x);
        gs[0] = s * (fN.x + fS.x);
        gs[1] = s * (fN.y + fS.y);
        ga[0] = s * (fN.x - fS.x);
        ga[1] = s * (fN.y - fS.y);
    };
    if (paired(io, cta, x, io.col[slot], d)) {
        // both slots of the pair: fields f, f+1 in one 4-column store per plane
        const int xe = x & ~1, tt = (x - xe) * G::T + t;
        const C* be = (C*)smem + xe * (G::M + G::M / 16);
        const C* bo = be + (G::M + G::M / 16);
        const int ce = 2 * (io.col[slot] + io.items[cta.x + xe].y);
        for (int m = tt; m < K; m += 2 * G::T) {
            const C cm = ch[m];
            R vs[4], va[4];
            fold(be, m, cm, vs, va);
            fold(bo, m, cm, vs + 2, va + 2);
            const int l = kN - d.k0[m];
            put_quad(gop, d.lo, d.lo2, (d.goff[2 * m] + l) * (long)d.ncolp + ce, vs, ns);
            put_quad(gop, d.lo, d.lo2, (d.goff[2 * m + 1] + l) * (long)d.ncolp + ce, va, ns);
        }
        return;
    }
    if (!live) return;
    const int col = 2 * (io.col[slot] + f);
    for (int m = t; m < K; m += G::T) {
        R vs[2], va[2];
        fold(buf, m, ch[m], vs, va);
        const int l = kN - d.k0[m];
        put_pair<R>(gop, d.lo, d.lo2, (d.goff[2 * m] + l) * (long)d.ncolp + col, vs[0], vs[1], ns);
        put_pair<R>(gop, d.lo, d.lo2, (d.goff[2 * m + 1] + l) * (long)d.ncolp + col, va[0], va[1], ns);
    }
}

template <typename R>
__global__ void __launch_bounds__(KC<R>::NT, KC<R>::MINB) k_r2c(const __grid_constant__ FftIO io)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 cta = io.ctas[blockIdx.x];
    switch (cta.z) {
        case 5: r2c_body<R, 5>(io, cta, smem_raw); break;
        case 6: r2c_body<R, 6>(io, cta, smem_raw); break;
        case 7: r2c_body<R, 7>(io, cta, smem_raw); break;
        case 8: r2c_body<R, 8>(io, cta, smem_raw); break;
        case 9: r2c_body<R, 9>(io, cta, smem_raw); break;
        case 10: r2c_body<R, 10>(io, cta, smem_raw); break;
        case 11: r2c_body<R, 11>(io, cta, smem_raw); break;
        case 12: r2c_body<R, 12>(io, cta, smem_raw); break;
        case 13: r2c_body<R, 13>(io, cta, smem_raw); break;
        default: break;
    }
}

// --------------------------------------------------------------- filters
// B = FFT_M(b)/M of the direct kernel b_t = c_t, t in [-(n+K-2), K-1] (mod M),
// in the digit-reversed order that the forward stages of each precision
// leave, each entry stored at filt_pos (the order depends on the points per
// thread, so the FP32 table is built with the FP32 stage plan).  Computed in
// FP64, one CTA per ring pair.
struct FiltIn {
    const double2* ch;
    int n, K, M;
    bool live;
    __device__ __forceinline__ double2 operator()(int s) const
    {
        if (!live) return make_double2(0, 0);
        int u;
        if (s < K) u = s;
        else if (s >= M - (n + K - 2)) u = M - s;  // |t| for t = s - M
        else return make_double2(0, 0);
        if (u >= n) u -= n;
        return chirp_at(ch, u, n);
    }
};
template <int LOGM, int LOGP>
struct FiltOut {
    double2* f64;
    float2* f32;
    double inv;
    bool live;
    __device__ __forceinline__ void operator()(int p, double2 v) const
    {
        if (!live) return;
        v.x *= inv;
        v.y *= inv;
        const int s = filt_pos<LOGM, LOGP>(p);
        if (f64) f64[s] = v;
        if (f32) f32[s] = make_float2((float)v.x, (float)v.y);
    }
};

template <int LOGM, int LOGP>
__device__ __forceinline__ void filt_body(const FftDesc& d, int k, double2* f64, float2* f32, unsigned char* smem)
{
    typedef Geo<LOGM, LOGP> G;
    // slot x = 0 builds the filter; the other slots run on zeros in their own
    // shared-memory slots so that every thread meets the barriers
    const int x = threadIdx.x / G::T, t = threadIdx.x % G::T;
    const bool live = x == 0;
    const int n = d.g.nlon[k], K = d.g.mmax[k] + 1;
    const FiltIn in{d.chirp64 + d.f.choff[k], n, K, G::M, live};
    const FiltOut<LOGM, LOGP> out{f64 ? f64 + d.f.floff[k] : nullptr, f32 ? f32 + d.f.floff[k] : nullptr, 1.0 / G::M, live};
    forward<double2, LOGM, LOGP>((double2*)smem + x * (G::M + G::M / 16), t, d.tw64, in, out);
}

// One kernel per table, each with the thread count of its stage plan over
// 8192 points of shared memory: FP64 512 threads, FP32 256.
template <typename R>
__global__ void __launch_bounds__(KC<R>::FILT_NT) k_fft_filters(FftDesc d, double2* f64, float2* f32)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LP = KC<R>::LOGP;
    const int k = blockIdx.x;
    switch (d.f.logM[k]) {
        case 5: filt_body<5, LP>(d, k, f64, f32, smem_raw); break;
        case 6: filt_body<6, LP>(d, k, f64, f32, smem_raw); break;
        case 7: filt_body<7, LP>(d, k, f64, f32, smem_raw); break;
        case 8: filt_body<8, LP>(d, k, f64, f32, smem_raw); break;
        case 9: filt_body<9, LP>(d, k, f64, f32, smem_raw); break;
        case 10: filt_body<10, LP>(d, k, f64, f32, smem_raw); break;
        case 11: filt_body<11, LP>(d, k, f64, f32, smem_raw); break;
        case 12: filt_body<12, LP>(d, k, f64, f32, smem_raw); break;
        case 13: filt_body<13, LP>(d, k, f64, f32, smem_raw); break;
        default: break;
    }
}

}  // namespace fft

}  // namespace st
