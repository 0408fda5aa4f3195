// Ring FFTs of the spectral transform (latitude rings of uneven length).
//
// A ring of nlon = 2h real points is transformed as h complex points
// z_l = f_{2l} + i f_{2l+1}.  The length-h DFT is a Bluestein chirp-z
// convolution over a power-of-two length M >= 2h - 1:
//   sum_q Z_q e^{+2 pi i q l/h} = w_l sum_q (Z_q w_q) conj(w_{l-q}),
// where w_t = e^{i pi t^2/h}.  The filter FFT_M(conj w)/M is precomputed per
// ring in bit-reversed order.  The forward FFT is a radix-2
// decimation-in-frequency pass (natural order in, bit-reversed out).  The
// filter product is taken in that order.  The inverse is a
// decimation-in-time pass (bit-reversed in, natural out).  So no permutation
// is ever performed.  The analysis direction uses DFT(y) = conj(IDFT(conj y)).
//
// Fusions (the transposition of the paper's all-to-all, Sec. 3.1.3, done as a
// change of layout):
//   c2r  reads the ring-major Fourier buffer four[ring][m][col] that the
//        Legendre epilogue wrote.  It applies i*m for d/dlambda and a per-ring
//        scale (1/cos(phi), or w/nlon for the adjoint), then writes the grid.
//   r2c  transforms a north ring and its southern mirror in one CTA.  It then
//        folds them, G_s = s (F_N + F_S) and G_a = s (F_N - F_S), with the
//        per-ring scale s (w/nlon, w/(nlon cos(phi)) or 1).  It writes the
//        m-major direct Legendre operand, optionally split into bf16 hi/lo.
#include "st_internal.cuh"

namespace st {

template <typename R> struct Cplx;
template <> struct Cplx<double> { typedef double2 T; };
template <> struct Cplx<float> { typedef float2 T; };

template <typename C> __device__ __forceinline__ C mk(double x, double y) { C r; r.x = x; r.y = y; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C conjg(C a) { a.y = -a.y; return a; }

__device__ __forceinline__ void sincos_pi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincos_pi(float x, float* s, float* c) { sincospif(x, s, c); }

// cos(2 pi k/16): the real parts of the sixteenth roots of unity; the
// imaginary part is cos(2 pi (k - 4)/16).
__host__ __device__ constexpr double w16c(int k)
{
    switch (k & 15) {
        case 0: return 1.00000000000000000000;
        case 1: return 0.92387953251128673848;
        case 2: return 0.70710678118654757274;
        case 3: return 0.38268343236508983729;
        case 4: return 0.00000000000000006123;
        case 5: return -0.38268343236508972627;
        case 6: return -0.70710678118654746172;
        case 7: return -0.92387953251128673848;
        case 8: return -1.00000000000000000000;
        case 9: return -0.92387953251128684951;
        case 10: return -0.70710678118654768376;
        case 11: return -0.38268343236509033689;
        case 12: return -0.00000000000000018370;
        case 13: return 0.38268343236509000382;
        case 14: return 0.70710678118654735069;
        case 15: return 0.92387953251128651644;
    }
    return 0.0;
}
__host__ __device__ constexpr double w16s(int k) { return w16c(k - 4); }

// In-register R-point DFT (R = 1..16, power of two), natural order in and out,
// kernel e^{SIGN 2 pi i r r'/R}: split into even/odd halves recursively.
template <int R, int SIGN, typename C>
struct RegDFT {
    __device__ __forceinline__ static void run(C* v)
    {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        RegDFT<R / 2, SIGN, C>::run(e);
        RegDFT<R / 2, SIGN, C>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            const C w = mk<C>(w16c(k * (16 / R)), SIGN * w16s(k * (16 / R)));
            const C t = cmul(o[k], w);
            v[k] = cadd(e[k], t);
            v[k + R / 2] = csub(e[k], t);
        }
    }
};
template <int SIGN, typename C>
struct RegDFT<1, SIGN, C> {
    __device__ __forceinline__ static void run(C*) {}
};

// Twiddles of one stage (span L = 2^logL, radix R = 2^lr) are stored as
// [r][j] = W_L^{j r}, j < L/R, so a warp reads them contiguously.  The block
// of (logL, lr) starts at 4 (2^logL - 2) + (lr - 1) 2^logL; the whole table
// holds 4 (2 Mmax - 2) entries.
__host__ __device__ inline int tw_off(int logL, int lr) { return 4 * ((1 << logL) - 2) + (lr - 1) * (1 << logL); }

// Shared-memory index with one pad element every 32, so that the strided
// butterfly accesses of the short spans spread over the banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }
__host__ __device__ inline int padded_len(int M) { return M + (M >> 5); }

// One in-place radix-R decimation-in-frequency stage over sub-transforms of
// length L = 2^logL: for block b and j < L/R, the R points b L + j + r L/R go
// through an R-point DFT (kernel e^{-2 pi i/R}); output r' is multiplied by
// W_L^{j r'} and written back to b L + j + r' L/R.
template <int LR, typename C>
__device__ __forceinline__ void dif_stage(C* buf, int stride, int nb, int logM, int logL,
                                          const C* __restrict__ tw, int)
{
    constexpr int R = 1 << LR;
    const int logq = logL - LR;
    const int lbf = logM - LR;  // log2 of butterflies per field
    const int total = nb << lbf;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = idx >> lbf, t = idx & ((1 << lbf) - 1);
        const int j = t & ((1 << logq) - 1);
        const int base = ((t >> logq) << logL) + j;
        C* x = buf + (long)b * stride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = x[pad(base + (r << logq))];
        RegDFT<R, -1, C>::run(v);
        const C* twr = tw + tw_off(logL, LR) + j;
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (r == 0) {
                x[pad(base)] = v[0];
            } else {
                x[pad(base + (r << logq))] = cmul(v[r], twr[r << logq]);
            }
        }
    }
    __syncthreads();
}

// The exact inverse of dif_stage up to the factor R (twiddle conjugated, then
// an R-point DFT with kernel e^{+2 pi i/R}).
template <int LR, typename C>
__device__ __forceinline__ void dit_stage(C* buf, int stride, int nb, int logM, int logL,
                                          const C* __restrict__ tw, int)
{
    constexpr int R = 1 << LR;
    const int logq = logL - LR;
    const int lbf = logM - LR;
    const int total = nb << lbf;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = idx >> lbf, t = idx & ((1 << lbf) - 1);
        const int j = t & ((1 << logq) - 1);
        const int base = ((t >> logq) << logL) + j;
        C* x = buf + (long)b * stride;
        const C* twr = tw + tw_off(logL, LR) + j;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const C u = x[pad(base + (r << logq))];
            v[r] = r ? cmulc(u, twr[r << logq]) : u;
        }
        RegDFT<R, 1, C>::run(v);
#pragma unroll
        for (int r = 0; r < R; r++) x[pad(base + (r << logq))] = v[r];
    }
    __syncthreads();
}

// ---------------------------------------------------------- fused Bluestein
// Stage plan of a length-M transform (32 <= M): a first DIF stage of radix
// 2^r0 (r0 = logM mod 4, or 4) at the full span M, then radix-16 DIF stages
// down to span 16.  The inverse runs the same stages backwards.  Three
// fusions keep data in registers:
//   first  the first DIF stage produces its inputs itself (gather, chirp,
//          zero padding) instead of reading them from shared memory;
//   middle the span-16 DIF stage, the filter product and the span-16 DIT
//          stage (no twiddles at span 16) run on the same 16 points;
//   last   the last DIT stage (span M) hands its outputs to the caller
//          (chirp and store) instead of writing shared memory.
__host__ __device__ inline int first_radix_bits(int logM) { return (logM & 3) ? (logM & 3) : 4; }

template <int LR, typename C, typename In>
__device__ __forceinline__ void dif_first(C* buf, int stride, int nb, int logM, const C* __restrict__ tw, const In& in)
{
    constexpr int R = 1 << LR;
    const int logq = logM - LR;
    const int total = nb << logq;
    const C* twb = tw + tw_off(logM, LR);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = idx >> logq, j = idx & ((1 << logq) - 1);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = in(b, j + (r << logq));
        RegDFT<R, -1, C>::run(v);
        C* x = buf + (long)b * stride;
        x[pad(j)] = v[0];
#pragma unroll
        for (int r = 1; r < R; r++) x[pad(j + (r << logq))] = cmul(v[r], twb[(r << logq) + j]);
    }
    __syncthreads();
}

template <int LR, typename C, typename Out>
__device__ __forceinline__ void dit_last(C* buf, int stride, int nb, int logM, const C* __restrict__ tw, const Out& out)
{
    constexpr int R = 1 << LR;
    const int logq = logM - LR;
    const int total = nb << logq;
    const C* twb = tw + tw_off(logM, LR);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = idx >> logq, j = idx & ((1 << logq) - 1);
        const C* x = buf + (long)b * stride;
        C v[R];
        v[0] = x[pad(j)];
#pragma unroll
        for (int r = 1; r < R; r++) v[r] = cmulc(x[pad(j + (r << logq))], twb[(r << logq) + j]);
        RegDFT<R, 1, C>::run(v);
#pragma unroll
        for (int r = 0; r < R; r++) out(b, j + (r << logq), v[r]);
    }
}

template <typename C>
__device__ __forceinline__ void middle(C* buf, int stride, int nb, int logM, const C* __restrict__ filt)
{
    const int lg = logM - 4;
    const int total = nb << lg;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int b = idx >> lg, base = (idx & ((1 << lg) - 1)) << 4;
        C* x = buf + (long)b * stride;
        C v[16];
#pragma unroll
        for (int r = 0; r < 16; r++) v[r] = x[pad(base + r)];
        RegDFT<16, -1, C>::run(v);
#pragma unroll
        for (int r = 0; r < 16; r++) v[r] = cmul(v[r], filt[base + r]);
        RegDFT<16, 1, C>::run(v);
#pragma unroll
        for (int r = 0; r < 16; r++) x[pad(base + r)] = v[r];
    }
    __syncthreads();
}

// Bluestein convolution with the ring's filter: in(b, p) supplies a_p (p < M,
// already chirped and zero-padded), out(b, p, conv_p) receives the circular
// convolution in natural order.  Not followed by a barrier.
template <typename C, typename In, typename Out>
__device__ void bluestein(C* buf, int stride, int nb, int logM, const C* __restrict__ filt,
                          const C* __restrict__ tw, const In& in, const Out& out)
{
    const int r0 = first_radix_bits(logM);
    switch (r0) {
        case 1: dif_first<1>(buf, stride, nb, logM, tw, in); break;
        case 2: dif_first<2>(buf, stride, nb, logM, tw, in); break;
        case 3: dif_first<3>(buf, stride, nb, logM, tw, in); break;
        default: dif_first<4>(buf, stride, nb, logM, tw, in); break;
    }
    for (int logL = logM - r0; logL > 4; logL -= 4) dif_stage<4>(buf, stride, nb, logM, logL, tw, 0);
    middle(buf, stride, nb, logM, filt);
    for (int logL = 8; logL <= logM - r0; logL += 4) dit_stage<4>(buf, stride, nb, logM, logL, tw, 0);
    switch (r0) {
        case 1: dit_last<1>(buf, stride, nb, logM, tw, out); break;
        case 2: dit_last<2>(buf, stride, nb, logM, tw, out); break;
        case 3: dit_last<3>(buf, stride, nb, logM, tw, out); break;
        default: dit_last<4>(buf, stride, nb, logM, tw, out); break;
    }
}

// --------------------------------------------------------------- filters
// filt = FFT_M(b)/M in the digit-reversed order that the DIF stages of
// bluestein() leave, b_t = conj(w_t) for |t| < h (mod M).  Built by the same
// stage sequence as the data transforms, so the two orders agree.
struct FiltIn {
    const double2* ch;
    int h, M;
    __device__ double2 operator()(int, int i) const
    {
        if (i < h) return conjg(ch[i]);
        if (i > M - h) return conjg(ch[M - i]);
        return mk<double2>(0, 0);
    }
};

__global__ void k_fft_filters(RingFFT f, const double2* __restrict__ chirp, double2* filt64, float2* filt32,
                              const double2* __restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = (double2*)smem_raw;
    const int k = blockIdx.x;
    const int h = f.h[k], logM = f.logM[k], M = 1 << logM;
    const FiltIn in{chirp + f.choff[k], h, M};
    const int r0 = first_radix_bits(logM);
    switch (r0) {
        case 1: dif_first<1>(buf, 0, 1, logM, tw, in); break;
        case 2: dif_first<2>(buf, 0, 1, logM, tw, in); break;
        case 3: dif_first<3>(buf, 0, 1, logM, tw, in); break;
        default: dif_first<4>(buf, 0, 1, logM, tw, in); break;
    }
    for (int logL = logM - r0; logL >= 4; logL -= 4) dif_stage<4>(buf, 0, 1, logM, logL, tw, 0);
    const double inv = 1.0 / M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double2 v = buf[pad(i)];
        v.x *= inv;
        v.y *= inv;
        filt64[f.floff[k] + i] = v;
        filt32[f.floff[k] + i] = make_float2((float)v.x, (float)v.y);
    }
}

static int ilog2(int x) { int l = 0; while ((1 << l) < x) l++; return l; }

int launch_fft_filters(Tables* t)
{
    size_t smem = (size_t)padded_len(t->Mmax) * sizeof(double2);
    if (smem > 227 * 1024) {
        set_error("ring FFT length %d exceeds the on-chip limit (T too large)", t->Mmax);
        return ST_ERR_UNSUPPORTED;
    }
    ST_CUDA_TRY(cudaFuncSetAttribute(k_fft_filters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fft_filters<<<t->N, 256, smem>>>(t->fft(), t->chirp64, t->filt64, t->filt32, t->tw64);
    ST_CUDA_TRY(cudaGetLastError());
    ST_CUDA_TRY(cudaDeviceSynchronize());
    return ST_OK;
}

// ------------------------------------------------------------- batching
// shared memory per CTA: the largest single-field need for T <= 2043 (M =
// 8192) fits, and FP32 leaves room for two 512-thread CTAs per SM
static size_t fft_cap_bytes(st_prec prec, bool pair) { return prec == ST_PREC_FP64 ? 180 * 1024 : (pair ? 110 : 100) * 1024; }
static size_t cplx_bytes(st_prec prec) { return prec == ST_PREC_FP64 ? 16 : 8; }

// fields per CTA for ring k (pair: r2c on a north/south pair, which also keeps h
// Fourier coefficients of the north ring on chip)
static int fft_batch_ex(const Tables* t, int k, st_prec prec, bool pair)
{
    size_t need = (size_t)padded_len(1 << t->logM[k]) + (pair ? t->hh[k] : 0);
    size_t B = fft_cap_bytes(prec, pair) / (need * cplx_bytes(prec));
    if (B < 1) B = 1;
    if (B > 256) B = 256;
    return (int)B;
}

int fft_batch(const Tables* t, int k, st_prec prec)
{
    if (k < 0) return fft_batch_ex(t, -1 - k, prec, true);
    return fft_batch_ex(t, k, prec, false);
}

static size_t fft_smem(const Tables* t, st_prec prec, bool pair)
{
    size_t mx = 0;
    for (int k = 0; k < t->N; k++) {
        size_t need = (size_t)padded_len(1 << t->logM[k]) + (pair ? t->hh[k] : 0);
        mx = std::max(mx, (size_t)fft_batch_ex(t, k, prec, pair) * need * cplx_bytes(prec));
    }
    return mx;
}

// FP32 kernels run 512 threads (2 CTAs per SM, 64 registers), FP64 kernels 256
template <typename R> struct FftThreads { enum { N = 512, MINB = 2 }; };
template <> struct FftThreads<double> { enum { N = 256, MINB = 1 }; };

// ------------------------------------------------------------------ c2r
template <typename R, typename C>
__device__ __forceinline__ C load_X(const R* __restrict__ F, int ncolp, int col, int m, int mmax, bool dl)
{
    if (m > mmax) return mk<C>(0, 0);
    R re = F[(long)m * ncolp + col];
    R im = m ? F[(long)m * ncolp + col + 1] : (R)0;
    if (dl) return mk<C>(-(R)m * im, (R)m * re);
    return mk<C>(re, im);
}

// a_q = Z_q w_q with Z_q = (X_q + conj X_{h-q}) + i (X_q - conj X_{h-q}) e^{i pi q/h}
// (the half-length packing of the Hermitian spectrum X of a real ring)
template <typename R>
struct C2RIn {
    typedef typename Cplx<R>::T C;
    const R* F;
    const C* ch;
    int ncolp, col0, mmax, h;
    bool dl;
    __device__ C operator()(int b, int q) const
    {
        if (q >= h) return mk<C>(0, 0);
        const int col = col0 + 2 * b;
        const C Xq = load_X<R, C>(F, ncolp, col, q, mmax, dl);
        const C Xh = load_X<R, C>(F, ncolp, col, h - q, mmax, dl);
        const C e = cadd(Xq, conjg(Xh)), d = csub(Xq, conjg(Xh));
        R sn, cs;
        sincos_pi((R)q / (R)h, &sn, &cs);
        const C t = cmul(d, mk<C>(cs, sn));
        return cmul(mk<C>(e.x - t.y, e.y + t.x), ch[q]);
    }
};

// f_{2l} + i f_{2l+1} = w_l conv_l, scaled, straight to the grid
template <typename R>
struct C2ROut {
    typedef typename Cplx<R>::T C;
    double* dst;
    const C* ch;
    long npts;
    int h;
    R sc;
    __device__ void operator()(int b, int l, C v) const
    {
        if (l >= h) return;
        const C z = cmul(v, ch[l]);
        *(double2*)(dst + (long)b * npts + 2 * l) = make_double2((double)(z.x * sc), (double)(z.y * sc));
    }
};

template <typename R>
__global__ void __launch_bounds__(FftThreads<R>::N, FftThreads<R>::MINB)
    k_c2r(const R* __restrict__ four, int ncolp, RingGeom g, RingFFT f, const typename Cplx<R>::T* __restrict__ chirp,
          const typename Cplx<R>::T* __restrict__ filt, const typename Cplx<R>::T* __restrict__ tw,
          const FFTWork* __restrict__ work, SynthOut out, long npts)
{
    typedef typename Cplx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = (C*)smem_raw;
    const FFTWork wk = work[blockIdx.x];
    const int k = wk.ring, a = wk.arr, nb = wk.nb;
    const int h = f.h[k], logM = f.logM[k], stride = padded_len(1 << logM);
    const C* ch = chirp + f.choff[k];
    double sc = 1.0;
    if (out.scale[a] == 1) sc = 1.0 / g.coslat[k];
    else if (out.scale[a] == 2) sc = g.w[k] / (double)g.nlon[k];
    const C2RIn<R> in{four + g.foff[k] * (long)ncolp, ch, ncolp, 2 * (out.src[a] + wk.f0), g.mmax[k], h,
                      out.dlam[a] != 0};
    const C2ROut<R> o{out.ptr[a] + (long)wk.f0 * npts + g.roff[k], ch, npts, h, (R)sc};
    bluestein(buf, stride, nb, logM, filt + f.floff[k], tw, in, o);
}

// ------------------------------------------------------------------ r2c
// a_q = conj(z_q) w_q, z_q = f_{2q} + i f_{2q+1} (DFT via the inverse kernel)
template <typename R>
struct R2CIn {
    typedef typename Cplx<R>::T C;
    const double* src;
    const C* ch;
    long npts;
    int h;
    __device__ C operator()(int b, int q) const
    {
        if (q >= h) return mk<C>(0, 0);
        const double2 d = *(const double2*)(src + (long)b * npts + 2 * q);
        return cmul(mk<C>(d.x, -d.y), ch[q]);
    }
};

// Z_q = conj(w_q conv_q) = DFT_h(z)_q, kept in shared memory for the fold
template <typename R>
struct R2COut {
    typedef typename Cplx<R>::T C;
    C* buf;
    const C* ch;
    int stride, h;
    __device__ void operator()(int b, int q, C v) const
    {
        if (q < h) buf[(long)b * stride + pad(q)] = conjg(cmul(v, ch[q]));
    }
};

template <typename R>
__global__ void __launch_bounds__(FftThreads<R>::N, FftThreads<R>::MINB)
    k_r2c(AnalIn in, RingGeom g, RingFFT f, LegGeom lg, const typename Cplx<R>::T* __restrict__ chirp,
          const typename Cplx<R>::T* __restrict__ filt, const typename Cplx<R>::T* __restrict__ tw,
          const FFTWork* __restrict__ work, long npts, R* gop, __nv_bfloat16* gop_lo, __nv_bfloat16* gop_lo2,
          int ncolp, int split)
{
    typedef typename Cplx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FFTWork wk = work[blockIdx.x];
    const int kN = wk.ring, kS = lg.nlat - 1 - kN, a = wk.arr, nb = wk.nb;
    const int h = f.h[kN], logM = f.logM[kN], mmax = g.mmax[kN], stride = padded_len(1 << logM);
    C* buf = (C*)smem_raw;
    C* side = buf + (long)nb * stride;
    const C* ch = chirp + f.choff[kN];
    const C* fl = filt + f.floff[kN];
    double sc = g.w[kN] / (double)g.nlon[kN];
    if (in.scale[a] == 1) sc /= g.coslat[kN];
    else if (in.scale[a] == 2) sc = 1.0;
    const R s = (R)sc;
    const int col0 = 2 * (in.dst[a] + wk.f0);
    for (int hemi = 0; hemi < 2; hemi++) {
        const int k = hemi ? kS : kN;
        const R2CIn<R> gin{in.ptr[a] + (long)wk.f0 * npts + g.roff[k], ch, npts, h};
        const R2COut<R> gout{buf, ch, stride, h};
        bluestein(buf, stride, nb, logM, fl, tw, gin, gout);
        __syncthreads();
        // F_m = E_m + e^{-i pi m/h} O_m from Z_m and conj Z_{h-m}; then the fold
        const int nm = mmax + 1;
        for (int idx = threadIdx.x; idx < nb * nm; idx += blockDim.x) {
            const int b = idx / nm, m = idx - b * nm;
            const C* x = buf + (long)b * stride;
            C Zm = x[pad(m)], Zc = conjg(x[pad(m == 0 ? 0 : h - m)]);
            C sm = cadd(Zm, Zc), d = csub(Zm, Zc);
            C E = mk<C>(0.5 * sm.x, 0.5 * sm.y);
            C O = mk<C>(0.5 * d.y, -0.5 * d.x);  // d / (2i)
            R sn, cs;
            sincos_pi((R)m / (R)h, &sn, &cs);
            C Fm = cadd(E, cmul(O, mk<C>(cs, -sn)));
            if (hemi == 0) {
                side[(long)b * h + m] = Fm;
            } else {
                C FN = side[(long)b * h + m];
                const int l = kN - lg.k0[m];
                const int col = col0 + 2 * b;
                long is = (lg.goff[2 * m] + l) * (long)ncolp + col;
                long ia = (lg.goff[2 * m + 1] + l) * (long)ncolp + col;
                put_split<R>(gop, gop_lo, gop_lo2, is, s * (FN.x + Fm.x), split);
                put_split<R>(gop, gop_lo, gop_lo2, is + 1, s * (FN.y + Fm.y), split);
                put_split<R>(gop, gop_lo, gop_lo2, ia, s * (FN.x - Fm.x), split);
                put_split<R>(gop, gop_lo, gop_lo2, ia + 1, s * (FN.y - Fm.y), split);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- launchers
int launch_c2r(Plan* p, const SynthOut& o, int cls, cudaStream_t s)
{
    const Tables* t = p->tab;
    size_t smem = fft_smem(t, p->opts.prec, false);
    for (int a = 0; a < o.narr; a++) {
        if (!o.ptr[a]) continue;
        SynthOut oa = o;
        // one launch per output array keeps the work list simple
        int n = p->n_c2r_work[cls][a];
        stage_begin(p, s);
        if (p->opts.prec == ST_PREC_FP64) {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_c2r<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            k_c2r<double><<<n, FftThreads<double>::N, smem, s>>>((const double*)p->ws_four, p->ncolp, t->ring(), t->fft(),
                                                t->chirp64, t->filt64, t->tw64, p->d_c2r_work[cls][a], oa,
                                                t->npts);
        } else {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_c2r<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            k_c2r<float><<<n, FftThreads<float>::N, smem, s>>>((const float*)p->ws_four, p->ncolp, t->ring(), t->fft(),
                                               t->chirp32, t->filt32, t->tw32, p->d_c2r_work[cls][a], oa,
                                               t->npts);
        }
        ST_CUDA_TRY(cudaGetLastError());
        stage_end(p, ST_STAGE_C2R, s);
        p->last_launches++;
    }
    return ST_OK;
}

int launch_r2c(Plan* p, const AnalIn& in, int cls, cudaStream_t s)
{
    const Tables* t = p->tab;
    size_t smem = fft_smem(t, p->opts.prec, true);
    for (int a = 0; a < in.narr; a++) {
        int n = p->n_r2c_work[cls][a];
        stage_begin(p, s);
        if (p->opts.prec == ST_PREC_FP64) {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_r2c<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            k_r2c<double><<<n, FftThreads<double>::N, smem, s>>>(in, t->ring(), t->fft(), t->leg(), t->chirp64, t->filt64, t->tw64,
                                                p->d_r2c_work[cls][a], t->npts, (double*)p->ws_four, nullptr,
                                                nullptr, p->ncolp, 0);
        } else {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_r2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            k_r2c<float><<<n, FftThreads<float>::N, smem, s>>>(in, t->ring(), t->fft(), t->leg(), t->chirp32, t->filt32, t->tw32,
                                               p->d_r2c_work[cls][a], t->npts, (float*)p->ws_four,
                                               (__nv_bfloat16*)p->ws_op_lo, (__nv_bfloat16*)p->ws_op_lo2, p->ncolp,
                                               nsplit(p->opts.prec));
        }
        ST_CUDA_TRY(cudaGetLastError());
        stage_end(p, ST_STAGE_R2C, s);
        p->last_launches++;
    }
    return ST_OK;
}

}  // namespace st
