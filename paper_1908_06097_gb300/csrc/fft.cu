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

// Batched in-place radix-2 DIF, natural -> bit-reversed, kernel e^{-2 pi i/L}.
// tw[t] = e^{-2 pi i t / Mmax}; tws = log2(Mmax) - logM.
template <typename C>
__device__ void fft_dif(C* buf, int nb, int logM, const C* __restrict__ tw, int tws)
{
    const int halfM = 1 << (logM - 1);
    const int total = nb * halfM;
    for (int s = 0; s < logM; s++) {
        const int lh = logM - s - 1;
        const int half = 1 << lh;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int b = idx >> (logM - 1);
            const int r = idx & (halfM - 1);
            const int j = r & (half - 1);
            const int i0 = ((r >> lh) << (lh + 1)) + j;
            C* x = buf + ((long)b << logM);
            C u = x[i0], v = x[i0 + half];
            x[i0] = cadd(u, v);
            x[i0 + half] = cmul(csub(u, v), tw[j << (s + tws)]);
        }
        __syncthreads();
    }
}

// Batched in-place radix-2 DIT, bit-reversed -> natural, kernel e^{+2 pi i/L}
// (unnormalised inverse of fft_dif).
template <typename C>
__device__ void fft_dit_inv(C* buf, int nb, int logM, const C* __restrict__ tw, int tws)
{
    const int halfM = 1 << (logM - 1);
    const int total = nb * halfM;
    for (int s = logM - 1; s >= 0; s--) {
        const int lh = logM - s - 1;
        const int half = 1 << lh;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int b = idx >> (logM - 1);
            const int r = idx & (halfM - 1);
            const int j = r & (half - 1);
            const int i0 = ((r >> lh) << (lh + 1)) + j;
            C* x = buf + ((long)b << logM);
            C u = x[i0], v = cmulc(x[i0 + half], tw[j << (s + tws)]);
            x[i0] = cadd(u, v);
            x[i0 + half] = csub(u, v);
        }
        __syncthreads();
    }
}

// Bluestein core: buf holds a_q = x_q w_q (zero-padded to M); on return
// buf[q] (q < h) holds conv_q; the caller multiplies by w_q.
template <typename C>
__device__ __forceinline__ void bluestein_conv(C* buf, int nb, int logM, const C* __restrict__ filt,
                                               const C* __restrict__ tw, int tws)
{
    fft_dif(buf, nb, logM, tw, tws);
    const int M = 1 << logM;
    for (int idx = threadIdx.x; idx < nb * M; idx += blockDim.x) buf[idx] = cmul(buf[idx], filt[idx & (M - 1)]);
    __syncthreads();
    fft_dit_inv(buf, nb, logM, tw, tws);
}

// --------------------------------------------------------------- filters
// filt = FFT_M(b)/M in bit-reversed order, b_t = conj(w_t) for |t| < h (mod M).
__global__ void k_fft_filters(RingFFT f, const double2* __restrict__ chirp, double2* filt64, float2* filt32,
                              const double2* __restrict__ tw, int logMmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = (double2*)smem_raw;
    const int k = blockIdx.x;
    const int h = f.h[k], logM = f.logM[k], M = 1 << logM;
    const double2* ch = chirp + f.choff[k];
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double2 v = mk<double2>(0, 0);
        if (i < h) v = conjg(ch[i]);
        else if (i > M - h) v = conjg(ch[M - i]);
        buf[i] = v;
    }
    __syncthreads();
    fft_dif(buf, 1, logM, tw, logMmax - logM);
    const double inv = 1.0 / M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double2 v = buf[i];
        v.x *= inv;
        v.y *= inv;
        filt64[f.floff[k] + i] = v;
        filt32[f.floff[k] + i] = make_float2((float)v.x, (float)v.y);
    }
}

static int ilog2(int x) { int l = 0; while ((1 << l) < x) l++; return l; }

int launch_fft_filters(Tables* t)
{
    size_t smem = (size_t)t->Mmax * sizeof(double2);
    if (smem > 227 * 1024) {
        set_error("ring FFT length %d exceeds the on-chip limit (T too large)", t->Mmax);
        return ST_ERR_UNSUPPORTED;
    }
    ST_CUDA_TRY(cudaFuncSetAttribute(k_fft_filters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fft_filters<<<t->N, 256, smem>>>(t->fft(), t->chirp64, t->filt64, t->filt32, t->tw64, ilog2(t->Mmax));
    ST_CUDA_TRY(cudaGetLastError());
    ST_CUDA_TRY(cudaDeviceSynchronize());
    return ST_OK;
}

// ------------------------------------------------------------- batching
static size_t fft_cap_bytes(st_prec prec) { return prec == ST_PREC_FP64 ? 180 * 1024 : 96 * 1024; }
static size_t cplx_bytes(st_prec prec) { return prec == ST_PREC_FP64 ? 16 : 8; }

// fields per CTA for ring k (pair: r2c on a north/south pair, which also keeps h
// Fourier coefficients of the north ring on chip)
static int fft_batch_ex(const Tables* t, int k, st_prec prec, bool pair)
{
    size_t need = ((size_t)1 << t->logM[k]) + (pair ? t->hh[k] : 0);
    size_t B = fft_cap_bytes(prec) / (need * cplx_bytes(prec));
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
        size_t need = ((size_t)1 << t->logM[k]) + (pair ? t->hh[k] : 0);
        mx = std::max(mx, (size_t)fft_batch_ex(t, k, prec, pair) * need * cplx_bytes(prec));
    }
    return mx;
}

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

template <typename R>
__global__ void __launch_bounds__(256) k_c2r(const R* __restrict__ four, int ncolp, RingGeom g, RingFFT f,
                                             const typename Cplx<R>::T* __restrict__ chirp,
                                             const typename Cplx<R>::T* __restrict__ filt,
                                             const typename Cplx<R>::T* __restrict__ tw, int logMmax,
                                             const FFTWork* __restrict__ work, SynthOut out, long npts)
{
    typedef typename Cplx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = (C*)smem_raw;
    const FFTWork wk = work[blockIdx.x];
    const int k = wk.ring, a = wk.arr, nb = wk.nb;
    const int h = f.h[k], logM = f.logM[k], M = 1 << logM, mmax = g.mmax[k];
    const C* ch = chirp + f.choff[k];
    const R* F = four + g.foff[k] * (long)ncolp;
    const int src0 = out.src[a] + wk.f0;
    const bool dl = out.dlam[a] != 0;
    for (int idx = threadIdx.x; idx < nb * M; idx += blockDim.x) {
        const int b = idx >> logM, q = idx & (M - 1);
        C v = mk<C>(0, 0);
        if (q < h) {
            const int col = 2 * (src0 + b);
            C Xq = load_X<R, C>(F, ncolp, col, q, mmax, dl);
            C Xh = load_X<R, C>(F, ncolp, col, h - q, mmax, dl);
            C e = cadd(Xq, conjg(Xh)), d = csub(Xq, conjg(Xh));
            R sn, cs;
            sincos_pi((R)q / (R)h, &sn, &cs);
            C t = cmul(d, mk<C>(cs, sn));
            C Z = mk<C>(e.x - t.y, e.y + t.x);  // e + i t
            v = cmul(Z, ch[q]);
        }
        buf[idx] = v;
    }
    __syncthreads();
    bluestein_conv(buf, nb, logM, filt + f.floff[k], tw, logMmax - logM);
    double sc = 1.0;
    if (out.scale[a] == 1) sc = 1.0 / g.coslat[k];
    else if (out.scale[a] == 2) sc = g.w[k] / (double)g.nlon[k];
    double* dst = out.ptr[a] + (long)wk.f0 * npts + g.roff[k];
    for (int idx = threadIdx.x; idx < nb * h; idx += blockDim.x) {
        const int b = idx / h, l = idx - b * h;
        C z = cmul(buf[((long)b << logM) + l], ch[l]);
        *(double2*)(dst + (long)b * npts + 2 * l) = make_double2((double)z.x * sc, (double)z.y * sc);
    }
}

// ------------------------------------------------------------------ r2c
template <typename R>
__device__ __forceinline__ void store_op(R* hi, __nv_bfloat16* lo, long i, double v, bool split)
{
    if (!split) {
        hi[i] = (R)v;
    } else {
        __nv_bfloat16 h = __double2bfloat16(v);
        ((__nv_bfloat16*)hi)[i] = h;
        lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_r2c(AnalIn in, RingGeom g, RingFFT f, LegGeom lg,
                                             const typename Cplx<R>::T* __restrict__ chirp,
                                             const typename Cplx<R>::T* __restrict__ filt,
                                             const typename Cplx<R>::T* __restrict__ tw, int logMmax,
                                             const FFTWork* __restrict__ work, long npts, R* gop,
                                             __nv_bfloat16* gop_lo, int ncolp, int split)
{
    typedef typename Cplx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FFTWork wk = work[blockIdx.x];
    const int kN = wk.ring, kS = lg.nlat - 1 - kN, a = wk.arr, nb = wk.nb;
    const int h = f.h[kN], logM = f.logM[kN], M = 1 << logM, mmax = g.mmax[kN];
    C* buf = (C*)smem_raw;
    C* side = buf + ((long)nb << logM);
    const C* ch = chirp + f.choff[kN];
    const C* fl = filt + f.floff[kN];
    double sc = g.w[kN] / (double)g.nlon[kN];
    if (in.scale[a] == 1) sc /= g.coslat[kN];
    else if (in.scale[a] == 2) sc = 1.0;
    const int col0 = 2 * (in.dst[a] + wk.f0);
    for (int hemi = 0; hemi < 2; hemi++) {
        const int k = hemi ? kS : kN;
        const double* src = in.ptr[a] + (long)wk.f0 * npts + g.roff[k];
        for (int idx = threadIdx.x; idx < nb * M; idx += blockDim.x) {
            const int b = idx >> logM, q = idx & (M - 1);
            C v = mk<C>(0, 0);
            if (q < h) {
                double2 d = *(const double2*)(src + (long)b * npts + 2 * q);
                v = cmul(mk<C>(d.x, -d.y), ch[q]);  // conj(z) w_q
            }
            buf[idx] = v;
        }
        __syncthreads();
        bluestein_conv(buf, nb, logM, fl, tw, logMmax - logM);
        // Z_q = conj(w_q conv_q) = DFT_h(z)_q
        for (int idx = threadIdx.x; idx < nb * h; idx += blockDim.x) {
            const int b = idx / h, q = idx - b * h;
            C* x = buf + ((long)b << logM);
            x[q] = conjg(cmul(x[q], ch[q]));
        }
        __syncthreads();
        const int nm = mmax + 1;
        for (int idx = threadIdx.x; idx < nb * nm; idx += blockDim.x) {
            const int b = idx / nm, m = idx - b * nm;
            const C* x = buf + ((long)b << logM);
            C Zm = x[m], Zc = conjg(x[m == 0 ? 0 : h - m]);
            C s = cadd(Zm, Zc), d = csub(Zm, Zc);
            C E = mk<C>(0.5 * s.x, 0.5 * s.y);
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
                store_op<R>(gop, gop_lo, is, sc * ((double)FN.x + (double)Fm.x), split);
                store_op<R>(gop, gop_lo, is + 1, sc * ((double)FN.y + (double)Fm.y), split);
                store_op<R>(gop, gop_lo, ia, sc * ((double)FN.x - (double)Fm.x), split);
                store_op<R>(gop, gop_lo, ia + 1, sc * ((double)FN.y - (double)Fm.y), split);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- launchers
int launch_c2r(Plan* p, const SynthOut& o, int cls, cudaStream_t s)
{
    const Tables* t = p->tab;
    const int lmx = ilog2(t->Mmax);
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
            k_c2r<double><<<n, 256, smem, s>>>((const double*)p->ws_four, p->ncolp, t->ring(), t->fft(),
                                                t->chirp64, t->filt64, t->tw64, lmx, p->d_c2r_work[cls][a], oa,
                                                t->npts);
        } else {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_c2r<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            k_c2r<float><<<n, 256, smem, s>>>((const float*)p->ws_four, p->ncolp, t->ring(), t->fft(),
                                               t->chirp32, t->filt32, t->tw32, lmx, p->d_c2r_work[cls][a], oa,
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
    const int lmx = ilog2(t->Mmax);
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
            k_r2c<double><<<n, 256, smem, s>>>(in, t->ring(), t->fft(), t->leg(), t->chirp64, t->filt64, t->tw64,
                                                lmx, p->d_r2c_work[cls][a], t->npts, (double*)p->ws_four, nullptr,
                                                p->ncolp, 0);
        } else {
            static bool once = false;
            if (!once) {
                ST_CUDA_TRY(cudaFuncSetAttribute(k_r2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
                once = true;
            }
            const bool split = p->opts.prec == ST_PREC_BF16X3;
            k_r2c<float><<<n, 256, smem, s>>>(in, t->ring(), t->fft(), t->leg(), t->chirp32, t->filt32, t->tw32, lmx,
                                               p->d_r2c_work[cls][a], t->npts, (float*)p->ws_four,
                                               split ? (__nv_bfloat16*)p->ws_op_lo : nullptr, p->ncolp, split);
        }
        ST_CUDA_TRY(cudaGetLastError());
        stage_end(p, ST_STAGE_R2C, s);
        p->last_launches++;
    }
    return ST_OK;
}

}  // namespace st
