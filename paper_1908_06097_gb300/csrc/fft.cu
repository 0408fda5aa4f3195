// Ring FFTs of the spectral transform: host side (descriptors, work lists,
// launches).  The kernels and the method are in fft_kernels.cuh; each kernel
// and precision is compiled in a translation unit of its own.
#include <string.h>

#include <algorithm>

#include "st_internal.cuh"

namespace st {

FftDesc fft_desc(const Plan* p)
{
    const Tables* t = p->tab;
    FftDesc d;
    memset(&d, 0, sizeof d);
    d.g = t->ring();
    d.f = t->fft();
    d.k0 = t->d_k0;
    d.goff = t->d_goff;
    d.chirp64 = t->chirp64;
    d.chirp32 = t->chirp32;
    d.filt64 = t->filt64;
    d.filt32 = t->filt32;
    d.tw64 = t->tw64;
    d.tw32 = t->tw32;
    d.four = p->ws_four;
    d.lo = (__nv_bfloat16*)p->ws_op_lo;
    d.lo2 = (__nv_bfloat16*)p->ws_op_lo2;
    d.g32 = (float*)p->ws_gop32;
    d.npts = t->npts;
    d.ngop_rows = t->ngop_rows;
    d.ncolp = p->ncolp;
    d.nlat = t->nlat;
    d.split = nsplit(p->opts.prec);
    d.nfld = p->nfld;
    d.status = p->d_status;
    d.checks = (p->opts.flags & ST_FLAG_CHECKS) ? 1 : 0;
    return d;
}

int fft_log_len(int nlon, int K)
{
    int l = 5;
    while ((1 << l) < nlon + 2 * K - 2) l++;
    return l;
}

// Work list of a plan: one item per (ring pair, field), sorted by transform
// length (longest first), then ring pair, then field; CTAs take points/M
// consecutive items of one length (points = fft_cta_points).
int build_fft_worklists(Plan* p)
{
    const Tables* t = p->tab;
    std::vector<int4> items;
    for (int k = 0; k < t->N; k++)
        if (owns_ring(p, k))
            for (int f = 0; f < p->nfld; f++) items.push_back(make_int4(k, f, 0, 0));
    std::stable_sort(items.begin(), items.end(),
                     [&](const int4& a, const int4& b) { return t->logM[a.x] > t->logM[b.x]; });
    const std::vector<int4> ctas =
        fft_ctas(items, [&](const int4& it) { return t->logM[it.x]; }, fft_cta_points(p->opts.prec));
    int4 *di = nullptr, *dc = nullptr;
    if (dev_malloc((void**)&di, std::max<size_t>(items.size(), 1) * sizeof(int4)) != cudaSuccess ||
        dev_malloc((void**)&dc, std::max<size_t>(ctas.size(), 1) * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        if (di) cudaFree(di);
        return ST_ERR_NOMEM;
    }
    p->d_fft_items = di;  // owned by the plan from here (freed with it)
    p->d_fft_ctas = dc;
    if (!items.empty()) ST_CUDA_TRY(cudaMemcpy(di, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!ctas.empty()) ST_CUDA_TRY(cudaMemcpy(dc, ctas.data(), ctas.size() * sizeof(int4), cudaMemcpyHostToDevice));
    p->n_fft_ctas = (int)ctas.size();
    return ST_OK;
}

int launch_fft(bool inverse, st_prec prec, const FftIO& io, int nctas, cudaStream_t s)
{
    if (nctas <= 0 || io.narr <= 0) return ST_OK;
    if (prec == ST_PREC_FP64) return inverse ? launch_c2r_f64(io, nctas, s) : launch_r2c_f64(io, nctas, s);
    return inverse ? launch_c2r_f32(io, nctas, s) : launch_r2c_f32(io, nctas, s);
}

int launch_c2r(Plan* p, const SynthOut& o, int, cudaStream_t s)
{
    FftIO io;
    memset(&io, 0, sizeof io);
    io.d0 = fft_desc(p);
    io.items = p->d_fft_items;
    io.ctas = p->d_fft_ctas;
    for (int a = 0; a < o.narr; a++) {
        if (!o.ptr[a]) continue;
        const int k = io.narr++;
        io.out[k] = o.ptr[a];
        io.col[k] = o.src[a];
        io.dlam[k] = (unsigned char)(o.dlam[a] != 0);
        io.scale[k] = (unsigned char)o.scale[a];
    }
    if (!io.narr) return ST_OK;
    stage_begin(p, ST_STAGE_C2R, s);
    int rc = launch_fft(true, p->opts.prec, io, p->n_fft_ctas, s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    stage_end(p, ST_STAGE_C2R, s);
    p->last_launches++;
    return ST_OK;
}

int launch_r2c(Plan* p, const AnalIn& in, int, cudaStream_t s, bool split_now)
{
    FftIO io;
    memset(&io, 0, sizeof io);
    io.d0 = fft_desc(p);
    io.items = p->d_fft_items;
    io.ctas = p->d_fft_ctas;
    for (int a = 0; a < in.narr; a++) {
        io.in[io.narr] = in.ptr[a];
        io.col[io.narr] = in.dst[a];
        io.scale[io.narr] = (unsigned char)in.scale[a];
        io.narr++;
    }
    stage_begin(p, ST_STAGE_R2C, s);
    int rc = launch_fft(false, p->opts.prec, io, p->n_fft_ctas, s);
    if (rc) {
        stage_fail(p);
        return rc;
    }
    if (io.d0.g32 && split_now) {
        // split paths: FP32 operand -> bf16 planes (timed with the r2c stage)
        int ncols = 0;  // slot a writes columns 2 (col[a] + f), +1, f < nfld
        for (int a = 0; a < io.narr; a++) ncols = std::max(ncols, 2 * (io.col[a] + p->nfld));
        rc = launch_split_gop(io.d0, nullptr, 1, ncols, s);
        if (rc) {
            stage_fail(p);
            return rc;
        }
        p->last_launches++;
    }
    stage_end(p, ST_STAGE_R2C, s);
    p->last_launches++;
    return ST_OK;
}

}  // namespace st
