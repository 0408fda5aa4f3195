// Transform entry points: each call enqueues a fixed kernel sequence on the
// caller's stream, with no synchronisation and no allocation.
//
//   inverse   pre (operand build) -> Legendre (+ N/S combine, transposed write)
//             [-> FP64 polar rows of the 1/cos(phi) syntheses] -> ring c2r FFT
//             (+ per-ring scale)
//   direct    ring r2c FFT (+ N/S fold, weights, transposed write) -> Legendre
//             -> post (scatter to spectral, uv recombination)
// The adjoints reuse the same kernels: A^T = c_m . direct-without-weights,
// B^T = (w/nlon) . inverse-with-halved-m>0 (see include/st.h).
#include <string.h>

#include "st_internal.cuh"

using namespace st;

static int check_plan(st_plan* pp, const char* fn)
{
    if (!pp) {
        set_error("%s: NULL plan", fn);
        return ST_ERR_ARG;
    }
    return ST_OK;
}

#define NEED(ptr, fn)                                   \
    do {                                                \
        if (!(ptr)) {                                   \
            set_error("%s: " #ptr " is NULL", fn);      \
            return ST_ERR_ARG;                          \
        }                                               \
    } while (0)

#define TRY(x)                     \
    do {                           \
        int rc_ = (x);             \
        if (rc_ != ST_OK) return rc_; \
    } while (0)

static int synth(Plan* p, int cls, double* g0, int src0, int sc0, int dl0, double* g1 = nullptr, int src1 = 0,
                 int sc1 = 0, int dl1 = 0, double* g2 = nullptr, int src2 = 0, int sc2 = 0, int dl2 = 0,
                 cudaStream_t s = 0)
{
    SynthOut o;
    memset(&o, 0, sizeof o);
    double* ptr[3] = {g0, g1, g2};
    int src[3] = {src0, src1, src2}, sc[3] = {sc0, sc1, sc2}, dl[3] = {dl0, dl1, dl2};
    for (int a = 0; a < 3; a++) {
        o.ptr[a] = ptr[a];
        o.src[a] = src[a];
        o.scale[a] = sc[a];
        o.dlam[a] = dl[a];
    }
    o.narr = 3;
    o.nf = p->nfld;
    return launch_c2r(p, o, cls, s);
}

static int analyse(Plan* p, int cls, const double* g0, const double* g1, int scale, cudaStream_t s,
                   bool split_now = true)
{
    AnalIn in;
    memset(&in, 0, sizeof in);
    in.ptr[0] = g0;
    in.ptr[1] = g1;
    in.dst[0] = 0;
    in.dst[1] = p->nfld;
    in.scale[0] = in.scale[1] = scale;
    in.narr = g1 ? 2 : 1;
    in.nf = p->nfld;
    return launch_r2c(p, in, cls, s, split_now);
}

extern "C" {

int st_inv_transform(st_plan* pp, const double* spec, double* grid, void* stream)
{
    TRY(check_plan(pp, "st_inv_transform"));
    NEED(spec, "st_inv_transform");
    NEED(grid, "st_inv_transform");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(launch_pre(p, PRE_PLAIN, spec, nullptr, p->nfld, s));
    TRY(launch_leg_inv(p, p->nfld, s));
    TRY(launch_polar(p, PRE_PLAIN, spec, nullptr, s));  // FP64 plans only
    return synth(p, 0, grid, 0, 0, 0, nullptr, 0, 0, 0, nullptr, 0, 0, 0, s);
}

int st_inv_transform_deriv(st_plan* pp, const double* spec, double* grid, double* dlam, double* dphi, void* stream)
{
    TRY(check_plan(pp, "st_inv_transform_deriv"));
    NEED(spec, "st_inv_transform_deriv");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    if (!grid && !dlam && !dphi) return ST_OK;
    if (dphi) {
        TRY(launch_pre(p, PRE_DERIV, spec, nullptr, p->nfld, s));
        TRY(launch_leg_inv(p, 2 * p->nfld, s));
        TRY(launch_polar(p, PRE_DERIV, spec, nullptr, s));
        return synth(p, 1, grid, 0, 0, 0, dlam, 0, 0, 1, dphi, p->nfld, 1, 0, s);
    }
    TRY(launch_pre(p, PRE_PLAIN, spec, nullptr, p->nfld, s));
    TRY(launch_leg_inv(p, p->nfld, s));
    TRY(launch_polar(p, PRE_PLAIN, spec, nullptr, s));  // FP64 plans only
    return synth(p, 0, grid, 0, 0, 0, dlam, 0, 0, 1, nullptr, 0, 0, 0, s);
}

int st_inv_transform_uv(st_plan* pp, const double* vor, const double* div, double* u, double* v, void* stream)
{
    TRY(check_plan(pp, "st_inv_transform_uv"));
    NEED(vor, "st_inv_transform_uv");
    NEED(div, "st_inv_transform_uv");
    NEED(u, "st_inv_transform_uv");
    NEED(v, "st_inv_transform_uv");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(launch_pre(p, PRE_UV, vor, div, p->nfld, s));
    TRY(launch_leg_inv(p, 2 * p->nfld, s));
    TRY(launch_polar(p, PRE_UV, vor, div, s));
    return synth(p, 1, u, 0, 1, 0, v, p->nfld, 1, 0, nullptr, 0, 0, 0, s);
}

int st_dir_transform(st_plan* pp, const double* grid, double* spec, void* stream)
{
    TRY(check_plan(pp, "st_dir_transform"));
    NEED(grid, "st_dir_transform");
    NEED(spec, "st_dir_transform");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(analyse(p, 0, grid, nullptr, 0, s));
    TRY(launch_leg_dir(p, p->nfld, p->T, s));
    return launch_post(p, POST_PLAIN, spec, nullptr, p->nfld, s);
}

int st_dir_transform_uv(st_plan* pp, const double* u, const double* v, double* vor, double* div, void* stream)
{
    TRY(check_plan(pp, "st_dir_transform_uv"));
    NEED(u, "st_dir_transform_uv");
    NEED(v, "st_dir_transform_uv");
    NEED(vor, "st_dir_transform_uv");
    NEED(div, "st_dir_transform_uv");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(analyse(p, 1, u, v, 1, s));
    TRY(launch_leg_dir(p, 2 * p->nfld, p->T + 1, s));
    TRY(launch_post(p, POST_UV, vor, div, p->nfld, s));
    return launch_wind_m1(p, vor, div, s);  // FP32 and split plans: m = 1 in double-float
}

int st_inv_adjoint(st_plan* pp, const double* grid_cot, double* spec_cot, void* stream)
{
    TRY(check_plan(pp, "st_inv_adjoint"));
    NEED(grid_cot, "st_inv_adjoint");
    NEED(spec_cot, "st_inv_adjoint");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(analyse(p, 0, grid_cot, nullptr, 2, s));
    TRY(launch_leg_dir(p, p->nfld, p->T, s));
    return launch_post(p, POST_CM, spec_cot, nullptr, p->nfld, s);
}

int st_dir_adjoint(st_plan* pp, const double* spec_cot, double* grid_cot, void* stream)
{
    TRY(check_plan(pp, "st_dir_adjoint"));
    NEED(spec_cot, "st_dir_adjoint");
    NEED(grid_cot, "st_dir_adjoint");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(launch_pre(p, PRE_HALF, spec_cot, nullptr, p->nfld, s));
    TRY(launch_leg_inv(p, p->nfld, s));
    return synth(p, 0, grid_cot, 0, 2, 0, nullptr, 0, 0, 0, nullptr, 0, 0, 0, s);
}

// ------------------------------------------------ the two halves of each direction
// For partitioned plans (st_plan_set_partition); on an unpartitioned plan the
// halves compose to st_inv_transform / st_dir_transform.

int st_inv_legendre(st_plan* pp, const double* spec, void* stream)
{
    TRY(check_plan(pp, "st_inv_legendre"));
    NEED(spec, "st_inv_legendre");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    TRY(launch_pre(p, PRE_PLAIN, spec, nullptr, p->nfld, s));
    TRY(launch_leg_inv(p, p->nfld, s));
    return launch_polar(p, PRE_PLAIN, spec, nullptr, s);  // FP64 plans only; own m
}

int st_inv_fourier(st_plan* pp, double* grid, void* stream)
{
    TRY(check_plan(pp, "st_inv_fourier"));
    NEED(grid, "st_inv_fourier");
    Plan* p = (Plan*)pp;
    p->last_launches = 0;
    return synth(p, 0, grid, 0, 0, 0, nullptr, 0, 0, 0, nullptr, 0, 0, 0, (cudaStream_t)stream);
}

int st_dir_fourier(st_plan* pp, const double* grid, void* stream)
{
    TRY(check_plan(pp, "st_dir_fourier"));
    NEED(grid, "st_dir_fourier");
    Plan* p = (Plan*)pp;
    p->last_launches = 0;
    // split paths: the operand stays in FP32 until st_dir_legendre splits it
    return analyse(p, 0, grid, nullptr, 0, (cudaStream_t)stream, false);
}

int st_dir_legendre(st_plan* pp, double* spec, void* stream)
{
    TRY(check_plan(pp, "st_dir_legendre"));
    NEED(spec, "st_dir_legendre");
    Plan* p = (Plan*)pp;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_launches = 0;
    if (p->ws_gop32) {
        FftDesc d = fft_desc(p);
        TRY(launch_split_gop(d, nullptr, 1, 2 * p->nfld, s));
        p->last_launches++;
    }
    TRY(launch_leg_dir(p, p->nfld, p->T, s));
    return launch_post(p, POST_PLAIN, spec, nullptr, p->nfld, s);
}

}  // extern "C"
