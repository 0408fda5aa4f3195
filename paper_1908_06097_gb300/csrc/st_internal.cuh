// Internal declarations of the GB300 spectral-transform library.
//
// Data layout in HBM (all row-major, no padding beyond what TMA needs):
//   Legendre table   block (m, p) = [K_{m,p}][Lp_m], p = parity of n - m,
//                    row k holds n = m + p + 2k (n <= T+1), column l the
//                    northern ring k0(m) + l; Lp_m = L_m rounded up to 8.
//   inverse operand  Aop block (m, p) = [K_{m,p}][ncolp], column c = 2 f + (re|im)
//   Fourier buffer   four[ring][m][ncolp], ring-major (the transposed layout)
//   direct operand   Gop block (m, p) = [Lp_m][ncolp] (folded, weighted)
//   direct result    Sop block (m, p) = [K_{m,p}][ncolp]
// The transposition between the m-major spectral side and the ring-major grid
// side is done by the Legendre epilogue (inverse) and by the ring-FFT epilogue
// (direct), so no kernel only moves data.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/st.h"

namespace st {

struct Plan;

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
#define ST_CUDA_TRY(expr)                                                               \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::st::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return ST_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

// Every device allocation of the library goes through dev_malloc, so that a
// test can make one of them fail (st_debug_fail_alloc).
cudaError_t dev_malloc(void** p, size_t bytes);

// ---------------------------------------------------------- device params
// Per-ring geometry (index k = 0..NLAT-1, north -> south).
struct RingGeom {
    const int* nlon;      // points on the ring
    const int* mmax;      // highest wavenumber carried
    const long* roff;     // first grid point of the ring
    const long* foff;     // first Fourier row (units of ncolp) of the ring: sum (mmax+1)
    const double* coslat; // cos(phi_k)
    const double* w;      // Gauss weight
    const double* sc64;   // per-ring scales [k][4]: 1, 1/cos(phi), w/nlon, w/(nlon cos(phi))
    const float* sc32;    // the same in FP32
};
enum { SC_ONE = 0, SC_INVCOS = 1, SC_WN = 2, SC_WNCOS = 3 };

// Per-wavenumber Legendre geometry.
struct LegGeom {
    const int* k0;    // first northern ring carrying m
    const int* L;     // number of northern rings carrying m
    const int* Lp;    // L rounded up to 8 (row length of a table / operand block)
    const long* toff; // [2m+p] element offset of table block (m,p)
    const long* aoff; // [2m+p] row offset of operand block (m,p) (rows of ncolp)
    const long* goff; // [2m+p] row offset of direct operand block (m,p)
    const double* eps; // eps_n^m for n = m..T+2 at eoff(m) + n - m (see eps_off)
    const double2* bc; // ((n+2) eps_{n+1}, (n-1) eps_n) at eps_off(T, m) + n - m (d/dphi recurrence)
    const double2* hc; // (-n eps_{n+1}, (n+1) eps_n), same index (wind recombination)
    const float2* bc32; // bc in FP32
    const float4* hc32; // hc as FP32 pairs: (hi(hc.x), lo(hc.x), hi(hc.y), lo(hc.y)), hi + lo = hc
    int T, N, nlat;
};

// start of wavenumber m in the eps table: sum_{m' < m} (T + 3 - m')
__host__ __device__ inline long eps_off(int T, int m) { return (long)m * (2 * T + 7 - m) / 2; }

// Polar rings of the 1/cos(phi) syntheses (d/dphi, winds): the northern rings
// k < np with cos(phi_k) < ST_POLAR_COS, and an FP64 table of P_n^m(mu_k) for
// them, n = m..T+1, at pt[poff[k (T+1) + m] + n - m] (built in long double).
#define ST_POLAR_COS 0.012
struct PolarGeom {
    int np;
    const long* poff;
    const double* pt;
    const double* fac;  // -1/(n(n+1)) for n = 0..T+1 (0 at n = 0): psi, chi from zeta, D
    const double* gt;   // G_n^m = (n+1) eps_n P_{n-1} - n eps_{n+1} P_{n+1} (cos(phi) dP/dphi), layout of pt
    const float* pt32;  // FP32 copies of pt, gt, fac
    const float* gt32;
    const float* fac32;
};

// Chirp-z plan of one ring pair k < N (north ring k and its mirror): the
// convolution length M = 2^logM >= nlon + 2 (mmax + 1) - 2.
struct RingFFT {
    const int* logM;
    const long* choff; // chirp offset: c_u = exp(i pi u^2/nlon), u = 0..nlon/2
    const long* floff; // filter offset (M entries, digit-reversed order)
};

// ------------------------------------------------------------------ tables
struct Tables {
    int T, kind, N, nlat, refcount;
    long npts;
    std::vector<double> mu, w, coslat;
    // colatitudes of the northern rings as Newton left them (long double),
    // kept as theta_hi + theta_lo: the polar tables are built at these nodes
    std::vector<double> theta_hi, theta_lo;
    std::vector<int> nlon, mmax, k0, L, Lp, K, logM;
    std::vector<long> roff, foff, toff, aoff, goff, choff, floff;
    long nfour_rows;  // sum over rings of (mmax+1)
    long ntab;        // elements of one table copy
    long nops_rows;   // rows of Aop / Sop (sum K)
    long ngop_rows;   // rows of Gop (sum 2 Lp)
    long nchirp, nfilt;
    int Mmax;
    // device copies
    int *d_nlon, *d_mmax, *d_k0, *d_L, *d_Lp, *d_logM;
    long *d_roff, *d_foff, *d_toff, *d_aoff, *d_goff, *d_choff, *d_floff;
    double *d_coslat, *d_w, *d_mu, *d_eps, *d_sc64;
    double2 *d_bc, *d_hc;
    float2* d_bc32;
    float4* d_hc32;
    int npolar;           // polar rings per hemisphere (see PolarGeom)
    long* d_poff;
    double *d_ptab, *d_fac, *d_gtab;
    float *d_ptab32, *d_gtab32, *d_fac32;
    float* d_sc32;
    // FP32 and split plans: P_n^1 at the northern rings k0[1] + l, as FP32
    // (hi, lo) pairs from long double, at pw1[l (T+2) + n], n = 0..T+1 (n = 0
    // is zero); the direct winds at m = 1 are summed from it in double-float
    float2* d_pw1;
    double* P64;
    float* P32;
    __nv_bfloat16 *Phi, *Plo, *Plo2;  // split table planes p0, p1, p2
    double2 *chirp64, *filt64, *tw64;
    float2 *chirp32, *filt32, *tw32;
    void* tmaps;  // device CUtensorMap[3][2(T+1)] of the split table planes
    // on-the-fly Legendre functions (ST_FLAG_OTF): recurrence inputs and
    // checkpoints in place of a stored table
    double2* d_Q;     // Q_m (mantissa, exponent), m = 0..T
    double* d_reps;   // 1/eps_n^m, indexed as d_eps
    void* ckpt;       // checkpoints, built with the first ST_FLAG_OTF plan
    long* d_ckoff;
    long nckpt;
    RingGeom ring() const { return {d_nlon, d_mmax, d_roff, d_foff, d_coslat, d_w, d_sc64, d_sc32}; }
    LegGeom leg() const { return {d_k0, d_L, d_Lp, d_toff, d_aoff, d_goff, d_eps, d_bc, d_hc, d_bc32, d_hc32, T, N, nlat}; }
    RingFFT fft() const { return {d_logM, d_choff, d_floff}; }
    PolarGeom polar() const { return {npolar, d_poff, d_ptab, d_fac, d_gtab, d_ptab32, d_gtab32, d_fac32}; }
};

Tables* tables_acquire(int T, int kind, int N, st_prec prec, bool otf, int* status);
int launch_otf_ckpt(Tables* t);
void tables_release(Tables* t);

// --------------------------------------------------------------- work lists
struct LegTile {  // one CTA of a grouped Legendre launch
    int m, p, r0, c0;  // wavenumber, parity (direct only), first row, first column
    int mb;            // member plan of a group (0 for a single plan)
};
// Legendre kernels: what they read of one plan in one call class, and their
// per-launch arguments (by value; desc = member descriptors of a group).
struct LegDesc {
    LegGeom lg;
    RingGeom rg;
    const void* P;     // SIMT: the plan's table (FP64 or FP32)
    const void* X;     // SIMT: inverse operand (inverse) or direct operand (direct)
    void* Y;           // Fourier buffer (inverse) or direct result (direct)
    const void* tmP;   // tensor cores: CUtensorMap[3][nb] of the split table planes
    const void* tmX;   // tensor cores: CUtensorMap[3][nb] of the split operand planes
    int* status;
    long long wait_limit;  // tensor cores: bound of every mbarrier wait (clocks)
    // FP64 plans without a stored table (ST_FLAG_OTF): recurrence inputs
    const double* mu;      // Gauss nodes
    const double2* Qm;     // Q_m = prod sqrt((2k+1)/(2k)) as (mantissa, exponent)
    const double* reps;    // 1/eps_n^m, indexed as lg.eps
    const void* ckpt;      // recurrence checkpoints (see legendre_simt.cu)
    const long* ckoff;     // [m] first checkpoint of m
    int otf;
    int df;  // ST_FLAG_DF64: double-float contractions (FP64 plans)
    int nb, ncolp, ncol, nmax;
};
// Persistent launches (group calls): ctr points at a zeroed work counter and
// the CTAs of a grid sized to what the GPU holds at once pull the work items
// 0 .. nwork-1 (ordered longest first) from it; ctr NULL: one CTA per item.
struct WorkQueue {
    int* ctr;
    int nwork;
};
// Runs body(item) for the CTA's items: item blockIdx.x for a plain launch,
// or, for a persistent launch, the items it pulls from the counter until the
// list is exhausted (one call site, so the body is inlined once).
template <typename F>
__device__ __forceinline__ void run_items(const WorkQueue& q, F body)
{
    __shared__ int s_item;
    for (int w = blockIdx.x;;) {
        if (q.ctr) {
            __syncthreads();  // the previous item is done and s_item read
            if (threadIdx.x == 0 && threadIdx.y == 0) s_item = atomicAdd(q.ctr, 1);
            __syncthreads();
            w = s_item;
            if (w >= q.nwork) break;
        }
        body(w);
        if (!q.ctr) break;
    }
}
// grid of a persistent launch: the CTAs of `kernel` the GPU holds at once,
// at most nwork
int persistent_grid(const void* kernel, int threads, int smem, int nwork);
struct LegArgs {
    LegDesc d0;
    const LegDesc* desc;
    const LegTile* tiles;
    int nmemb;  // entries of desc (group launches)
    WorkQueue q;
};
// Work-list check of every Legendre kernel, before any barrier or allocation
// (the whole CTA returns on a bad tile): the tile's member, wavenumber,
// parity and first column must lie inside the plan.  A bad tile sets
// ST_ERR_CHECK in the plan's status word (or the status word of member 0 of a
// group when the member index itself is bad) and its CTA does nothing.
__device__ __forceinline__ bool leg_tile_ok(const LegArgs& A, const LegTile& tl)
{
    const bool mb_ok = A.desc ? (tl.mb >= 0 && tl.mb < A.nmemb) : tl.mb == 0;
    const LegDesc& D = A.desc ? A.desc[mb_ok ? tl.mb : 0] : A.d0;
    const bool ok = mb_ok && tl.m >= 0 && tl.m <= D.lg.T && (tl.p == 0 || tl.p == 1) && tl.r0 >= 0 && tl.c0 >= 0 &&
                    tl.c0 < D.ncolp;
    if (!ok && threadIdx.x == 0 && threadIdx.y == 0) atomicMax(D.status, (int)ST_ERR_CHECK);
    return ok;
}
LegDesc leg_desc(const Plan* p, bool inverse, int nleg, int nmax);
int launch_leg(bool inverse, st_prec prec, const LegArgs& A, int ntiles, int bn, cudaStream_t s);
// Ring-FFT work: an item is one transform (x = ring pair, y = field,
// z = member plan of a group); a CTA entry is (x = first item, y = items,
// z = logM) and covers 8192 points.

// ------------------------------------------------------------------- plan
enum CallKind { CALL_INV = 0, CALL_DIR = 1 };

// Partition of a plan among ranks (st_plan_set_partition): the rank owns the
// wavenumbers m with m_owner[m] == rank (Legendre and spectral stages) and the
// northern ring pairs k with ring_owner[k] == rank (ring FFTs).  The exchange
// row lists are built once: for each direction (0 inverse: Fourier buffer
// rows foff[k] + m; 1 direct: operand rows goff[2m + p] + l), the rows sent
// to every peer and the rows received from every peer, concatenated by peer.
struct PartInfo {
    int nranks, rank;
    std::vector<int> m_owner, ring_owner;
    std::vector<long> send_cnt[2], recv_cnt[2];
    long* d_send[2];
    long* d_recv[2];
    unsigned char* d_mown;  // [T+1]: 1 where this rank owns m
    long nsend[2], nrecv[2];
};

struct Plan {
    int T, nfld;
    st_grid grid;
    st_opts opts;
    Tables* tab;
    int ncolp;        // columns of the operands: 2 * (2 nfld) rounded up to 8
    int leg_bn[2];    // Legendre tile widths (inverse, direct): default or autotuned
    int last_launches;
    // workspaces (bytes); reused across call kinds
    void* ws_four;  // Fourier buffer, or the direct operand (aliased)
    void* ws_op;    // inverse operand, or the direct result (aliased)
    void* ws_op_lo; // split plane p1 of the operands (BF16X3, BF16X6)
    void* ws_op_lo2; // split plane p2 of the operands (BF16X6)
    void* ws_gop32; // split paths: FP32 direct operand written by the r2c fold,
                    // split into the planes by k_split_gop
    size_t ws_four_b, ws_op_b, ws_lo_b;  // sizes of ws_four, ws_op, ws_op_lo (= ws_op_lo2)
    int* d_status;  // device status word
    long long wait_limit;  // bound of the tensor-core kernels' mbarrier waits (clocks)
    PartInfo* part;        // NULL: the plan owns every wavenumber and ring pair
    // st_debug_corrupt_worklist: the entries it overwrote (what != 0)
    int dbg_what;
    LegTile dbg_tile;
    int4 dbg_item;
    // work lists for nleg in {nfld, 2 nfld}
    LegTile *d_inv_tiles[2], *d_dir_tiles[2];
    int n_inv_tiles[2], n_dir_tiles[2];
    int4 *d_fft_items, *d_fft_ctas;  // ring-FFT work list (see above)
    int n_fft_ctas;
    int2* d_spec_chunks;  // (m, n0) chunks of 32 coefficients, n <= T+1
    int n_spec_chunks;
    size_t bytes;
    void *amaps, *gmaps;  // device CUtensorMap[3][2(T+1)] of the split operands
    // optional per-stage CUDA-event timing
    cudaEvent_t* ev;      // 2 * ST_EV_POOL events
    int* ev_stage;        // stage of pair i
    int ev_used, ev_overflow;
};

enum { ST_EV_POOL = 4096 };
// default bound of a device-side wait: about a second at the GB300 SM clock
constexpr long long ST_WAIT_LIMIT_DEFAULT = 1LL << 31;
// bracket one kernel launch with events when the plan times its stages
void stage_begin(Plan* p, int stage, cudaStream_t s);
void stage_fail(Plan* p);  // a stage that returns an error: closes its NVTX range
void stage_end(Plan* p, int stage, cudaStream_t s);

// ------------------------------------------------------------ launchers
// Field-class descriptors passed by value.
struct SynthOut {       // inverse ring FFT outputs
    double* ptr[4];     // up to 4 grid arrays of nf fields each
    int src[4];         // Legendre field index of field 0 of array a
    int dlam[4];        // 1: multiply F_m by i m (d/dlambda)
    int scale[4];       // 0: none, 1: 1/cos(phi), 2: w/nlon
    int narr, nf;
};
struct AnalIn {         // direct ring FFT inputs
    const double* ptr[2];
    int dst[2];         // Legendre field index of field 0 of array a
    int scale[2];       // 0: w/nlon (direct), 1: w/(nlon cos phi) (direct uv), 2: 1 (adjoint)
    int narr, nf;
};

enum PreMode { PRE_PLAIN = 0, PRE_DERIV = 1, PRE_UV = 2, PRE_HALF = 3 };
enum PostMode { POST_PLAIN = 0, POST_UV = 1, POST_CM = 2 };

// Spectral pre/post kernels: what they read of one plan, and their per-launch
// arguments (by value).  A group launch gives desc (member descriptors) and
// work (x = member, y = chunk, z = first field per CTA); pa/pb are the
// members' spectral inputs (pre) or outputs (post).
enum { ST_GROUP_MAX = 256 };
struct SpecDesc {
    LegGeom lg;
    const int2* chunks;  // (m, n0): 32 degrees of one m
    void* op;            // inverse operand (pre) / direct result (post), plane 0
    __nv_bfloat16 *lo, *lo2;
    double radius;
    int* status;         // the plan's device status word
    int T, ncolp, split, nf;
    int checks;          // ST_FLAG_CHECKS: report non-finite inputs as ST_ERR_CHECK
};
struct SpecArgs {
    SpecDesc d0;
    const SpecDesc* desc;
    const int4* work;
    WorkQueue q;           // group launches: persistent over the work list
    int mode, nmax_extra;  // nmax = T + nmax_extra
    double* pa[ST_GROUP_MAX];
    double* pb[ST_GROUP_MAX];
};
SpecDesc spec_desc(const Plan* p);
int launch_spec(bool pre, st_prec prec, const SpecArgs& A, dim3 grid, cudaStream_t s);
int launch_pre(Plan* p, PreMode mode, const double* a, const double* b, int nf, cudaStream_t s);
// recompute the Fourier rows of the polar rings of a 1/cos(phi) synthesis in
// FP64 (PRE_DERIV: the d/dphi half; PRE_UV: U and V), after the Legendre step
int launch_polar(Plan* p, PreMode mode, const double* a, const double* b, cudaStream_t s);
int launch_post(Plan* p, PostMode mode, double* a, double* b, int nf, cudaStream_t s);
// FP32 and split plans: recompute the m = 1 coefficients of the direct winds
// (vorticity, divergence) from the FP32 direct operand with double-float
// Legendre sums, after launch_post(POST_UV); no-op on FP64 plans
int launch_wind_m1(Plan* p, double* vor, double* div, cudaStream_t s);
int launch_leg_inv(Plan* p, int nleg, cudaStream_t s);
int launch_leg_dir(Plan* p, int nleg, int nmax, cudaStream_t s);
int launch_c2r(Plan* p, const SynthOut& o, int cls, cudaStream_t s);
int launch_r2c(Plan* p, const AnalIn& in, int cls, cudaStream_t s, bool split_now = true);
int launch_table_gen(Tables* t, st_prec prec);
int launch_fft_filters(Tables* t);

int build_fft_worklists(Plan* p);
int build_leg_worklists(Plan* p);  // Legendre tiles, spectral chunks and ring-FFT items
void free_leg_worklists(Plan* p);
void part_free(Plan* p);
// ownership under a partition (true for an unpartitioned plan)
inline bool owns_m(const Plan* p, int m) { return !p->part || p->part->m_owner[m] == p->part->rank; }
inline bool owns_ring(const Plan* p, int k) { return !p->part || p->part->ring_owner[k] == p->part->rank; }
// host copies of a plan's Legendre tile lists for call class cls (0: nleg =
// nfld, 1: nleg = 2 nfld), longest first
void leg_tiles(const Plan* p, int cls, int bn_inv, int bn_dir, std::vector<LegTile>& inv, std::vector<LegTile>& dir);
// Legendre tile shapes: rows per tile, and the candidate widths the autotuner
// tries (variant 0 is the default)
int leg_bm(st_prec prec);
int leg_bn_candidate(st_prec prec, int variant);
// time one Legendre launch (min of reps, ms) on stream 0
float time_leg(bool inverse, st_prec prec, const LegArgs& A, int ntiles, int bn, int reps);
// CTA entries (x = first item, y = items, z = logM) over ring-FFT items sorted
// by transform length; logM_of(item) gives an item's length, points the CTA's
// size (fft_cta_points)
// points of one ring-FFT CTA (8192 in every precision)
inline int fft_cta_points(st_prec) { return 8192; }
template <typename F>
std::vector<int4> fft_ctas(const std::vector<int4>& items, F logM_of, int points)
{
    std::vector<int4> ctas;
    for (size_t i = 0; i < items.size();) {
        const int lm = logM_of(items[i]), nx = points >> lm;
        size_t j = i;
        while (j < items.size() && (int)(j - i) < nx && logM_of(items[j]) == lm) j++;
        ctas.push_back(make_int4((int)i, (int)(j - i), lm, 0));
        i = j;
    }
    return ctas;
}

// Ring-FFT kernels: what they read of one plan (device pointers).
struct FftDesc {
    RingGeom g;
    RingFFT f;
    const int* k0;
    const long* goff;
    const double2 *chirp64, *filt64, *tw64;
    const float2 *chirp32, *filt32, *tw32;
    void* four;  // Fourier buffer (c2r input) or direct operand plane 0 (r2c output)
    __nv_bfloat16 *lo, *lo2;
    float* g32;  // split paths: FP32 direct operand (the r2c output), else NULL
    long npts;
    long ngop_rows;  // rows of the direct operand
    int* status;     // the plan's device status word
    int ncolp, nlat, split, nfld;
    int checks;      // ST_FLAG_CHECKS: report a non-finite grid input (r2c)
};
// Per-launch I/O of the ring-FFT kernels (passed by value).  Slot
// s = member * narr + array; gridDim.y = narr arrays per member.
enum { ST_FFT_SLOTS = 256 };
struct FftIO {
    FftDesc d0;             // the plan, when desc is NULL (single-plan launch)
    const FftDesc* desc;    // device array of member descriptors (group launch)
    const int4* items;
    const int4* ctas;
    int narr;
    int nmemb;  // entries of desc (group launches)
    double* out[ST_FFT_SLOTS];        // c2r: grid arrays
    const double* in[ST_FFT_SLOTS];   // r2c: grid arrays
    int col[ST_FFT_SLOTS];            // Legendre field of field 0 of the slot
    unsigned char dlam[ST_FFT_SLOTS]; // c2r: multiply F_m by i m
    unsigned char scale[ST_FFT_SLOTS];  // c2r: 0 none, 1 1/cos, 2 w/nlon; r2c: 0 w/nlon, 1 w/(nlon cos), 2 none
};
FftDesc fft_desc(const Plan* p);
int fft_log_len(int nlon, int K);
int launch_fft(bool inverse, st_prec prec, const FftIO& io, int nctas, cudaStream_t s);
// per kernel and precision (one translation unit each)
int launch_c2r_f32(const FftIO& io, int nctas, cudaStream_t s);
int launch_c2r_f64(const FftIO& io, int nctas, cudaStream_t s);
int launch_r2c_f32(const FftIO& io, int nctas, cudaStream_t s);
int launch_r2c_f64(const FftIO& io, int nctas, cudaStream_t s);
// split paths: the FP32 direct operand into the bf16 planes, every row,
// columns < ncols (ncols 0: 2 nfld of each member), for one plan (desc NULL:
// d0) or for nmemb group members (desc: device array of their descriptors)
int launch_split_gop(const FftDesc& d0, const FftDesc* desc, int nmemb, int ncols, cudaStream_t s);
int tc_table_maps(Tables* t, void** d_maps);
int tc_plan_maps(Plan* p, void** d_amaps, void** d_gmaps);

inline long round_up(long x, long a) { return (x + a - 1) / a * a; }
inline bool is_split(st_prec p) { return p == ST_PREC_BF16X3 || p == ST_PREC_BF16X6; }
inline int nsplit(st_prec p) { return p == ST_PREC_BF16X6 ? 3 : (p == ST_PREC_BF16X3 ? 2 : 0); }

// double -> float, round to nearest even, by integer operations on the IEEE
// encodings (GB300's FP64 pipe, where the hardware conversion runs, is
// narrow).  Results below the smallest normal float (2^-126) are rounded to
// the float subnormals (or to zero, or up to 2^-126); beyond the float range,
// infinity; NaN, a quiet NaN.
__device__ __forceinline__ float dbl2flt_rn(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned s = hi & 0x80000000u, e = (hi >> 20) & 0x7FFu;
    const int ef = (int)e - 896;  // float exponent field
    // 52-bit mantissa -> 23 bits: add half an ulp minus one, plus the kept
    // lsb (ties to even), then drop 29 bits; a carry moves into the exponent
    // (and from 254 into infinity)
    const unsigned long long m = ((unsigned long long)(hi & 0xFFFFFu) << 32) | lo;
    const unsigned long long r = m + 0x0FFFFFFFull + ((m >> 29) & 1ull);
    unsigned bits = s + ((unsigned)ef << 23) + (unsigned)(r >> 29);
    // float subnormal range (rare): the hardware conversion, which rounds
    // there as IEEE 754 asks; the integer steps above stay the common path
    if (ef <= 0) bits = __float_as_uint(__double2float_rn(d));
    bits = (ef >= 255 && e != 0x7FFu) ? (s | 0x7F800000u) : bits;         // overflow
    bits = e == 0x7FFu ? (s | 0x7F800000u | (m ? 0x400000u : 0u)) : bits;  // inf, NaN
    return __uint_as_float(bits);
}
__device__ __forceinline__ float to_flt(float x) { return x; }
__device__ __forceinline__ float to_flt(double x) { return dbl2flt_rn(x); }

// float -> double, exact for every float (subnormals, infinities and NaNs
// included), by integer operations, branch free
__device__ __forceinline__ double to_dbl(double x) { return x; }
__device__ __forceinline__ double to_dbl(float f)
{
    const unsigned u = __float_as_uint(f), s = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    // normal, infinity, NaN: re-bias the exponent (0xFF maps to 0x7FF)
    unsigned hi = s | ((e == 0xFFu ? 0x7FFu : e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0u) {  // zero or subnormal: normalise the mantissa
        const int k = 31 - __clz((int)(m | 1u));  // top bit of m (m = 0: k = 0)
        const unsigned long long F = (unsigned long long)(m ^ (1u << k)) << (52 - k);
        hi = m ? (s | ((unsigned)(k + 874) << 20) | (unsigned)(F >> 32)) : s;
        lo = m ? (unsigned)F : 0u;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// Write v into split planes (nsplit 2 or 3: p0 = bf16(x), p1 = bf16(x - p0),
// p2 = bf16(x - p0 - p1), x = fp32(v); the residuals are exact in FP32) or,
// for nsplit 0, as the native real type.
template <typename R, typename V>
__device__ __forceinline__ void put_split(R* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long i, V v, int ns)
{
    if (ns == 0) {
        p0[i] = (R)v;
        return;
    }
    const float x = to_flt(v);
    const __nv_bfloat16 a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r1);
    ((__nv_bfloat16*)p0)[i] = a;
    p1[i] = b;
    if (ns == 3) p2[i] = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

}  // namespace st
