/*
 * st.h -- C ABI of the GB300 spectral-transform library (libst_gb300.so).
 *
 * The operation is the spectral-transform dwarf that the ESCAPE report treats
 * as the main challenge of a spectral weather model (Sec. 2.2.2, Sec. 3): the
 * inverse (spectral -> grid) and direct (grid -> spectral) spherical-harmonic
 * transform on a reduced Gaussian grid, taken every timestep.  It has three
 * steps: FFTs along latitude rings, a transposition between the grid/Fourier
 * and the Fourier/spectral layouts, and a Legendre transform for each zonal
 * wavenumber m.  In the paper that transposition is an all-to-all between
 * GPUs, with device-side pack and unpack (Sec. 3.1.1, Sec. 3.1.3.1).  Here one
 * GPU holds every field, and the transposition is a change of memory layout
 * done inside the kernels.  The report does not print the mathematics.
 * This library computes these definitions:
 *
 *   grid      octahedral O(N): ring i = 1..N from each pole has 4i+16 points;
 *             full Gaussian: 4N points on every ring.  NLAT = 2N rings, north
 *             to south, at the Gauss-Legendre nodes mu_k.  lambda_j = 2 pi j/nlon.
 *   basis     orthonormal associated Legendre functions: int P_n^m^2 dmu = 1,
 *             no Condon-Shortley phase.  Ring k carries m <= mmax_k =
 *             min(T, nlon_k/2 - 1).
 *   inverse   f(k,j) = Re F_0 + 2 Re sum_{m=1}^{mmax_k} F_m(k) e^{i m lambda_j},
 *             where F_m(k) = sum_{n=m}^{T} a_n^m P_n^m(mu_k).
 *   direct    a_n^m = sum_{k: m<=mmax_k} w_k P_n^m(mu_k) (1/nlon_k) sum_j f(k,j) e^{-i m lambda_j}
 *
 * I/O layouts (always float64, in device memory, owned by the caller):
 *   spectral  double[nfld][ncoef][2] (re, im), m-major: m = 0..T, then
 *             n = m..T; ncoef = (T+1)(T+2)/2.  On input Im a_n^0 is ignored;
 *             on output it is written as 0.
 *   grid      double[nfld][npts], rings north -> south, each starting at
 *             lambda = 0 and running eastward.
 *
 * Conventions:
 *   - Every call returns an st_status.  On failure it sets a thread-local
 *     message, which st_last_error() returns.
 *   - Transform calls enqueue on the caller's CUDA stream (a cudaStream_t
 *     passed as void*; NULL means the legacy default stream).  They never
 *     synchronise and never allocate, so they can be captured in a CUDA
 *     graph.  The caller keeps the buffers valid until the stream work ends.
 *   - A plan owns its tables and workspaces.  Do not run one plan on two
 *     streams at the same time.  Plans with the same (T, grid) share one set
 *     of read-only Legendre tables.
 *   - Precision affects only the internals of the Legendre step and the FFTs.
 *     FP64: everything in float64.  FP32: FP32 SIMT Legendre and FP32 FFTs.
 *     BF16X3: tensor-core Legendre with each operand split into two bf16
 *     parts (hi + lo).  It sums hi*hi + hi*lo + lo*hi and accumulates in FP32,
 *     which is about 2^-16 relative per term (16 significant bits).  Its FFTs
 *     are FP32.
 *     BF16X6: tensor-core Legendre with each operand split into three bf16
 *     parts (p0 + p1 + p2, 24 significant bits).  It sums the six products
 *     whose order is at least 2^-16 of the leading one (p0p0, p0p1, p1p0,
 *     p0p2, p1p1, p2p0) in FP32, so it keeps FP32-level accuracy on the
 *     tensor cores.  Its FFTs are FP32.
 *   - Errors found on the device (bounded waits that time out, failed
 *     internal checks) set a device status word, which st_sync_status reads.
 *     No kernel traps.
 */
#ifndef ST_H
#define ST_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_plan st_plan;
typedef struct st_group st_group;

typedef enum {
    ST_OK = 0,
    ST_ERR_ARG = 1,         /* bad argument (NULL, size, mismatch) */
    ST_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    ST_ERR_NOMEM = 3,       /* device or host allocation failed */
    ST_ERR_UNSUPPORTED = 4, /* valid request this build does not support */
    ST_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    ST_ERR_CHECK = 6        /* an internal device-side check failed */
} st_status;

typedef enum { ST_GRID_OCTAHEDRAL = 0, ST_GRID_FULL_GAUSSIAN = 1 } st_grid_kind;
typedef enum { ST_PREC_FP64 = 0, ST_PREC_FP32 = 1, ST_PREC_BF16X3 = 2, ST_PREC_BF16X6 = 3 } st_prec;

/* N latitudes per hemisphere; the cubic-octahedral grid TCo T uses N = T + 1. */
typedef struct { st_grid_kind kind; int N; } st_grid;

/* Options (NULL = defaults: FP64, radius 1, flags 0, no tuning cache).
 *   radius      sphere radius a used by the uv variants (winds scale with a).
 *   flags       ST_FLAG_* bits below.
 *   tune_cache  optional path of a text file where the tile autotuner keeps its
 *               choices (read at create, appended after a search); NULL = none. */
typedef struct { st_prec prec; double radius; int flags; const char* tune_cache; } st_opts;

#define ST_FLAG_AUTOTUNE 1     /* time candidate Legendre tile widths at plan (or group) creation */
#define ST_FLAG_STAGE_TIMING 2 /* record CUDA events around every kernel (see st_plan_stage_times) */
#define ST_FLAG_OTF 8          /* FP64 plans only: store no table of the Legendre functions; the Legendre
                                * kernels regenerate them by their recurrence in n, from checkpoints every
                                * 128 degrees (about 1/64 of the table, 0.12 GB instead of 7 GB at
                                * TCo1279).  Results agree with the stored-table path to rounding.
                                * ST_ERR_UNSUPPORTED with another precision or in a group. */
#define ST_FLAG_DF64 16        /* FP64 plans only (not with ST_FLAG_OTF): the Legendre contractions run in
                                * double-float arithmetic (pairs of FP32 values, about 48 significant bits)
                                * on the FP32 pipes, which GB300 issues 64 times faster than FP64.  Table,
                                * operands, ring FFTs, polar rows and outputs stay FP64.  Accuracy: the
                                * FP64 path's error grows by up to about 2^5 (2^-48 against 2^-53 per
                                * operation).  Values of magnitude 3.4e38 or more are out of range.
                                * ST_ERR_UNSUPPORTED with another precision, with ST_FLAG_OTF, or in a
                                * group.  The paper fixes no arithmetic precision (Sec. 3); this is a
                                * faster path at about FP64 accuracy, where the FP64 Legendre sums
                                * take two thirds of an FP64 transform on GB300. */
#define ST_FLAG_CHECKS 4       /* failure detection: the kernels that read the caller's spectral or grid
                                * input report a non-finite value as ST_ERR_CHECK (st_sync_status); the
                                * transform still runs.  The work-list checks of every kernel (a bad
                                * entry is skipped and reported as ST_ERR_CHECK) are always on. */

/* Environment: ST_TC_ONE_TILE=1 makes the split-precision (BF16X3, BF16X6)
 * Legendre stages run the one-CTA-per-tile tensor-core kernels instead of the
 * default persistent ones (one CTA per SM over the tile list).  Both give the
 * same bits; the variable is read once, at the first such launch of the
 * process, and exists for comparison. */

/* Kernel stages reported by st_plan_stage_times. */
enum {
    ST_STAGE_PRE = 0,     /* spectral operand build (derivative / wind recurrences) */
    ST_STAGE_LEG_INV = 1, /* inverse Legendre + north/south combine + transposed write */
    ST_STAGE_C2R = 2,     /* inverse ring FFTs */
    ST_STAGE_R2C = 3,     /* direct ring FFTs + fold + transposed write (split
                           * precisions: + the split of the FP32 operand into
                           * bf16 planes, a second kernel timed in this stage) */
    ST_STAGE_LEG_DIR = 4, /* direct Legendre */
    ST_STAGE_POST = 5,    /* spectral scatter / wind recombination */
    ST_NSTAGES = 6
};

/* Create a plan for truncation T on grid `grid` for `nfld` fields per call.
 * Defines: the set-up of the transform that the paper runs every timestep
 * (Sec. 3, Sec. 3.1.1); the grid, nodes and basis are the definitions at the
 * top of this header (the paper names the resolutions, TCo639 in
 * Sec. 3.1.4 and TCo1279 and TCo1999 in Sec. 3.2.2, but prints neither).
 * Builds the Gauss nodes and the Legendre tables on the device (FP64
 * recurrence, then converted to the plan's precision) and allocates every
 * workspace.  Synchronises the current device.  Requirements: T >= 1;
 * N >= T + 1 for the octahedral grid and 4N >= 2T + 2 for the full grid;
 * 1 <= nfld.  Returns ST_ERR_ARG or ST_ERR_NOMEM on failure. */
int st_plan_create(st_plan** out, int T, st_grid grid, int nfld, const st_opts* opts);

/* Free a plan and its workspaces (the shared tables are freed with their
 * last plan).  Defines: no operation of the paper (resource release).
 * NULL-safe.  Synchronises the device. */
int st_plan_destroy(st_plan* p);

/* Sizes of a plan (grid definition at the top of this header).  Every
 * pointer may be NULL.  *nlon and *ring_off point
 * into host arrays that the plan owns: nlat ring lengths, and nlat+1 offsets
 * into the npts grid points. */
int st_plan_info(const st_plan* p, long* npts, long* ncoef, int* nlat, const int** nlon,
                 const long** ring_off);

/* Copy the NLAT Gauss-Legendre nodes mu_k (descending) and weights w_k into
 * host arrays of NLAT doubles each (the caller owns them; NULL skips one).
 * Defines: the quadrature of the direct transform above (the paper names
 * the TCo resolutions, Sec. 3.1.4 and Sec. 3.2.2, not their grid; nodes and
 * weights are as in the definitions at the top of this header).  ST_ERR_ARG for a NULL plan. */
int st_plan_latitudes(const st_plan* p, double* mu_host, double* w_host);

/* Inverse transform: spec [nfld][ncoef][2] -> grid [nfld][npts] (device
 * arrays owned by the caller; they must not overlap).
 * Defines: the spectral-to-grid half of the spherical-harmonic transform of
 * the dwarf (Sec. 2.2.2, Sec. 3): Legendre sums per m, the transposition that
 * the paper does as an all-to-all with device-side packing (Sec. 3.1.1,
 * Sec. 3.1.3.1), then the ring FFTs; "inverse" above.  Kernels: pre,
 * Legendre (+ transposed write), ring c2r.  ST_ERR_ARG for a NULL plan or
 * pointer; ST_ERR_CUDA if a launch fails.  Device-side faults of the
 * bounded waits are reported by st_sync_status. */
int st_inv_transform(st_plan* p, const double* spec, double* grid, void* cuda_stream);

/* Direct transform: grid [nfld][npts] -> spec [nfld][ncoef][2] (device
 * arrays owned by the caller).
 * Defines: the grid-to-spectral half of the dwarf's transform (Sec. 3,
 * Sec. 3.1.1): ring FFTs, the transposition (Sec. 3.1.3.1), Legendre
 * quadrature per m; "direct" above.  Errors as st_inv_transform. */
int st_dir_transform(st_plan* p, const double* grid, double* spec, void* cuda_stream);

/* Inverse transform with derivatives.
 * Defines: the derivative fields that a spectral model's timestep transforms
 * with its scalars (Sec. 3; the paper does not list them, so the fields are
 * this library's reading of the TCo1279 workload: a scalar and its
 * meridional derivative).  grid = f, dlam = df/dlambda, and
 * dphi = df/dphi, the derivative in latitude on the unit sphere.  dphi is
 * computed by the spectral recurrence to degree T+1, then the 1/cos(phi)
 * scale on the grid.  Any of the three outputs may be NULL, which skips it. */
int st_inv_transform_deriv(st_plan* p, const double* spec, double* grid, double* dlam,
                           double* dphi, void* cuda_stream);

/* Winds from vorticity and divergence.
 * Defines: the vorticity/divergence-to-wind synthesis of a spectral model's
 * timestep (Sec. 3; the paper names the dwarf, not its fields: this is the
 * reading that the ~548 fields of TCo1279 are 137 levels of vorticity,
 * divergence and two scalars).  vor and div each hold nfld fields; u, v
 * are grid arrays of nfld fields (device, caller-owned).  Errors as
 * st_inv_transform.
 * psi = -a^2 vor/(n(n+1)) and chi = -a^2 div/(n(n+1)).  Then
 * u = (1/a)(-dpsi/dphi + dchi/dlambda / cos(phi)) and
 * v = (1/a)(dpsi/dlambda / cos(phi) + dchi/dphi).  a = opts.radius. */
int st_inv_transform_uv(st_plan* p, const double* vor, const double* div, double* u, double* v,
                        void* cuda_stream);

/* Defines: the wind-to-vorticity/divergence analysis, counterpart of
 * st_inv_transform_uv (Sec. 3; same reading).  Errors as st_inv_transform.
 * Vorticity and divergence from winds, the direct counterpart of
 * st_inv_transform_uv: zeta = (1/(a cos phi))(dv/dlambda - d(u cos phi)/dphi),
 * D = (1/(a cos phi))(du/dlambda + d(v cos phi)/dphi), projected on P_n^m.
 * The d/dphi term is integrated by parts onto (1-mu^2) dP/dmu, which needs
 * the degree-T+1 Legendre transform of u/cos(phi) and v/cos(phi).  On FP32
 * and split plans the m = 1 coefficients are summed again in double-float
 * from the same FP32 Fourier operand, with an extra kernel after the
 * recombination.  At m = 1 the recombination differences neighbouring degrees
 * of sums whose terms are about 1e3 times the result, so FP32 sums would be
 * off by about 1e-4 there (all other m: a few 1e-6). */
int st_dir_transform_uv(st_plan* p, const double* u, const double* v, double* vor, double* div,
                        void* cuda_stream);

/* Defines: no passage of the paper (it has no adjoints); this is the exact
 * transpose of the linear map st_inv_transform computes, for gradients.
 * grid_cot [nfld][npts] in, spec_cot [nfld][ncoef][2] out (device, caller-
 * owned).  Errors as st_inv_transform.
 * Adjoint (transpose) of st_inv_transform under the real Euclidean inner
 * products on the grid and on the (Re, Im) spectral pairs; Im a_n^0 is
 * excluded and written as 0:
 *   spec_cot_n^m = c_m sum_k P_n^m(mu_k) sum_j grid_cot(k,j) e^{-i m lambda_j},
 * with c_0 = 1 and c_{m>0} = 2. */
int st_inv_adjoint(st_plan* p, const double* grid_cot, double* spec_cot, void* cuda_stream);

/* Defines: no passage of the paper; the exact transpose of
 * st_dir_transform.  spec_cot in, grid_cot out (device, caller-owned).
 * Errors as st_inv_transform.
 * Adjoint (transpose) of st_dir_transform:
 *   grid_cot(k,j) = (w_k/nlon_k) sum_{m<=mmax_k} Re(S_m(k) e^{i m lambda_j}),
 * with S_m(k) = sum_n spec_cot_n^m P_n^m(mu_k). */
int st_dir_adjoint(st_plan* p, const double* spec_cot, double* grid_cot, void* cuda_stream);

/* A group of plans (any truncations and field counts, same precision): the
 * many independent transforms of one timestep run as ONE kernel launch per
 * stage.  Defines: the batching of independent transforms onto one GPU; the
 * paper's counterpart is its load-balancing by oversubscribing GPUs with
 * several ranks (Sec. 3.1.4.2), replaced here by one work list ordered
 * longest first.  Creating the group merges the members' work lists (every work item
 * tagged with its member, ordered longest first across members) and uploads
 * a descriptor of every member; it allocates device memory and synchronises.
 * At most 256 plans; the plans must outlive the group and must not be used
 * on another stream while a group call that contains them runs (the group
 * uses their workspaces).  ST_ERR_ARG for a NULL plan or mixed precisions,
 * ST_ERR_NOMEM if the merged lists do not fit. */
int st_group_create(st_group** out, st_plan* const* plans, int nplans);

/* Defines: st_inv_transform / st_dir_transform of every member (Sec. 3).
 * Inverse / direct transforms of every member: spec[i], grid[i] are member
 * i's I/O arrays (device pointers, in the layouts above, with member i's
 * field count).  The pointer arrays themselves are host memory and are read
 * during the call; the device pointers are passed by value to the kernels,
 * so a captured CUDA graph replays with the arrays given at capture.  Each
 * call enqueues a fixed number of kernels: three for the inverse (pre,
 * Legendre, ring FFT); three for the direct (ring FFT, Legendre, post) in
 * FP64 and FP32, four in BF16X3 and BF16X6 (the ring FFT writes the FP32
 * operand and one more kernel splits it into the bf16 planes).  It never
 * synchronises and never allocates.  ST_ERR_ARG if a pointer is NULL. */
int st_group_inv(st_group* g, const double* const* spec, double* const* grid, void* cuda_stream);
int st_group_dir(st_group* g, const double* const* grid, double* const* spec, void* cuda_stream);

/* Free a group's merged lists and descriptors (not its plans).  Defines no
 * operation of the paper.  NULL-safe; synchronises the device. */
int st_group_destroy(st_group* g);

/* Kernel launches enqueued by the last st_group_inv / st_group_dir call
 * (accounting; no operation of the paper).  0 for a NULL group. */
int st_group_last_launches(const st_group* g);

/* ---------------------------------------------------- several GPUs
 * The paper's decomposition of the transform (Sec. 3.1.1): every GPU (rank)
 * owns some zonal wavenumbers m, for which it runs the Legendre transform over
 * every latitude, and some latitude ring pairs, for which it runs the ring
 * FFTs; in between, every rank exchanges Fourier coefficients with every other
 * rank once per direction, with the buffer packing on the GPU (Sec. 3.1.3.1)
 * and the messages overlapped (Sec. 3.1.3.2).  The library provides the
 * partitioned plan, the two halves of each direction and the pack/unpack of
 * the exchange; the all-to-all itself is the caller's collective (e.g. NCCL).
 *
 * Partition a plan: m_owner[T+1] gives the rank of every wavenumber and
 * ring_owner[N] the rank of every northern ring pair (with its southern
 * mirror); this plan becomes rank `rank` of `nranks`.  Its Legendre and
 * spectral kernels then cover only its wavenumbers and its ring FFTs only its
 * ring pairs, and the row lists of the exchange are built (the one allocation;
 * the transform calls stay allocation-free).  Synchronises the device.
 * ST_ERR_ARG for an owner outside [0, nranks); ST_ERR_NOMEM. */
int st_plan_set_partition(st_plan* p, int nranks, int rank, const int* m_owner, const int* ring_owner);

/* Rows this rank sends to and receives from every rank in direction dir
 * (0: inverse, Fourier coefficients (ring, m); 1: direct, folded Legendre
 * operand rows (m, parity, ring)), and the bytes of one row (2 nfld values of
 * 8 bytes for FP64 plans, 4 otherwise).  send_rows, recv_rows: host arrays of
 * nranks (NULL skips).  The send buffer holds the rows for rank 0, then for
 * rank 1, ...; the receive buffer the rows from rank 0, then from rank 1, ...
 * ST_ERR_ARG for a plan without a partition. */
int st_exchange_counts(const st_plan* p, int dir, long* send_rows, long* recv_rows, int* row_bytes);

/* Gather this rank's outgoing rows of direction dir into buf (device memory
 * of at least sum(send_rows) * row_bytes bytes, owned by the caller), or
 * scatter the incoming rows from buf into the plan's workspace.  Enqueued on
 * the stream.  ST_ERR_ARG for a plan without a partition or a NULL buf. */
int st_exchange_pack(st_plan* p, int dir, void* buf, void* cuda_stream);
int st_exchange_unpack(st_plan* p, int dir, const void* buf, void* cuda_stream);

/* The halves of the transforms (Sec. 3.1.1).  Inverse: st_inv_legendre
 * computes, for this rank's wavenumbers, the Fourier coefficients of every
 * ring from spec (its rows of the other wavenumbers are not read) into the
 * plan's workspace; after the exchange of direction 0, st_inv_fourier runs
 * the ring FFTs of this rank's ring pairs into grid (other rings untouched).
 * Direct: st_dir_fourier analyses this rank's ring pairs of grid into the
 * workspace; after the exchange of direction 1, st_dir_legendre writes the
 * coefficients of this rank's wavenumbers into spec (others untouched).  On
 * an unpartitioned plan the halves compose to st_inv_transform and
 * st_dir_transform.  Errors as st_inv_transform. */
int st_inv_legendre(st_plan* p, const double* spec, void* cuda_stream);
int st_inv_fourier(st_plan* p, double* grid, void* cuda_stream);
int st_dir_fourier(st_plan* p, const double* grid, void* cuda_stream);
int st_dir_legendre(st_plan* p, double* spec, void* cuda_stream);

/* Failure detection (no passage of the paper; the paper's runs have none).
 * Synchronise the device, then return the worst device status word seen by
 * this plan's kernels since the last call (ST_OK, ST_ERR_TIMEOUT or
 * ST_ERR_CHECK), and clear it.  Also reports a sticky CUDA error as
 * ST_ERR_CUDA. */
int st_sync_status(st_plan* p);

/* Failure detection.  Set the bound, in SM clocks, of every mbarrier wait in
 * this plan's tensor-core kernels (BF16X3, BF16X6; the other kernels have no
 * waits).  0 restores the default, 2^31 clocks (about one second).  A wait
 * that runs out sets ST_ERR_TIMEOUT in the plan's status word
 * (st_sync_status); the kernel then stops issuing work, waits with a fixed
 * limit of 2^31 clocks for the asynchronous copies and MMAs it already
 * issued, frees its tensor memory and returns, so the context stays usable.
 * Outputs of such a call are undefined.  Takes effect for calls enqueued
 * afterwards.  ST_ERR_ARG for a NULL plan or a negative limit. */
int st_plan_set_wait_limit(st_plan* p, long long clocks);

/* Test hook of the failure detection (no passage of the paper): make the
 * n-th device allocation made by the library from now on fail as if the
 * device were out of memory (n >= 1), or disarm the hook (n = 0).  The
 * failing call (e.g. st_plan_create) returns ST_ERR_NOMEM and frees what it
 * had allocated.  Process-wide; not for production use.  ST_ERR_ARG if
 * n < 0. */
int st_debug_fail_alloc(int n);

/* Test hook of the failure detection (no passage of the paper): overwrite
 * one entry of the plan's device work lists with an out-of-range value that
 * the kernels' own checks catch (what = 1: the first inverse Legendre tile
 * gets a wavenumber above T; what = 2: the first ring-FFT work item gets a
 * ring pair past the grid), or put back the entry overwritten before
 * (what = 0).  The kernel that meets the bad entry skips it and sets
 * ST_ERR_CHECK; outputs of such a call are undefined.  Synchronises the
 * device.  Not for production use.  ST_ERR_ARG for a NULL plan or another
 * value of what. */
int st_debug_corrupt_worklist(st_plan* p, int what);

/* Test hook (no passage of the paper): fill the plan's workspaces that every
 * call rewrites (the Fourier buffer / direct operand, the inverse operand /
 * direct result, and the split planes) with all-ones bytes, a NaN in every
 * precision, on `stream`.  A transform called afterwards must give the same
 * bits as before: no kernel may read a workspace entry that the same call
 * has not written (padding rows and columns included).  Not for production
 * use.  ST_ERR_ARG for a NULL plan. */
int st_debug_poison_workspaces(st_plan* p, void* stream);

/* Self-test hook (no passage of the paper): out[i] = the library's
 * integer-only double -> float conversion of in[i] (round to nearest even,
 * subnormals, overflow to infinity, NaN), back[i] = its float -> double
 * conversion of out[i]; device arrays of n elements.  The kernels convert
 * their grid I/O with these instead of the FP64 pipe, and a test compares
 * them with the hardware conversion.  ST_ERR_ARG for NULL arrays or n < 0. */
int st_debug_convert(const double* in, float* out, double* back, long n, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none).  The string
 * belongs to the library and stays valid until the thread's next failing
 * call. */
const char* st_last_error(void);

/* Number of kernel launches that the last transform call on this plan
 * enqueued (for launch accounting; no operation of the paper).  0 for NULL. */
int st_plan_last_launches(const st_plan* p);

/* Defines no operation of the paper (the tile autotuner of this library).
 * Legendre tile widths (output columns per CTA tile) of the inverse and direct
 * launches: the defaults, or the autotuner's choice for a plan created with
 * ST_FLAG_AUTOTUNE.  The autotuner times each candidate width (FP64: 64, 32;
 * FP32 and the split paths: 128, 64) on the plan's own workspaces and keeps
 * the fastest.  With opts.tune_cache it first looks for a line
 * "legendre T=.. N=.. kind=.. nfld=.. prec=.. inv=.. dir=.." in that file and
 * appends one after timing.  Either pointer may be NULL. */
int st_plan_tuning(const st_plan* p, int* bn_inv, int* bn_dir);

/* Tracing (no passage of the paper; its per-stage timelines, Sec. 3.1.3.2
 * Fig. 3, came from a profiler).
 * For a plan created with ST_FLAG_STAGE_TIMING: synchronise the device, then
 * add to ms[s] (s < nstages <= ST_NSTAGES) the summed device time of every
 * kernel of stage s since the previous call, and to launches[s] their count
 * (launches may be NULL).  The times come from CUDA events recorded on the
 * launching stream.  ST_ERR_ARG if the plan was created without the flag.
 * ST_ERR_UNSUPPORTED if more launches were timed than the plan's event pool
 * holds (4096); the excess launches were not timed. */
int st_plan_stage_times(st_plan* p, double* ms, long* launches, int nstages);

/* Inverse transform that allocates nothing (the paper has no counterpart).
 * It is for callers that cannot call cudaMalloc while they transform, for
 * example code running under an allocator hook or a frozen memory pool.  It
 * computes exactly what st_inv_transform computes, with the same kernels.
 * The scratch those kernels need between them (spectral operand and Fourier
 * buffer) comes from one static device array of 32 MiB.  Every GPU that
 * calls it holds that array until the process exits.  Arguments and layouts
 * are those of st_inv_transform.  FP64 and FP32 plans only.  A plan whose
 * scratch exceeds the array is rejected with ST_ERR_ARG and a message giving
 * the size; for FP64 this happens at about T=255 with 10 fields.
 * The first call on a device looks up the array's device address (set-up,
 * once per device); make that call before any stream capture.  Under CUDA's
 * lazy module loading that first call is also when the 32 MiB are claimed.
 * The cached address does not survive a cudaDeviceReset: do not call this
 * after resetting the device.  All calls share the array: calls that overlap
 * on the GPU (two streams, or two plans at once) race on it, so the caller
 * must serialise them.  Each call writes every scratch element before
 * reading it, so nothing left by an earlier call is used. */
int st_inv_transform_noalloc(const st_plan* p, const double* spec, double* grid, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ST_H */
