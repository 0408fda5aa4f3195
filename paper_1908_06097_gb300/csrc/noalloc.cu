// Inverse transform whose scratch lives in a fixed device array.
//
// Some callers cannot call cudaMalloc while they transform: code that runs
// while a memory pool is frozen, inside an allocator hook, or under a
// framework that owns every device allocation.  This entry point lets them
// run the inverse transform of an existing plan without allocating anything.
// The two scratch buffers that an inverse transform needs between its kernels
// (the spectral operand and the ring-major Fourier buffer) are carved out of
// the file-scope array below instead of the plan's own workspace.  The caller
// still passes the input spectra and the output grid.
//
// Limits and rules:
//   - the scratch is ST_NOALLOC_SCRATCH_BYTES (32 MiB); every GPU that loads
//     this library keeps that much device memory until the process exits;
//   - FP64 and FP32 plans only (the tensor-core path reads its operands
//     through tensor maps bound to the plan's workspace);
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (set-up, once per device); make that first call
//     before any stream capture.  With CUDA's lazy module loading, that
//     lookup is also what loads this file's device module, so the 32 MiB are
//     claimed at the first call rather than when the library is loaded.  The
//     address is cached per device; a cudaDeviceReset invalidates it, so a
//     process that resets a device must not call this entry point afterwards;
//   - every call shares the array: calls that overlap on the GPU (on two
//     streams, or two plans at once) race on it.  Each call writes every
//     scratch element it reads before reading it, so nothing needs clearing
//     and the contents left by an earlier call are never used.
#include <string.h>

#include <atomic>

#include "st_internal.cuh"

namespace st {

#define ST_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[ST_NOALLOC_SCRATCH_BYTES];

// device address of the array, per device; several host threads may fill a
// slot at once, and they all store the same value
static std::atomic<void*> g_scratch_dev[64];

static int noalloc_scratch(void** out)
{
    int dev = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("st_inv_transform_noalloc: device %d out of range", dev);
        return ST_ERR_UNSUPPORTED;
    }
    void* ptr = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!ptr) {
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("st_inv_transform_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return ST_ERR_CUDA;
        }
        g_scratch_dev[dev].store(ptr, std::memory_order_release);
    }
    *out = ptr;
    return ST_OK;
}

}  // namespace st

using namespace st;

extern "C" int st_inv_transform_noalloc(const st_plan* pp, const double* spec, double* grid, void* stream)
{
    if (!pp || !spec || !grid) {
        set_error("st_inv_transform_noalloc: NULL argument");
        return ST_ERR_ARG;
    }
    const Plan* p = (const Plan*)pp;
    if (is_split(p->opts.prec)) {
        set_error("st_inv_transform_noalloc: FP64 and FP32 plans only");
        return ST_ERR_UNSUPPORTED;
    }
    const Tables* t = p->tab;
    const size_t eb = p->opts.prec == ST_PREC_FP64 ? 8 : 4;
    const size_t op_bytes = round_up((long)((size_t)t->nops_rows * p->ncolp * eb), 256);
    const size_t four_bytes = (size_t)t->nfour_rows * p->ncolp * eb;
    if (op_bytes + four_bytes > ST_NOALLOC_SCRATCH_BYTES) {
        set_error("st_inv_transform_noalloc: plan needs %zu bytes of scratch, more than the %u-byte static "
                  "array (reduce T or nfld)",
                  op_bytes + four_bytes, (unsigned)ST_NOALLOC_SCRATCH_BYTES);
        return ST_ERR_ARG;
    }
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // a shallow copy of the plan that points at the static scratch; tables,
    // work lists and the status word stay the plan's own (read-only here)
    Plan q;
    memcpy((void*)&q, (const void*)p, sizeof(Plan));
    q.ws_op = scratch;
    q.ws_four = (unsigned char*)scratch + op_bytes;
    q.ws_op_lo = nullptr;
    q.ev = nullptr;
    q.last_launches = 0;
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_pre(&q, PRE_PLAIN, spec, nullptr, q.nfld, s);
    if (!rc) rc = launch_leg_inv(&q, q.nfld, s);
    if (!rc) rc = launch_polar(&q, PRE_PLAIN, spec, nullptr, s);  // as st_inv_transform (FP64 plans)
    if (!rc) {
        SynthOut o;
        memset(&o, 0, sizeof o);
        o.ptr[0] = grid;
        o.narr = 1;
        o.nf = q.nfld;
        rc = launch_c2r(&q, o, 0, s);
    }
    return rc;
}
