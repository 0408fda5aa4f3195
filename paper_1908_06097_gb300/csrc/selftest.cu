// Self-test of the library's integer-only float/double conversions
// (dbl2flt_rn, to_dbl in st_internal.cuh), which the ring FFTs and the
// spectral kernels use instead of the hardware conversion on the narrow FP64
// pipe: a test compares them bit for bit with the hardware conversion.
#include "st_internal.cuh"

namespace {

__global__ void k_convert(const double* __restrict__ in, long n, float* __restrict__ out, double* __restrict__ back)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float f = st::dbl2flt_rn(in[i]);
        out[i] = f;
        back[i] = st::to_dbl(f);
    }
}

}  // namespace

extern "C" int st_debug_convert(const double* in, float* out, double* back, long n, void* stream)
{
    if (!in || !out || !back || n < 0) {
        st::set_error("st_debug_convert: bad argument");
        return ST_ERR_ARG;
    }
    if (n == 0) return ST_OK;
    const long nb = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_convert<<<(int)nb, 256, 0, (cudaStream_t)stream>>>(in, n, out, back);
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}
