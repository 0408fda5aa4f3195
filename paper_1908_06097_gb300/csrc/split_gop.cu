// Split of the direct Legendre operand into bf16 planes (split paths).
//
// The r2c fold (fft_kernels.cuh) writes the folded, weighted Fourier rows of
// the direct operand G[(m, p) block][ring][column] in FP32.  Here every value
// x of the written columns becomes p0 = bf16(x), p1 = bf16(x - p0) and, for
// BF16X6, p2 = bf16(x - p0 - p1), all round-to-nearest, in the three plane
// arrays that the tensor-core Legendre kernel reads through its tensor maps
// (plane 0 in the Fourier buffer, planes 1 and 2 in their own arrays; same
// row and column layout as the FP32 operand).  The values are those the fold
// would have stored itself; done here, the fold's scattered stores are one
// per row instead of one per plane, and the split is a coalesced stream.
#include <algorithm>

#include "st_internal.cuh"

namespace st {

namespace {

constexpr int SPLIT_NT = 256;

__device__ __forceinline__ void split2(float x0, float x1, __nv_bfloat162& a, __nv_bfloat162& b, __nv_bfloat162& c)
{
    a.x = __float2bfloat16_rn(x0);
    a.y = __float2bfloat16_rn(x1);
    const float r0 = x0 - __bfloat162float(a.x), r1 = x1 - __bfloat162float(a.y);
    b.x = __float2bfloat16_rn(r0);
    b.y = __float2bfloat16_rn(r1);
    c.x = __float2bfloat16_rn(r0 - __bfloat162float(b.x));
    c.y = __float2bfloat16_rn(r1 - __bfloat162float(b.y));
}

// One thread per 8 consecutive columns of a row (rows are multiples of 8
// columns): two 16-byte loads, one 16-byte store per plane.  Each thread
// issues UNR such loads (a grid stride apart) before their stores, so that
// enough bytes are in flight to cover the DRAM latency.  blockIdx.y is the
// member (0 for a plan call).
constexpr int UNR = 4;

__global__ void __launch_bounds__(SPLIT_NT) k_split_gop(const __grid_constant__ FftDesc d0,
                                                       const FftDesc* __restrict__ desc, int ncols)
{
    const FftDesc& d = desc ? desc[blockIdx.y] : d0;
    const int ncolp = d.ncolp;
    int nc = ncols > 0 ? ncols : 2 * d.nfld;
    nc = min((nc + 7) & ~7, ncolp);
    const unsigned q = (unsigned)(nc >> 3);  // column octets per row
    const unsigned n = (unsigned)d.ngop_rows * q;
    const float* src = d.g32;
    __nv_bfloat16* p0 = (__nv_bfloat16*)d.four;
    __nv_bfloat16* p1 = d.lo;
    __nv_bfloat16* p2 = d.lo2;
    const bool three = d.split == 3;
    const unsigned stride = gridDim.x * SPLIT_NT;
    for (unsigned i0 = blockIdx.x * SPLIT_NT + threadIdx.x; i0 < n; i0 += UNR * stride) {
        long e[UNR];
        float4 x[UNR][2];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const unsigned i = i0 + u * stride;  // < n + UNR * stride < 2^32 (n < 2^31)
            const unsigned r = i / q, c = (i - r * q) * 8;
            e[u] = (long)r * ncolp + c;
            if (i < n) {
                x[u][0] = *(const float4*)(src + e[u]);
                x[u][1] = *(const float4*)(src + e[u] + 4);
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (i0 + u * stride >= n) break;
            __nv_bfloat162 a[4], b[4], cc[4];
            split2(x[u][0].x, x[u][0].y, a[0], b[0], cc[0]);
            split2(x[u][0].z, x[u][0].w, a[1], b[1], cc[1]);
            split2(x[u][1].x, x[u][1].y, a[2], b[2], cc[2]);
            split2(x[u][1].z, x[u][1].w, a[3], b[3], cc[3]);
            *(uint4*)(p0 + e[u]) = *(const uint4*)a;
            *(uint4*)(p1 + e[u]) = *(const uint4*)b;
            if (three) *(uint4*)(p2 + e[u]) = *(const uint4*)cc;
        }
    }
}

}  // namespace

int launch_split_gop(const FftDesc& d0, const FftDesc* desc, int nmemb, int ncols, cudaStream_t s)
{
    if (nmemb <= 0) return ST_OK;
    if (!desc) {
        // the quad count of the last row must fit the kernel's 32-bit index
        const long q = (std::min((long)((ncols + 7) & ~7), (long)d0.ncolp)) / 8;
        if (!d0.g32 || d0.ngop_rows * q >= (1L << 31)) {
            set_error("launch_split_gop: operand of %ld rows x %ld column octets not supported", d0.ngop_rows, q);
            return ST_ERR_UNSUPPORTED;
        }
    }
    int dev = 0, nsm = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    ST_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // 8 resident CTAs of 256 threads per SM, grid-stride over each member
    k_split_gop<<<dim3(nsm * 8, nmemb), SPLIT_NT, 0, s>>>(d0, desc, ncols);
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
