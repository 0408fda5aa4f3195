// C2R ring-FFT kernel, FP64 (see fft_kernels.cuh).
#include "fft_kernels.cuh"

namespace st {

int launch_c2r_f64(const FftIO& io, int nctas, cudaStream_t s)
{
    static bool ready = false;
    if (!ready) {
        ST_CUDA_TRY(cudaFuncSetAttribute(fft::k_c2r<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         fft::smem_bytes<double>()));
        ready = true;
    }
    fft::k_c2r<double><<<dim3(nctas, io.narr), fft::KC<double>::NT, fft::smem_bytes<double>(), s>>>(io);
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
