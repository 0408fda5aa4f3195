// R2C ring-FFT kernel, FP32 (see fft_kernels.cuh).
#include "fft_kernels.cuh"

namespace st {

int launch_r2c_f32(const FftIO& io, int nctas, cudaStream_t s)
{
    static bool ready = false;
    if (!ready) {
        ST_CUDA_TRY(cudaFuncSetAttribute(fft::k_r2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         fft::smem_bytes<float>()));
        ready = true;
    }
    fft::k_r2c<float><<<dim3(nctas, io.narr), fft::KC<float>::NT, fft::smem_bytes<float>(), s>>>(io);
    ST_CUDA_TRY(cudaGetLastError());
    return ST_OK;
}

}  // namespace st
