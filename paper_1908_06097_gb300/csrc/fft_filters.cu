// Bluestein filter tables of the ring FFTs (see fft_kernels.cuh).
#include <string.h>

#include "fft_kernels.cuh"

namespace st {

int launch_fft_filters(Tables* t)
{
    if (t->Mmax > 8192) {
        set_error("ring FFT length %d exceeds the on-chip limit of 8192 (T too large)", t->Mmax);
        return ST_ERR_UNSUPPORTED;
    }
    // both tables are computed in FP64 from the same chirps; the double
    // precision slot size bounds both launches
    const int smem = fft::filt_smem_bytes();
    ST_CUDA_TRY(cudaFuncSetAttribute(fft::k_fft_filters<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ST_CUDA_TRY(cudaFuncSetAttribute(fft::k_fft_filters<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    Plan tmp;
    memset((void*)&tmp, 0, sizeof tmp);
    tmp.tab = t;
    tmp.opts.prec = ST_PREC_FP64;
    FftDesc d = fft_desc(&tmp);
    fft::k_fft_filters<double><<<t->N, fft::KC<double>::FILT_NT, smem>>>(d, t->filt64, nullptr);
    fft::k_fft_filters<float><<<t->N, fft::KC<float>::FILT_NT, smem>>>(d, nullptr, t->filt32);
    ST_CUDA_TRY(cudaGetLastError());
    ST_CUDA_TRY(cudaDeviceSynchronize());
    return ST_OK;
}

}  // namespace st
