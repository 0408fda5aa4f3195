// Tensor-core (tcgen05) Legendre step of the BF16x3 path.
#include "st_internal.cuh"

namespace st {

int launch_leg_inv_tc(Plan*, int, int, cudaStream_t)
{
    set_error("BF16X3 Legendre kernel not built yet");
    return ST_ERR_UNSUPPORTED;
}

int launch_leg_dir_tc(Plan*, int, int, cudaStream_t)
{
    set_error("BF16X3 Legendre kernel not built yet");
    return ST_ERR_UNSUPPORTED;
}

}  // namespace st
