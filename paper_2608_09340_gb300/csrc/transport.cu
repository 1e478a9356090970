// The packet walk for line-profile mode 2 (the Voigt slice; production) and
// the batched multi-model launch. The walk itself is in transport_impl.cuh;
// transport_modes.cu instantiates it for modes 1 and 3.
#include "transport_impl.cuh"

namespace krl {

cudaError_t launch_transport(const TransportArgs& A, int precision, unsigned features, int grid, int block,
                             cudaStream_t s)
{
    if (A.ph_mode == 1 || A.ph_mode == 3 || A.ph_mode == 4)
        return launch_transport_ph(A, A.ph_mode, precision, features, grid, block, s);
    return precision == KRL_PREC_FP64 ? dispatch<double, 2>(A, features, grid, block, s)
                                      : dispatch<float, 2>(A, features, grid, block, s);
}

cudaError_t launch_transport_batch(const BatchArgs& B, int precision, unsigned features, int grid, int block,
                                   cudaStream_t s)
{
    return precision == KRL_PREC_FP64 ? dispatch_batch<double>(B, features, grid, block, s)
                                      : dispatch_batch<float>(B, features, grid, block, s);
}

cudaError_t launch_emiss_deposit(const TransportArgs& A, unsigned features, int sm_count, cudaStream_t s)
{
    const bool vel = (features & F_VEL) != 0;
    auto kern = vel ? k_emiss_deposit<true> : k_emiss_deposit<false>;
    int occ = 0;                     // resident CTAs per SM on the current device
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDepositBlock, 0);
    if (e != cudaSuccess) return e;
    kern<<<sm_count * (occ > 0 ? occ : 1), kDepositBlock, 0, s>>>(A);
    return cudaGetLastError();
}

int transport_batch_max_block() { return kBatchBlock; }

int transport_batch_occupancy(int precision, unsigned features, int block)
{
    return precision == KRL_PREC_FP64 ? batch_occ_dispatch<double>(features, block)
                                      : batch_occ_dispatch<float>(features, block);
}

int transport_max_block(int precision, unsigned features)
{
    return (precision == KRL_PREC_FP32 && !(features & F_RICH)) ? 512 : 256;
}

int transport_occupancy(int precision, unsigned features, int block, int ph_mode)
{
    if (ph_mode == 1 || ph_mode == 3 || ph_mode == 4) return transport_occupancy_ph(ph_mode, precision, features, block);
    return precision == KRL_PREC_FP64 ? occ_dispatch<double, 2>(features, block)
                                      : occ_dispatch<float, 2>(features, block);
}

}  // namespace krl
