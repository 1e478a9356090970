// The packet walk instantiated for line-profile modes 1 (two-dimensional
// Voigt table and sampler in global memory) and 3 (core-wing blend),
// Sec. 2.3.1, and for mode 2 with its tables in constant memory (internal
// mode 4, krl_tune.table_space: the placement the paper recommends, kept to
// measure it against the shared-memory walk). A translation unit of its own
// so that it compiles in parallel with the production walk.
#define KRL_TABLES_IN_CONSTANT 1
#include "transport_impl.cuh"

namespace krl {

cudaError_t launch_transport_ph(const TransportArgs& A, int ph_mode, int precision, unsigned features, int grid,
                                int block, cudaStream_t s)
{
    const bool d = precision == KRL_PREC_FP64;
    if (ph_mode == 1) return d ? dispatch<double, 1>(A, features, grid, block, s) : dispatch<float, 1>(A, features, grid, block, s);
    if (ph_mode == 3) return d ? dispatch<double, 3>(A, features, grid, block, s) : dispatch<float, 3>(A, features, grid, block, s);
    if (ph_mode == 4 && !d) {
        // this line's slice and sampler into the constant bank, in stream
        // order before the launch (one line at a time per device: runs with
        // this placement must not overlap)
        cudaError_t e = cudaMemcpyToSymbolAsync(c_voigt, A.voigt_lnH, sizeof(float) * kVoigtN, 0,
                                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyToSymbolAsync(c_usx, A.us_x, sizeof(float) * kUsNx, 0, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyToSymbolAsync(c_uslncdf, A.us_lncdf, sizeof(float) * kUsNx * kUsNu, 0,
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        return dispatch<float, 4>(A, features, grid, block, s);
    }
    return cudaErrorInvalidValue;
}

int transport_occupancy_ph(int ph_mode, int precision, unsigned features, int block)
{
    const bool d = precision == KRL_PREC_FP64;
    if (ph_mode == 1) return d ? occ_dispatch<double, 1>(features, block) : occ_dispatch<float, 1>(features, block);
    if (ph_mode == 3) return d ? occ_dispatch<double, 3>(features, block) : occ_dispatch<float, 3>(features, block);
    if (ph_mode == 4 && !d) return occ_dispatch<float, 4>(features, block);
    return 0;
}

}  // namespace krl
