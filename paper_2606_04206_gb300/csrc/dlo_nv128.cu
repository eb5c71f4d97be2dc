// dlo_nv128.cu -- the forward and backward kernels for rods of at most 128 vertices.
#include "dlo_bwd_kernel.cuh"
#include "dlo_fwd_kernel.cuh"

namespace dlo {

cudaError_t launch_forward_nv128(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_fwd_t<128, true>(P, grid, warps, st) : launch_fwd_t<128, false>(P, grid, warps, st);
}
int forward_occ_nv128(bool c, int warps) { return c ? fwd_occ_t<128, true>(warps) : fwd_occ_t<128, false>(warps); }
cudaError_t launch_backward_nv128(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_bwd_t<128, true>(P, grid, warps, st) : launch_bwd_t<128, false>(P, grid, warps, st);
}
int backward_occ_nv128(bool c, int warps) { return c ? bwd_occ_t<128, true>(warps) : bwd_occ_t<128, false>(warps); }

}  // namespace dlo
