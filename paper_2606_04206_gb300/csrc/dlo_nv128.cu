// dlo_nv128.cu -- the forward and backward kernels for rods of at most 128 vertices.
#include "dlo_bwd_kernel.cuh"
#include "dlo_fwd_kernel.cuh"

namespace dlo {

cudaError_t launch_forward_nv128(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_fwd_t<128, true>(P, grid, warps, st) : launch_fwd_t<128, false>(P, grid, warps, st);
}
int forward_occ_nv128(bool c, int warps) { return c ? fwd_occ_t<128, true>(warps) : fwd_occ_t<128, false>(warps); }
cudaError_t launch_rec_nv128(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_rec_t<128, true>(P, grid, warps, st) : launch_rec_t<128, false>(P, grid, warps, st);
}
int rec_occ_nv128(bool c, int warps) { return c ? rec_occ_t<128, true>(warps) : rec_occ_t<128, false>(warps); }
cudaError_t launch_rev_nv128(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_rev_t<128, true>(P, grid, warps, st) : launch_rev_t<128, false>(P, grid, warps, st);
}
int rev_occ_nv128(bool c, int warps) { return c ? rev_occ_t<128, true>(warps) : rev_occ_t<128, false>(warps); }

}  // namespace dlo
