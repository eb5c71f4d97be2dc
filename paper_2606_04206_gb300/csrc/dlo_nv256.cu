// dlo_nv256.cu -- the forward and backward kernels for rods of at most 256 vertices.
#include "dlo_bwd_kernel.cuh"
#include "dlo_fwd_kernel.cuh"

namespace dlo {

cudaError_t launch_forward_nv256(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_fwd_t<256, true>(P, grid, warps, st) : launch_fwd_t<256, false>(P, grid, warps, st);
}
int forward_occ_nv256(bool c, int warps) { return c ? fwd_occ_t<256, true>(warps) : fwd_occ_t<256, false>(warps); }
cudaError_t launch_rec_nv256(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_rec_t<256, true>(P, grid, warps, st) : launch_rec_t<256, false>(P, grid, warps, st);
}
int rec_occ_nv256(bool c, int warps) { return c ? rec_occ_t<256, true>(warps) : rec_occ_t<256, false>(warps); }
cudaError_t launch_rev_nv256(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st) {
    return c ? launch_rev_t<256, true>(P, grid, warps, st) : launch_rev_t<256, false>(P, grid, warps, st);
}
int rev_occ_nv256(bool c, int warps) { return c ? rev_occ_t<256, true>(warps) : rev_occ_t<256, false>(warps); }

}  // namespace dlo
