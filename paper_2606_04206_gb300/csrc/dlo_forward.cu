// dlo_forward.cu -- dispatch of the persistent forward kernel to its size classes (the kernel
// is in dlo_fwd_kernel.cuh, instantiated per size class in dlo_nv*.cu).
#include "dlo_kernels.h"

namespace dlo {

cudaError_t launch_forward(const FwdParams& P, int nv_max, bool contact, int grid, int warps, cudaStream_t st) {
    switch (nv_max) {
        case 32: return launch_forward_nv32(P, contact, grid, warps, st);
        case 64: return launch_forward_nv64(P, contact, grid, warps, st);
        case 128: return launch_forward_nv128(P, contact, grid, warps, st);
        case 192: return launch_forward_nv192(P, contact, grid, warps, st);
        case 224: return launch_forward_nv224(P, contact, grid, warps, st);
        case 256: return launch_forward_nv256(P, contact, grid, warps, st);
    }
    return cudaErrorInvalidValue;
}

int forward_blocks_per_sm(int nv_max, bool contact, int warps) {
    switch (nv_max) {
        case 32: return forward_occ_nv32(contact, warps);
        case 64: return forward_occ_nv64(contact, warps);
        case 128: return forward_occ_nv128(contact, warps);
        case 192: return forward_occ_nv192(contact, warps);
        case 224: return forward_occ_nv224(contact, warps);
        case 256: return forward_occ_nv256(contact, warps);
    }
    return 0;
}

}  // namespace dlo
