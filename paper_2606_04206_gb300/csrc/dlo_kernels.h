// dlo_kernels.h -- launch entry points of the device kernels (host side of each .cu file).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "dlo_internal.h"

namespace dlo {

// Shared memory of one rod group (one rod of at most NV vertices) in the persistent kernels:
// ten float4 arrays of NV (positions, start positions, velocities, base frames + twist,
// base tangents + rest lengths, hinge state, three per-hinge gradient slots, new reference
// frames) and, with self-contact, 4 NV pair slots (two float4 of projection data each,
// one packed index pair) plus an int4 fixed-point accumulator per vertex.
constexpr int kPairsPerVertex = 4;
__host__ __device__ constexpr size_t warp_smem_bytes(int NV, bool contact) {
    return (size_t)(10 * NV) * 16 +
           (contact ? ((size_t)(2 * kPairsPerVertex * NV) * 16 + (size_t)NV * 16 + (size_t)(kPairsPerVertex * NV) * 4)
                    : 0);
}

// Per size class (dlo_nv*.cu).
cudaError_t launch_forward_nv32(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv32(bool c, int warps);
cudaError_t launch_rec_nv32(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv32(bool c, int warps);
cudaError_t launch_rev_nv32(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv32(bool c, int warps);
cudaError_t launch_forward_nv64(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv64(bool c, int warps);
cudaError_t launch_rec_nv64(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv64(bool c, int warps);
cudaError_t launch_rev_nv64(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv64(bool c, int warps);
cudaError_t launch_forward_nv128(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv128(bool c, int warps);
cudaError_t launch_rec_nv128(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv128(bool c, int warps);
cudaError_t launch_rev_nv128(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv128(bool c, int warps);
cudaError_t launch_forward_nv192(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv192(bool c, int warps);
cudaError_t launch_rec_nv192(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv192(bool c, int warps);
cudaError_t launch_rev_nv192(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv192(bool c, int warps);
cudaError_t launch_forward_nv224(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv224(bool c, int warps);
cudaError_t launch_rec_nv224(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv224(bool c, int warps);
cudaError_t launch_rev_nv224(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv224(bool c, int warps);
cudaError_t launch_forward_nv256(const FwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int forward_occ_nv256(bool c, int warps);
cudaError_t launch_rec_nv256(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rec_occ_nv256(bool c, int warps);
cudaError_t launch_rev_nv256(const BwdParams& P, bool c, int grid, int warps, cudaStream_t st);
int rev_occ_nv256(bool c, int warps);
// the backward's recompute and reverse kernels (dlo_adjoint.cu dispatches to the size classes)
cudaError_t launch_rec(const BwdParams& P, int nv_max, bool contact, int grid, int warps, cudaStream_t st);
int rec_blocks_per_sm(int nv_max, bool contact, int warps);
cudaError_t launch_rev(const BwdParams& P, int nv_max, bool contact, int grid, int warps, cudaStream_t st);
int rev_blocks_per_sm(int nv_max, bool contact, int warps);
// Shared memory of one rod: its arrays plus a 256-byte header for group reductions.
// per rod: the arrays above, 256 B of group-reduction scratch and the 512 B gripper block
__host__ __device__ constexpr size_t rod_smem_bytes(int NV, bool contact) { return warp_smem_bytes(NV, contact) + 768; }

// Rod size classes: a rod of nv vertices runs in the kernels instantiated for the smallest
// class that holds it (shared memory is sized per class; 192 and 224 let two rods of up to
// 224 vertices share an SM in the backward, where a 256-vertex rod needs 124 KB).
constexpr int kNumSizeClasses = 6;
__host__ __device__ constexpr int size_class_at(int k) {
    return k == 0 ? 32 : k == 1 ? 64 : k == 2 ? 128 : k == 3 ? 192 : k == 4 ? 224 : 256;
}
__host__ __device__ constexpr int size_class(int nv) {
    return nv <= 32 ? 32 : nv <= 64 ? 64 : nv <= 128 ? 128 : nv <= 192 ? 192 : nv <= 224 ? 224 : 256;
}

// Threads that step one rod of size class NV (one vertex per thread up to 128 vertices).
__host__ __device__ constexpr int threads_per_rod(int NV) { return NV < 128 ? NV : 128; }

cudaError_t launch_forward(const FwdParams& P, int nv_max, bool contact, int grid, int warps, cudaStream_t st);
int forward_blocks_per_sm(int nv_max, bool contact, int warps);

struct InitParams {
    const RodInfo* rods;
    int B;
    const float4* xin;       // [V][4] positions (w ignored)
    const float4* vin;       // [V][4] or null
    const float* thin;       // [Etot] or null
    const float2* mass;      // [V] (mass, inverse mass)
    const float2* ES;        // [Etot] (rest length, 1/inertia)
    float4* rest;            // [V] rest hinge data (kbar0 x, kbar0 y, mbar, unused)
    StateRef S;
    const float* GP0;        // [B][2][12] initial gripper poses
    int rest_mode;           // 1: compute the rest twist from xin into rest[].z only
};
cudaError_t launch_init(const InitParams& P, cudaStream_t st);

}  // namespace dlo
