// dlo_reaction.cu -- the rigid-contact impulses that dlo_step accumulated per vertex (four
// slots: planes, boxes, gripper 0, gripper 1), summed per rod in a fixed order.
#include "dlo_runtime.h"

namespace dlo {
namespace {

constexpr int kRT = 128;

__global__ void reaction_reduce(const RodInfo* rods, const float4* slots, float4* per_rod) {
    __shared__ float4 sh[kRT][4];
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    float4 acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < R.nv; i += kRT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 a = slots[4LL * (R.v0 + i) + k];
            acc[k] = make_float4(acc[k].x + a.x, acc[k].y + a.y, acc[k].z + a.z, 0.f);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = kRT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 a = sh[threadIdx.x][k], b = sh[threadIdx.x + s][k];
                sh[threadIdx.x][k] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) per_rod[4LL * rod + threadIdx.x] = sh[0][threadIdx.x];
}

}  // namespace
}  // namespace dlo

using namespace dlo;

extern "C" dlo_status dlo_reaction(dlo_ctx* c, float* per_rod, float* per_vertex, int reset) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!c->d_reaction) return set_err(c, DLO_ERR_STATE, "the context was created without opt.reaction");
    if (((uintptr_t)per_rod & 15u) || ((uintptr_t)per_vertex & 15u))
        return set_err(c, DLO_ERR_INVALID_ARG, "per_rod and per_vertex must be 16-byte aligned");
    cudaError_t e = cudaSuccess;
    if (per_rod) {
        reaction_reduce<<<c->B, kRT, 0, c->stream>>>(c->d_rods, c->d_reaction, reinterpret_cast<float4*>(per_rod));
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && per_vertex)
        e = cudaMemcpyAsync(per_vertex, c->d_reaction, 64 * (size_t)c->V, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->d_reaction, 0, 64 * (size_t)c->V, c->stream);
    return cuda_err(c, e, "dlo_reaction");
}
