// dlo_fwd_kernel.cuh -- the persistent forward kernel: one warp per rod, rod state in shared
// memory across all substeps and frames of a launch (the substep itself is in dlo_step.cuh).
#pragma once
#include "dlo_step.cuh"

namespace dlo {

// ------------------------------------------------------------------ the persistent kernel
__device__ __forceinline__ void write_state(const StateRef& D, long long offV, long long offE, long long offB,
                                            const RodInfo& R, int rod, int lane, const float4* X, const float4* V,
                                            const float4* ED, const float4* ET, const float4* HG, const float* gp) {
    for (int i = lane; i < R.nv; i += 32) {
        D.X[offV + R.v0 + i] = X[i];
        D.Vl[offV + R.v0 + i] = V[i];
        D.HG[offV + R.v0 + i] = HG[i];
    }
    for (int j = lane; j < R.ne; j += 32) {
        D.ED[offE + R.e0 + j] = ED[j];
        D.ET[offE + R.e0 + j] = ET[j];
    }
    if (lane < 24) D.GP[offB + 24LL * rod + lane] = gp[lane];
}

template <int NV, bool CONTACT>
__global__ void __launch_bounds__(256) fwd_kernel(FwdParams P) {
    extern __shared__ float4 dyn_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Smem<NV, CONTACT> s(dyn_smem + warp * (warp_smem_bytes(NV, CONTACT) / 16));
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= P.n_order) break;
        const int rod = P.order[item];
        const RodInfo R = P.rods[rod];
        const int nsub = P.force_nsub > 0 ? P.force_nsub : R.nsub;
        const float h = P.scene.dt / (float)nsub;
        for (int i = lane; i < R.nv; i += 32) {
            float4 x = P.S.X[R.v0 + i];
            s.X[i] = x;
            s.X0[i] = x;
            s.V[i] = P.S.Vl[R.v0 + i];
            s.HG[i] = P.S.HG[R.v0 + i];
        }
        for (int j = lane; j < R.ne; j += 32) {
            s.ED[j] = P.S.ED[R.e0 + j];
            s.ET[j] = P.S.ET[R.e0 + j];
        }
        // gripper poses of the frame start (every lane holds a copy)
        Pose F;
        F.load(P.S.GP + 24LL * rod);
        __syncwarp();
        unsigned bad = 0;
        for (int f = 0; f < P.frames; ++f) {
            const int gf = P.frame0 + f;
            if (P.ck_every > 0 && gf % P.ck_every == 0 && gf / P.ck_every < P.ck_count) {
                const long long c = gf / P.ck_every;
                write_state(P.ck, c * P.ck_strideV, c * P.ck_strideE, c * P.ck_strideB, R, rod, lane, s.X, s.V,
                            s.ED, s.ET, s.HG, F.p);
            }
            float act[12];
#pragma unroll
            for (int k = 0; k < 12; ++k)
                act[k] = P.actions ? P.actions[((long long)f * P.B + rod) * 12 + k] : 0.f;
            bool ovf = false;
            const int np = run_frame<NV, CONTACT>(P.scene, P.KIN, P.ES, R, s, lane, nsub, h, F, act, ovf,
                                                  [](int) {});
            if (ovf) bad |= 2u;
            bool nf = false;
            for (int i = lane; i < R.nv; i += 32) {
                float4 x = s.X[i], v = s.V[i];
                nf |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) && isfinite(v.y) &&
                        isfinite(v.z) && isfinite(v.w));
                if (P.xframes) reinterpret_cast<float4*>(P.xframes)[(long long)f * P.nvert_total + R.v0 + i] = x;
            }
            if (__any_sync(kFull, nf)) bad |= 1u;
            if (f + 1 == P.frames) {
                if (R.flags & ROD_INEXT) {
                    double r = 0.0;
                    for (int j = lane; j < R.ne; j += 32) {
                        int j1 = (j + 1 == R.nv) ? 0 : j + 1;
                        V3<float> e = f3(s.X[j1]) - f3(s.X[j]);
                        r += fabs((double)sqrtf(dot(e, e)) - (double)s.ET[j].w);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
                    if (lane == 0) P.residual[rod] = r;
                }
                if (lane == 0) P.npairs[rod] = np;
            }
        }
        write_state(P.S, 0, 0, 0, R, rod, lane, s.X, s.V, s.ED, s.ET, s.HG, F.p);
        if (lane == 0 && bad) atomicOr(&P.status[rod], bad);
        __syncwarp();
    }
}

template <int NV, bool C>
static cudaError_t launch_fwd_t(const FwdParams& P, int grid, int warps, cudaStream_t st) {
    size_t smem = warp_smem_bytes(NV, C) * warps;
    auto k = fwd_kernel<NV, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * warps, smem, st>>>(P);
    return cudaGetLastError();
}

template <int NV, bool C>
static int fwd_occ_t(int warps) {
    size_t smem = warp_smem_bytes(NV, C) * warps;
    auto k = fwd_kernel<NV, C>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * warps, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

}  // namespace dlo
