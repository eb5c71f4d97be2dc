// dlo_fwd_kernel.cuh -- the persistent forward kernel: a group of TPR threads per rod, rod
// state in shared memory across all substeps and frames of a launch (the substep itself is in
// dlo_step.cuh).  Rods are taken from a work queue in decreasing cost.
#pragma once
#include "dlo_step.cuh"

namespace dlo {

constexpr int kFwdMaxThreads = 512;   // per CTA (register budget of the forward kernel)

template <int TPR>
__device__ __forceinline__ void write_state(const StateRef& D, long long offV, long long offE, long long offB,
                                            const RodInfo& R, int rod, const Grp<TPR>& g, const float4* X,
                                            const float4* V, const float4* ED, const float4* ET, const float4* HG,
                                            const float* gp) {
    for (int i = g.tid; i < R.nv; i += TPR) {
        D.X[offV + R.v0 + i] = X[i];
        D.Vl[offV + R.v0 + i] = V[i];
        D.HG[offV + R.v0 + i] = HG[i];
    }
    for (int j = g.tid; j < R.ne; j += TPR) {
        D.ED[offE + R.e0 + j] = ED[j];
        D.ET[offE + R.e0 + j] = ET[j];
    }
    if (g.tid == 0)
        for (int k = 0; k < 24; ++k) D.GP[offB + 24LL * rod + k] = gp[k];
}

template <int NV, bool CONTACT>
__global__ void __launch_bounds__(kFwdMaxThreads) fwd_kernel(FwdParams P) {
    constexpr int TPR = threads_per_rod(NV);
    extern __shared__ float4 dyn_smem[];
    const int slot = threadIdx.x / TPR;
    Smem<NV, CONTACT> s(dyn_smem + slot * (rod_smem_bytes(NV, CONTACT) / 16));
    const Grp<TPR> g{(int)(threadIdx.x % TPR), 1 + slot, s.red};
    if (CONTACT)   // the contact accumulators start at zero; every sweep leaves them at zero
        for (int i = g.tid; i < NV; i += TPR) s.acc[i] = make_int4(0, 0, 0, 0);
    for (;;) {
        const int item = grp_bcast0<TPR>(g.tid == 0 ? atomicAdd(P.counter, 1) : 0, g);
        if (item >= P.n_order) break;
        const int rod = P.order[item];
        bounds_begin<TPR>(g);
        if (!in_bounds(rod >= 0 && rod < P.B && P.rods[rod].nv <= NV &&
                           P.rods[rod].v0 + P.rods[rod].nv <= P.nvert_total, s.red)) {
            g.sync();
            bounds_end<TPR>(g, P.status, (rod >= 0 && rod < P.B) ? rod : 0);
            continue;
        }
        // with self-contact read from memory where used: a register copy spills the
        // contact variant of the kernel (its broad phase and sweeps) past the launch bound
        RodRef<CONTACT> R = P.rods[rod];
        const int nsub = P.force_nsub > 0 ? P.force_nsub : R.nsub;
        const float h = P.scene.dt / (float)nsub;
        for (int i = g.tid; i < R.nv; i += TPR) {
            float4 x = P.S.X[R.v0 + i];
            s.X[i] = x;
            s.X0[i] = x;
            s.V[i] = P.S.Vl[R.v0 + i];
            s.HG[i] = P.S.HG[R.v0 + i];
        }
        for (int j = g.tid; j < R.ne; j += TPR) {
            s.ED[j] = P.S.ED[R.e0 + j];
            s.ET[j] = P.S.ET[R.e0 + j];
        }
        // gripper poses of the frame start
        if (g.tid < 24) s.fp[g.tid] = P.S.GP[24LL * rod + g.tid];
        g.sync();
        unsigned bad = 0;
        int np_max = 0;
        for (int f = 0; f < P.frames; ++f) {
            const int gf = P.frame0 + f;
            if (P.ck_every > 0 && gf % P.ck_every == 0 && gf / P.ck_every < P.ck_count) {
                const long long c = gf / P.ck_every;
                write_state<TPR>(P.ck, c * P.ck_strideV, c * P.ck_strideE, c * P.ck_strideB, R, rod, g, s.X, s.V,
                                 s.ED, s.ET, s.HG, s.fp);
            }
            if (g.tid < 12) s.act[g.tid] = P.actions ? P.actions[((long long)f * P.B + rod) * 12 + g.tid] : 0.f;
            g.sync();
            bool ovf = false;
            float mv = 0.f;
            const int np = run_frame<NV, CONTACT, TPR, true>(P.scene, P.KIN, P.ES, R, s, g, nsub, h, ovf,
                                                       [](int) -> const Rec* { return nullptr; },
                                                       P.reaction ? P.reaction + 4LL * R.v0 : nullptr, &mv);
            if (ovf) bad |= 2u;
            np_max = max(np_max, np);
            unsigned fl = 0u;
            for (int i = g.tid; i < R.nv; i += TPR) {
                float4 x = s.X[i], v = s.V[i];
                if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) && isfinite(v.y) &&
                      isfinite(v.z) && isfinite(v.w)))
                    fl |= 1u;
                if (P.xframes) reinterpret_cast<float4*>(P.xframes)[(long long)f * P.nvert_total + R.v0 + i] = x;
            }
            // candidates are found once per frame at its start, with a margin of contact_d - 2r:
            // two vertices that each moved less than half of it cannot have closed it
            if ((R.flags & ROD_SELF) && !(mv < 0.5f * (R.contact_d - 2.f * R.radius))) fl |= 4u;
            bad |= grp_or<TPR>(fl, g);
            if (f + 1 == P.frames) {
                if (R.flags & ROD_INEXT) {
                    // sum |C_j| in FP64, each edge length from the float32 positions in FP64
                    double r = 0.0;
                    for (int j = g.tid; j < R.ne; j += TPR) {
                        int j1 = (j + 1 == R.nv) ? 0 : j + 1;
                        const double ex = (double)s.X[j1].x - (double)s.X[j].x;
                        const double ey = (double)s.X[j1].y - (double)s.X[j].y;
                        const double ez = (double)s.X[j1].z - (double)s.X[j].z;
                        if (s.ET[j].w > 0.f)   // not a break edge
                            r += fabs(sqrt(ex * ex + ey * ey + ez * ez) - (double)s.ET[j].w);
                    }
                    r = grp_sum<TPR>(r, g);
                    if (g.tid == 0) P.residual[rod] = r;
                }
                if (g.tid == 0) P.npairs[rod] = np_max;
                if (CONTACT && P.pair_list) {   // the last frame's candidates
                    uint32_t* dst = P.pair_list + (size_t)rod * (1 + kPairListStride);
                    for (int k = g.tid; k < np; k += TPR) dst[1 + k] = s.pairs[k];
                    if (g.tid == 0) dst[0] = (uint32_t)np;
                }
            }
        }
        write_state<TPR>(P.S, 0, 0, 0, R, rod, g, s.X, s.V, s.ED, s.ET, s.HG, s.fp);
        if (g.tid == 0 && bad) atomicOr(&P.status[rod], bad);
        g.sync();
        bounds_end<TPR>(g, P.status, rod);
    }
}

// rods per CTA allowed by the thread budget
template <int NV>
__host__ __device__ constexpr int fwd_max_rpc() { return kFwdMaxThreads / threads_per_rod(NV); }

template <int NV, bool C>
static cudaError_t launch_fwd_t(const FwdParams& P, int grid, int rpc, cudaStream_t st) {
    size_t smem = rod_smem_bytes(NV, C) * rpc;
    auto k = fwd_kernel<NV, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads_per_rod(NV) * rpc, smem, st>>>(P);
    return cudaGetLastError();
}

template <int NV, bool C>
static int fwd_occ_t(int rpc) {
    if (rpc > fwd_max_rpc<NV>() || rpc < 1) return 0;
    size_t smem = rod_smem_bytes(NV, C) * rpc;
    auto k = fwd_kernel<NV, C>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads_per_rod(NV) * rpc, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

}  // namespace dlo
