// dlo_adjoint.cu -- hand-written adjoint of the rod stepper with gradient checkpointing.
//
// DLO-Lab (Sec. 3.3) differentiates whole trajectories by caching one state per segment and,
// for each segment in reverse, re-running the forward simulation before back-propagating.
// Here the checkpoints live in HBM (written by the forward kernel every K frames) and one
// thread group runs the whole backward of one rod:
//   for each segment, last first: reload its checkpoint, recompute its frames storing the
//   frame-start states (per-rod scratch); for each frame, last first: recompute it storing
//   the substep-start states; for each substep, last first: recompute it once more recording
//   its intermediates (velocity before contact, PBD iteration snapshots, displacement before
//   friction), then apply the vector-Jacobian product of every phase in reverse order.
// Second-order terms of the elastic forces are exact: the hinge gradient (a hand reverse pass)
// is re-run on dual numbers, giving d/de [dU/dz](x + e lambda) for every input z, which is
// the transpose-Jacobian product of the force (U's Hessian is symmetric).  Branches (contact
// on/off, yield, strain-limit activity, pair sets) follow the recomputed forward.
#include <algorithm>
#include <cstring>
#include <vector>

#include "dlo_runtime.h"
#include "dlo_kernels.h"
#include "dlo_physics.cuh"

namespace dlo {

// ------------------------------------------------------------------ initial frames adjoint
// Reverse of the frame construction of dlo_set_state (space-parallel transport, holonomy
// spread for loops): cotangents of the initial base (t, d1) -> positions. FP64, one thread
// per rod.
__device__ __forceinline__ V3<double> ld(float4 a) { return V3<double>{(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ V3<double> unit_d(V3<double> a) { return a / sqrt(dot(a, a)); }
__device__ __forceinline__ V3<double> adapt_fwd(V3<double> w, V3<double> t) { return unit_d(w - dot(w, t) * t); }
// reverse of u = adapt(w, t): returns lambda_w, adds lambda_t
__device__ __forceinline__ V3<double> adapt_rev(V3<double> w, V3<double> t, V3<double> lu, V3<double>& lt) {
    V3<double> dd = w - dot(w, t) * t;
    double n = sqrt(dot(dd, dd));
    V3<double> u = dd / n;
    V3<double> ldd = (lu - dot(lu, u) * u) / n;
    lt += -dot(w, t) * ldd - dot(ldd, t) * w;
    return ldd - dot(ldd, t) * t;
}
// reverse of u = transport(a, b, d): adds lambda_a, lambda_b, returns lambda_d
__device__ __forceinline__ V3<double> transport_rev(V3<double> A, V3<double> Bv, V3<double> d, V3<double> lu,
                                                    V3<double>& la, V3<double>& lb) {
    double c = dot(A, Bv);
    V3<double> k = cross(A, Bv);
    double kd = dot(k, d), luk = dot(lu, k), opc = 1.0 + c;
    double lc = dot(lu, d) - kd * luk / (opc * opc);
    V3<double> lk = cross(d, lu) + (kd / opc) * lu + (luk / opc) * d;
    la += lc * Bv + cross(Bv, lk);
    lb += lc * A + cross(lk, A);
    return c * lu + cross(lu, k) + (luk / opc) * k;
}

__global__ void frames_adjoint_kernel(const RodInfo* rods, int B, const float4* X0, const float4* gtb0,
                                      const float4* gd1b0, float4* gx0, V3<double>* work) {
    const int rod = blockIdx.x * blockDim.x + threadIdx.x;
    if (rod >= B) return;
    const RodInfo R = rods[rod];
    const int nv = R.nv, ne = R.ne, v0 = R.v0, e0 = R.e0;
    const bool closed = R.flags & ROD_CLOSED;
    V3<double>* T = work + 4 * (size_t)v0;          // tangents [ne]
    V3<double>* Dh = T + nv;                       // uncorrected frames [ne]
    V3<double>* Lt = Dh + nv;                      // tangent cotangents [ne]
    V3<double>* Ldh = Lt + nv;                     // cotangents of the uncorrected frames [ne]
    auto X = [&](int i) { return ld(X0[v0 + i]); };
    for (int j = 0; j < ne; ++j) T[j] = unit_d(X(j + 1 == nv ? 0 : j + 1) - X(j));
    V3<double> ax = fabs(T[0].z) < 0.9 ? V3<double>{0.0, 0.0, 1.0} : V3<double>{1.0, 0.0, 0.0};
    Dh[0] = adapt_fwd(ax, T[0]);
    for (int j = 1; j < ne; ++j) Dh[j] = adapt_fwd(transport_d(T[j - 1], T[j], Dh[j - 1]), T[j]);
    double psi = 0.0;
    V3<double> wl{0, 0, 0}, u{0, 0, 0};
    if (closed) {
        wl = transport_d(T[ne - 1], T[0], Dh[ne - 1]);
        u = adapt_fwd(wl, T[0]);
        psi = atan2(dot(cross(Dh[0], u), T[0]), dot(Dh[0], u));
    }
    for (int j = 0; j < ne; ++j) Lt[j] = ld(gtb0[e0 + j]);
    // cotangents of the uncorrected frames from the (corrected) output frames
    double lpsi = 0.0;
    for (int j = 0; j < ne; ++j) {
        V3<double> l1 = ld(gd1b0[e0 + j]);
        if (closed) {
            double phi = -psi * (double)j / (double)ne, cph = cos(phi), sph = sin(phi);
            Ldh[j] = cph * l1 + sph * cross(l1, T[j]);
            Lt[j] += sph * cross(Dh[j], l1);
            double lphi = dot(l1, -sph * Dh[j] + cph * cross(T[j], Dh[j]));
            lpsi += -(double)j / (double)ne * lphi;
        } else {
            Ldh[j] = l1;
        }
    }
    if (closed) {
        double y = dot(cross(Dh[0], u), T[0]), x = dot(Dh[0], u), r2 = x * x + y * y;
        double ly = lpsi * x / r2, lx = -lpsi * y / r2;
        V3<double> lu = ly * cross(T[0], Dh[0]) + lx * Dh[0];
        Ldh[0] += ly * cross(u, T[0]) + lx * u;
        Lt[0] += ly * cross(Dh[0], u);
        V3<double> lw = adapt_rev(wl, T[0], lu, Lt[0]);
        Ldh[ne - 1] += transport_rev(T[ne - 1], T[0], Dh[ne - 1], lw, Lt[ne - 1], Lt[0]);
    }
    for (int j = ne - 1; j >= 1; --j) {
        V3<double> w = transport_d(T[j - 1], T[j], Dh[j - 1]);
        V3<double> lw = adapt_rev(w, T[j], Ldh[j], Lt[j]);
        Ldh[j - 1] += transport_rev(T[j - 1], T[j], Dh[j - 1], lw, Lt[j - 1], Lt[j]);
    }
    adapt_rev(ax, T[0], Ldh[0], Lt[0]);
    for (int j = 0; j < ne; ++j) {
        const int j1 = j + 1 == nv ? 0 : j + 1;
        V3<double> e = X(j1) - X(j);
        double l = sqrt(dot(e, e));
        V3<double> t = e / l;
        V3<double> le = (Lt[j] - dot(Lt[j], t) * t) / l;
        float4 a0 = gx0[v0 + j], a1 = gx0[v0 + j1];
        gx0[v0 + j] = make_float4(a0.x - (float)le.x, a0.y - (float)le.y, a0.z - (float)le.z, a0.w);
        gx0[v0 + j1] = make_float4(a1.x + (float)le.x, a1.y + (float)le.y, a1.z + (float)le.z, a1.w);
    }
}

cudaError_t launch_backward(const BwdParams& P, int nv, bool c, int grid, int warps, cudaStream_t st) {
    switch (nv) {
        case 32: return launch_backward_nv32(P, c, grid, warps, st);
        case 64: return launch_backward_nv64(P, c, grid, warps, st);
        case 128: return launch_backward_nv128(P, c, grid, warps, st);
        case 192: return launch_backward_nv192(P, c, grid, warps, st);
        case 224: return launch_backward_nv224(P, c, grid, warps, st);
        case 256: return launch_backward_nv256(P, c, grid, warps, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_frames_adjoint(const RodInfo* rods, int B, const float4* X0, const float4* gtb0,
                                  const float4* gd1b0, float4* gx0, V3<double>* work, cudaStream_t st) {
    frames_adjoint_kernel<<<(B + 127) / 128, 128, 0, st>>>(rods, B, X0, gtb0, gd1b0, gx0, work);
    return cudaGetLastError();
}

int backward_blocks_per_sm(int nv, bool c, int warps) {
    switch (nv) {
        case 32: return backward_occ_nv32(c, warps);
        case 64: return backward_occ_nv64(c, warps);
        case 128: return backward_occ_nv128(c, warps);
        case 192: return backward_occ_nv192(c, warps);
        case 224: return backward_occ_nv224(c, warps);
        case 256: return backward_occ_nv256(c, warps);
    }
    return 0;
}

}  // namespace dlo

using namespace dlo;

// Launch shape and workspace of the backward for checkpoint interval K: per size class the
// rods per CTA and CTAs that keep the most rods resident, each resident rod's recompute
// scratch (frame-start states of one segment, substep-start states and records of one
// frame), plus the batch-wide frame cotangents and the FP64 work of the frame adjoint.
dlo_status bwd_plan(dlo_ctx* c, int force, int K, BwdPlan& out) {
    const size_t nb_ = c->buckets.size();
    out.slot_b.assign(nb_, 0);
    out.offset.assign(nb_, 0);
    out.warps.assign(nb_, 0);
    out.grid.assign(nb_, 0);
    out.nsmax.assign(nb_, 0);
    size_t need = 0;
    for (size_t k = 0; k < nb_; ++k) {
        const Bucket& bk = c->buckets[k];
        int w = 0, nb = 0;
        for (int rpc = 1; rpc <= 16; ++rpc) {
            const int b = backward_blocks_per_sm(bk.nv_max, bk.contact, rpc);
            if (b >= 1 && rpc * b >= w * nb) {
                w = rpc;
                nb = b;
            }
        }
        if (w < 1) return set_err(c, DLO_ERR_INVALID_ARG, "rod too large for the backward kernel's shared memory");
        int ns = force;
        if (!ns)
            for (int b = 0; b < c->B; ++b)
                if (size_class(c->rods_h[b].nv) == bk.nv_max)
                    ns = std::max(ns, c->nsub[b]);
        out.nsmax[k] = ns;
        const size_t NV = bk.nv_max;
        out.slot_b[k] = 16 * ((size_t)K * (5 * NV + 6) +
                              (size_t)ns * ((7 + 2 * kPairsPerVertex) * NV + (size_t)4 * c->opt.n_iter_pbd * NV));
        out.warps[k] = w;
        out.grid[k] = (int)std::min<long long>((long long)nb * c->sm_count, (bk.n + w - 1) / w);
        // each class has its own region: the classes run concurrently on their streams
        out.offset[k] = need;
        need += (out.slot_b[k] * (size_t)out.grid[k] * w + 255) & ~(size_t)255;
    }
    out.bytes = need + 2 * 16 * (size_t)c->Et + 4 * sizeof(V3<double>) * (size_t)c->V + 1024;
    return DLO_OK;
}

extern "C" dlo_status dlo_backward(dlo_ctx* c, const float* dL_dx_T, const float* dL_dv_T, const float* dL_dtheta_T,
                                   float* dL_dactions, float* dL_dmaterial, float* dL_dx0, float* dL_dv0,
                                   float* dL_dtheta0) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!c->rec_active || c->rec_done != c->rec_frames || c->rec_frames == 0)
        return set_err(c, DLO_ERR_STATE, "dlo_backward needs a completed rollout armed by dlo_begin_rollout");
    for (const void* p : {(const void*)dL_dx_T, (const void*)dL_dv_T, (const void*)dL_dx0, (const void*)dL_dv0})
        if (p && ((uintptr_t)p & 15u)) return set_err(c, DLO_ERR_INVALID_ARG, "float4 arrays must be 16-byte aligned");
    if (c->opt.self_contact && c->opt.n_iter_pbd < 1)
        return set_err(c, DLO_ERR_INVALID_ARG, "self-contact gradients need at least one projection iteration");
    const int force = c->rec_nsub > 0 ? c->rec_nsub : 0;
    BwdPlan plan;
    dlo_status pst = bwd_plan(c, force, c->ck_every, plan);
    if (pst != DLO_OK) return pst;
    const size_t need = plan.bytes;
    const std::vector<size_t>& slot_b = plan.slot_b;
    const std::vector<int>&warps = plan.warps, &grid = plan.grid, &nsmax = plan.nsmax;
    const std::vector<size_t>& offset = plan.offset;
    if (need > c->bw_bytes) {
        dev_free(c, c->bw_mem);
        c->bw_mem = dev_alloc(c, need);
        c->bw_bytes = c->bw_mem ? need : 0;
        if (!c->bw_mem) return set_err(c, DLO_ERR_OOM, "backward scratch allocation failed");
    }
    char* p = reinterpret_cast<char*>(c->bw_mem);
    float4* gtb0 = reinterpret_cast<float4*>(p);
    float4* gd1b0 = gtb0 + c->Et;
    V3<double>* work = reinterpret_cast<V3<double>*>(gd1b0 + c->Et);
    char* scratch = reinterpret_cast<char*>(work + 4 * (size_t)c->V);
    scratch = reinterpret_cast<char*>(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    {
        cudaError_t fe = fork_classes(c);
        if (fe != cudaSuccess) return cuda_err(c, fe, "fork");
    }
    for (size_t k = 0; k < c->buckets.size(); ++k) {
        const Bucket& bk = c->buckets[k];
        BwdParams P{};
        P.rods = c->d_rods;
        P.order = bk.d_order;
        P.n_order = bk.n;
        P.counter = c->d_counters + kNumSizeClasses + k;
        P.ck = c->ck;
        P.ck_strideV = c->V;
        P.ck_strideE = c->Et;
        P.ck_strideB = 24LL * c->B;
        P.ck_every = c->ck_every;
        P.ck_count = c->ck_count;
        P.KIN = c->d_kin;
        P.ES = c->d_es;
        P.actions = c->rec_actions;
        P.frames = c->rec_frames;
        P.B = c->B;
        P.force_nsub = force;
        P.dLdx = reinterpret_cast<const float4*>(dL_dx_T);
        P.dLdv = reinterpret_cast<const float4*>(dL_dv_T);
        P.dLdth = dL_dtheta_T;
        P.gact = dL_dactions;
        P.gmat = dL_dmaterial;
        P.gx0 = reinterpret_cast<float4*>(dL_dx0);
        P.gv0 = reinterpret_cast<float4*>(dL_dv0);
        P.gth0 = dL_dtheta0;
        P.gtb0 = gtb0;
        P.gd1b0 = gd1b0;
        P.scratch = scratch + offset[k];
        P.slot_bytes = slot_b[k];
        P.K = c->ck_every;
        P.nsub_max = nsmax[k];
        P.scene = c->scene;
        cudaStream_t sk = class_stream(c, k);
        cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), sk);
        if (e == cudaSuccess) e = launch_backward(P, bk.nv_max, bk.contact, grid[k], warps[k], sk);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "backward launch");
    }
    {
        cudaError_t je = join_classes(c);
        if (je != cudaSuccess) return cuda_err(c, je, "join");
    }
    if (c->rec_from_set && dL_dx0) {
        frames_adjoint_kernel<<<(c->B + 127) / 128, 128, 0, c->stream>>>(c->d_rods, c->B, c->ck.X, gtb0, gd1b0,
                                                                        reinterpret_cast<float4*>(dL_dx0), work);
        c->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(c, e, "frames adjoint launch");
    }
    return check_status(c);
}
