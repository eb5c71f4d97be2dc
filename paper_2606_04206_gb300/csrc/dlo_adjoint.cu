// dlo_adjoint.cu -- host side of the hand-written adjoint with gradient checkpointing, and the
// FP64 adjoint of the initial reference frames.
//
// DLO-Lab (Sec. 3.3) differentiates whole trajectories by caching one state per segment and,
// for each segment in reverse, re-running the forward simulation before back-propagating.
// Here the checkpoints live in HBM (written by the forward kernel every K frames).  The
// rollout is reversed in chunks of C frames, last first; per chunk, rec_kernel re-runs the
// chunk's frames from their start state storing every substep's records, then rev_kernel
// reverses them (dlo_bwd_kernel.cuh).  C is a multiple of K when C >= K, so that every chunk
// starts at a checkpoint; otherwise the frame-start states of each segment are stored first.
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

cudaError_t launch_rec(const BwdParams& P, int nv, bool c, int grid, int warps, cudaStream_t st) {
    switch (nv) {
        case 32: return launch_rec_nv32(P, c, grid, warps, st);
        case 64: return launch_rec_nv64(P, c, grid, warps, st);
        case 128: return launch_rec_nv128(P, c, grid, warps, st);
        case 192: return launch_rec_nv192(P, c, grid, warps, st);
        case 224: return launch_rec_nv224(P, c, grid, warps, st);
        case 256: return launch_rec_nv256(P, c, grid, warps, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rev(const BwdParams& P, int nv, bool c, int grid, int warps, cudaStream_t st) {
    switch (nv) {
        case 32: return launch_rev_nv32(P, c, grid, warps, st);
        case 64: return launch_rev_nv64(P, c, grid, warps, st);
        case 128: return launch_rev_nv128(P, c, grid, warps, st);
        case 192: return launch_rev_nv192(P, c, grid, warps, st);
        case 224: return launch_rev_nv224(P, c, grid, warps, st);
        case 256: return launch_rev_nv256(P, c, grid, warps, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_frames_adjoint(const RodInfo* rods, int B, const float4* X0, const float4* gtb0,
                                  const float4* gd1b0, float4* gx0, V3<double>* work, cudaStream_t st) {
    frames_adjoint_kernel<<<(B + 127) / 128, 128, 0, st>>>(rods, B, X0, gtb0, gd1b0, gx0, work);
    return cudaGetLastError();
}

int rec_blocks_per_sm(int nv, bool c, int warps) {
    switch (nv) {
        case 32: return rec_occ_nv32(c, warps);
        case 64: return rec_occ_nv64(c, warps);
        case 128: return rec_occ_nv128(c, warps);
        case 192: return rec_occ_nv192(c, warps);
        case 224: return rec_occ_nv224(c, warps);
        case 256: return rec_occ_nv256(c, warps);
    }
    return 0;
}

int rev_blocks_per_sm(int nv, bool c, int warps) {
    switch (nv) {
        case 32: return rev_occ_nv32(c, warps);
        case 64: return rev_occ_nv64(c, warps);
        case 128: return rev_occ_nv128(c, warps);
        case 192: return rev_occ_nv192(c, warps);
        case 224: return rev_occ_nv224(c, warps);
        case 256: return rev_occ_nv256(c, warps);
    }
    return 0;
}

}  // namespace dlo

using namespace dlo;

namespace {

// record sizes (float4) of one rod of the class: cf. sub_rec / frame_rec / seg_state / cot_state
size_t frame_rec_h(int NV, int n_iter, int nsub) {
    return (size_t)(8 + NV) + (size_t)nsub * (size_t)(7 + 2 * n_iter + 2 * kPairsPerVertex) * NV;
}

// rods per CTA and CTAs per SM that keep the most rods resident
void best_shape(int nv, bool contact, bool rec, int& w, int& nb) {
    w = 0;
    nb = 0;
    for (int rpc = 1; rpc <= 16; ++rpc) {
        const int b = rec ? rec_blocks_per_sm(nv, contact, rpc) : rev_blocks_per_sm(nv, contact, rpc);
        if (b >= 1 && rpc * b >= w * nb) {
            w = rpc;
            nb = b;
        }
    }
}

}  // namespace

// Plan of the chunked backward for checkpoint interval K: frames per chunk C (the records of
// one chunk of every rod within rec_budget, at most 64 frames), per-rod buffer sizes and the
// workspace of all rods at once.
dlo_status bwd_plan(dlo_ctx* c, int force, int K, BwdPlan& out, size_t rec_budget) {
    const size_t nb_ = c->buckets.size();
    if (!rec_budget) {
        const size_t budget = c->opt.hbm_budget ? c->opt.hbm_budget : ((size_t)80 << 30);
        rec_budget = std::min<size_t>((size_t)8 << 30, budget / 8);
    }
    out.nsmax.assign(nb_, 0);
    out.C.assign(nb_, 1);
    out.r3_rod.assign(nb_, 0);
    out.l2_rod.assign(nb_, 0);
    out.cs_rod.assign(nb_, 0);
    out.offset.assign(nb_, 0);
    size_t per_frame = 0;
    for (size_t k = 0; k < nb_; ++k) {
        const Bucket& bk = c->buckets[k];
        int w, nb;
        best_shape(bk.nv_max, bk.contact, false, w, nb);
        if (w < 1) return set_err(c, DLO_ERR_INVALID_ARG, "rod too large for the backward kernel's shared memory");
        best_shape(bk.nv_max, bk.contact, true, w, nb);
        if (w < 1) return set_err(c, DLO_ERR_INVALID_ARG, "rod too large for the recompute kernel's shared memory");
        int ns = force;
        if (!ns)
            for (int b = 0; b < c->B; ++b)
                if (size_class(c->rods_h[b].nv) == bk.nv_max) ns = std::max(ns, c->nsub[b]);
        out.nsmax[k] = ns;
        per_frame += 16 * (size_t)bk.n * frame_rec_h(bk.nv_max, c->opt.n_iter_pbd, ns);
    }
    int C = (int)std::max<size_t>(1, std::min<size_t>(64, rec_budget / std::max<size_t>(per_frame, 1)));
    if (C >= K) C = (C / K) * K;   // chunks start at checkpoints
    size_t need = 0;
    for (size_t k = 0; k < nb_; ++k) {
        const Bucket& bk = c->buckets[k];
        const int NV = bk.nv_max;
        out.C[k] = C;
        out.r3_rod[k] = (size_t)C * frame_rec_h(NV, c->opt.n_iter_pbd, out.nsmax[k]);
        out.l2_rod[k] = C < K ? (size_t)K * (5 * (size_t)NV + 6) : 0;
        out.cs_rod[k] = 5 * (size_t)NV + 6;
        out.offset[k] = need;   // each class has its own region: the classes run concurrently
        need += (16 * (size_t)bk.n * (out.r3_rod[k] + out.l2_rod[k] + out.cs_rod[k]) + 255) & ~(size_t)255;
    }
    out.fixed = (2 * 16 * (size_t)c->Et + 4 * sizeof(V3<double>) * (size_t)c->V + 1024 + 255) & ~(size_t)255;
    out.bytes = out.fixed + need;
    return DLO_OK;
}

dlo_status enqueue_backward_class(dlo_ctx* c, const BwdPlan& plan, size_t k, cudaStream_t st, int item0, int n,
                                  float4* R3, float4* L2, float4* CS, int C, const BwdParams& common) {
    const Bucket& bk = c->buckets[k];
    BwdParams P = common;
    P.order = bk.d_order;
    P.item0 = item0;
    P.n_items = n;
    P.counter = c->d_counters + kNumSizeClasses + k;
    P.nsub_max = plan.nsmax[k];
    P.R3 = R3;
    P.L2 = L2;
    P.CS = CS;
    backward_rod_f4(c, plan, k, C, P.r3_rod, P.l2_rod, P.cs_rod);
    int rec_w, rec_nb, rev_w, rev_nb;
    best_shape(bk.nv_max, bk.contact, true, rec_w, rec_nb);
    best_shape(bk.nv_max, bk.contact, false, rev_w, rev_nb);
    const int rec_grid = (int)std::min<long long>((long long)rec_nb * c->sm_count, (n + rec_w - 1) / rec_w);
    const int rev_grid = (int)std::min<long long>((long long)rev_nb * c->sm_count, (n + rev_w - 1) / rev_w);
    const int K = c->ck_every, F = c->rec_frames;
    // the chunks, first to last: from every checkpoint when C >= K (C a multiple of K), else
    // within each segment
    std::vector<std::pair<int, int>> chunks;
    if (C >= K) {
        for (int fa = 0; fa < F; fa += C) chunks.push_back({fa, std::min(fa + C, F)});
    } else {
        for (int f0 = 0; f0 < F; f0 += K) {
            const int f1 = std::min(f0 + K, F);
            for (int fa = f0; fa < f1; fa += C) chunks.push_back({fa, std::min(fa + C, f1)});
        }
    }
    for (size_t q = chunks.size(); q-- > 0;) {
        const int fa = chunks[q].first, fb = chunks[q].second;
        const int f0 = (fa / K) * K;
        cudaError_t e = cudaSuccess;
        if (C < K && fb == std::min(f0 + K, F)) {   // entering a segment: its frame-start states
            P.mode = 0;
            P.fa = f0;
            P.fb = f0;
            e = cudaMemsetAsync(P.counter, 0, sizeof(int), st);
            if (e == cudaSuccess) e = launch_rec(P, bk.nv_max, bk.contact, rec_grid, rec_w, st);
            c->launches++;
        }
        P.mode = 1;
        P.fa = fa;
        P.fb = fb;
        if (e == cudaSuccess) e = cudaMemsetAsync(P.counter, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_rec(P, bk.nv_max, bk.contact, rec_grid, rec_w, st);
        P.first_chunk = fb == F;
        P.last_chunk = fa == 0;
        if (e == cudaSuccess) e = cudaMemsetAsync(P.counter, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_rev(P, bk.nv_max, bk.contact, rev_grid, rev_w, st);
        c->launches += 2;
        if (e != cudaSuccess) return cuda_err(c, e, "backward launch");
    }
    return DLO_OK;
}

void backward_rod_f4(dlo_ctx* c, const BwdPlan& plan, size_t k, int C, size_t& r3, size_t& l2, size_t& cs) {
    const int NV = c->buckets[k].nv_max, K = c->ck_every;
    r3 = (size_t)C * frame_rec_h(NV, c->opt.n_iter_pbd, plan.nsmax[k]);
    l2 = C < K ? (size_t)K * (5 * (size_t)NV + 6) : 0;
    cs = plan.cs_rod[k];
}

int backward_resident_rods(dlo_ctx* c, size_t k) {
    int w, nb;
    best_shape(c->buckets[k].nv_max, c->buckets[k].contact, false, w, nb);
    return w * nb * c->sm_count;
}

// the inputs and outputs shared by every launch of one backward
BwdParams backward_common(dlo_ctx* c, int force, const float* dL_dx_T, const float* dL_dv_T, const float* dL_dtheta_T,
                          float* dL_dactions, float* dL_dmaterial, float* dL_dx0, float* dL_dv0, float* dL_dtheta0,
                          float4* gtb0, float4* gd1b0) {
    BwdParams P{};
    P.rods = c->d_rods;
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
    P.status = c->d_status;
    P.scene = c->scene;
    return P;
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
    dlo_status pst = bwd_plan(c, force, c->ck_every, plan, c->rec_budget);
    if (pst != DLO_OK) return pst;
    if (plan.bytes > c->bw_bytes) {
        dev_free(c, c->bw_mem);
        c->bw_mem = dev_alloc(c, plan.bytes);
        c->bw_bytes = c->bw_mem ? plan.bytes : 0;
        if (!c->bw_mem) return set_err(c, DLO_ERR_OOM, "backward workspace allocation failed");
    }
    char* p = reinterpret_cast<char*>(c->bw_mem);
    float4* gtb0 = reinterpret_cast<float4*>(p);
    float4* gd1b0 = gtb0 + c->Et;
    V3<double>* work = reinterpret_cast<V3<double>*>(gd1b0 + c->Et);
    char* region = p + plan.fixed;
    const BwdParams common = backward_common(c, force, dL_dx_T, dL_dv_T, dL_dtheta_T, dL_dactions, dL_dmaterial,
                                             dL_dx0, dL_dv0, dL_dtheta0, gtb0, gd1b0);
    {
        cudaError_t fe = fork_classes(c);
        if (fe != cudaSuccess) return cuda_err(c, fe, "fork");
    }
    for (size_t k = 0; k < c->buckets.size(); ++k) {
        const int n = c->buckets[k].n;
        float4* R3 = reinterpret_cast<float4*>(region + plan.offset[k]);
        float4* L2 = R3 + (size_t)n * plan.r3_rod[k];
        float4* CS = L2 + (size_t)n * plan.l2_rod[k];
        dlo_status st = enqueue_backward_class(c, plan, k, class_stream(c, k), 0, n, R3, L2, CS, plan.C[k], common);
        if (st != DLO_OK) return st;
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
