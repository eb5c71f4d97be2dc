// dlo_runtime.cu -- device allocation, size-class buckets, the step launch and rollout recording
// (gradient checkpointing, DLO-Lab Sec. 3.3: one state snapshot per segment, kept in HBM).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dlo_kernels.h"
#include "dlo_runtime.h"

using namespace dlo;


template <class T>
static T* alloc_up(dlo_ctx* c, const std::vector<T>& h, dlo_status& st) {
    if (st != DLO_OK) return nullptr;
    T* d = reinterpret_cast<T*>(dev_alloc(c, sizeof(T) * std::max<size_t>(h.size(), 1)));
    if (!d) {
        st = set_err(c, DLO_ERR_OOM, "device allocation failed");
        return nullptr;
    }
    if (!h.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) st = cuda_err(c, e, "upload");
    }
    return d;
}

static void* alloc_zero(dlo_ctx* c, size_t bytes, dlo_status& st) {
    if (st != DLO_OK) return nullptr;
    void* d = dev_alloc(c, bytes);
    if (!d) {
        st = set_err(c, DLO_ERR_OOM, "device allocation failed");
        return nullptr;
    }
    cudaError_t e = cudaMemsetAsync(d, 0, bytes, c->stream);
    if (e != cudaSuccess) st = cuda_err(c, e, "memset");
    return d;
}

// Forward launch of one size class over `frames` frames without actions or recording.
static cudaError_t launch_bucket(dlo_ctx* c, size_t k, int warps, int grid, int frames) {
    const Bucket& bk = c->buckets[k];
    FwdParams P{};
    P.rods = c->d_rods;
    P.order = bk.d_order;
    P.n_order = bk.n;
    P.counter = c->d_counters + k;
    P.S = c->S;
    P.KIN = c->d_kin;
    P.ES = c->d_es;
    P.frames = frames;
    P.B = c->B;
    P.nvert_total = c->V;
    P.status = c->d_status;
    P.residual = c->d_residual;
    P.npairs = c->d_npairs;
    P.scene = c->scene;
    cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_forward(P, bk.nv_max, bk.contact, grid, warps, c->stream);
    c->launches++;
    return e;
}

// Rods per CTA by measurement (the autotuner): every count whose occupancy keeps at least
// half of the most resident rods is timed on two frames from the rest state, after one
// warm-up launch, and the fastest is kept.  The caller resets the state afterwards.
static dlo_status autotune_rods_per_cta(dlo_ctx* c) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_err(c, cudaGetLastError(), "event");
    }
    dlo_status st = DLO_OK;
    for (size_t k = 0; k < c->buckets.size() && st == DLO_OK; ++k) {
        Bucket& bk = c->buckets[k];
        int most = 0;
        for (int rpc = 1; rpc <= 16; ++rpc) most = std::max(most, rpc * forward_blocks_per_sm(bk.nv_max, bk.contact, rpc));
        float best_ms = 1e30f;
        int best_w = bk.warps, best_g = bk.grid;
        cudaError_t e = launch_bucket(c, k, bk.warps, bk.grid, 1);   // warm-up (module load, clocks)
        for (int rpc = 1; rpc <= 16 && e == cudaSuccess; ++rpc) {
            const int nb = forward_blocks_per_sm(bk.nv_max, bk.contact, rpc);
            if (nb < 1 || 2 * rpc * nb < most) continue;
            const int grid = (int)std::min<long long>((long long)nb * c->sm_count, (bk.n + rpc - 1) / rpc);
            e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) e = launch_bucket(c, k, rpc, grid, 2);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best_w = rpc;
                best_g = grid;
            }
        }
        if (e != cudaSuccess) st = cuda_err(c, e, "autotune");
        bk.warps = best_w;
        bk.grid = best_g;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

dlo_status runtime_allocate(dlo_ctx* c, const std::vector<RodInfo>& rods, const std::vector<float4>& kin,
                            const std::vector<float2>& mass, const std::vector<float2>& es,
                            const std::vector<float4>& rest, const std::vector<float>& gp0,
                            const std::vector<float4>& xr4) {
    dlo_status st = DLO_OK;
    c->d_rods = alloc_up(c, rods, st);
    c->d_kin = alloc_up(c, kin, st);
    c->d_mass = alloc_up(c, mass, st);
    c->d_es = alloc_up(c, es, st);
    c->d_rest = alloc_up(c, rest, st);
    c->d_gp0 = alloc_up(c, gp0, st);
    c->S.X = alloc_up(c, xr4, st);
    c->S.Vl = reinterpret_cast<float4*>(alloc_zero(c, 16 * c->V, st));
    c->S.HG = reinterpret_cast<float4*>(alloc_zero(c, 16 * c->V, st));
    c->S.ED = reinterpret_cast<float4*>(alloc_zero(c, 16 * c->Et, st));
    c->S.ET = reinterpret_cast<float4*>(alloc_zero(c, 16 * c->Et, st));
    c->S.GP = reinterpret_cast<float*>(alloc_zero(c, sizeof(float) * 24 * c->B, st));
    c->d_status = reinterpret_cast<unsigned*>(alloc_zero(c, sizeof(unsigned) * c->B, st));
    c->d_residual = reinterpret_cast<double*>(alloc_zero(c, sizeof(double) * c->B, st));
    c->d_npairs = reinterpret_cast<int*>(alloc_zero(c, sizeof(int) * c->B, st));
    if (c->opt.reaction) c->d_reaction = reinterpret_cast<float4*>(alloc_zero(c, 64 * c->V, st));
    if (c->opt.self_contact)
        c->d_pair_list = reinterpret_cast<uint32_t*>(
            alloc_zero(c, sizeof(uint32_t) * (1 + (size_t)kPairListStride) * c->B, st));
    if (st != DLO_OK) return st;
    // size classes; rods of a class in decreasing cost so the persistent warps balance
    std::vector<std::vector<int>> cls(kNumSizeClasses);
    for (int b = 0; b < c->B; ++b)
        for (int k = 0; k < kNumSizeClasses; ++k)
            if (size_class_at(k) == size_class(rods[b].nv)) cls[k].push_back(b);
    for (int k = 0; k < kNumSizeClasses; ++k) {
        if (cls[k].empty()) continue;
        std::vector<int>& ids = cls[k];
        std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) {
            return (long long)rods[a].nv * rods[a].nsub > (long long)rods[b].nv * rods[b].nsub;
        });
        Bucket bk;
        bk.nv_max = size_class_at(k);
        bk.contact = c->opt.self_contact != 0;
        bk.n = (int)ids.size();
        bk.d_order = alloc_up(c, ids, st);
        if (st != DLO_OK) return st;
        // rods per CTA: the count (within the thread budget) that keeps the most rods resident;
        // the measured autotune below may pick another
        int best = 0, best_nb = 0;
        for (int rpc = 1; rpc <= 16; ++rpc) {
            if (c->opt.warps_per_cta > 0 && rpc != c->opt.warps_per_cta) continue;
            const int nb = forward_blocks_per_sm(bk.nv_max, bk.contact, rpc);
            if (nb >= 1 && rpc * nb >= best * best_nb) {
                best = rpc;
                best_nb = nb;
            }
        }
        if (best < 1) return set_err(c, DLO_ERR_INVALID_ARG, "rod too large for shared memory");
        bk.warps = best;
        long long want = (bk.n + best - 1) / best;
        bk.grid = (int)std::min<long long>((long long)best_nb * c->sm_count, want);
        c->buckets.push_back(bk);
    }
    if (c->buckets.size() > 1) {   // one stream per size class (see dlo_ctx::side)
        c->side.resize(c->buckets.size(), nullptr);
        c->joins.resize(c->buckets.size(), nullptr);
        cudaError_t e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
        for (size_t k = 0; k < c->buckets.size() && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->joins[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_err(c, e, "size-class streams");
    }
    // work-queue heads: one per size class for the forward, one per class for the backward
    c->d_counters = reinterpret_cast<int*>(alloc_zero(c, sizeof(int) * 2 * kNumSizeClasses, st));
    if (st != DLO_OK) return st;
    // rest twist from the rest frames, then the rest state
    InitParams P{};
    P.rods = c->d_rods;
    P.B = c->B;
    P.xin = c->S.X;
    P.mass = c->d_mass;
    P.ES = c->d_es;
    P.rest = c->d_rest;
    P.S = c->S;
    P.GP0 = c->d_gp0;
    P.rest_mode = 1;
    st = cuda_err(c, launch_init(P, c->stream), "rest init");
    if (st != DLO_OK) return st;
    P.rest_mode = 0;
    st = cuda_err(c, launch_init(P, c->stream), "state init");
    c->launches += 2;
    if (st == DLO_OK && c->opt.warps_per_cta == 0) {
        // measured autotune of rods per CTA; then the rest state is set again (positions
        // re-uploaded, frames, velocities and poses re-initialised, status cleared)
        st = autotune_rods_per_cta(c);
        if (st == DLO_OK)
            st = cuda_err(c, cudaMemcpyAsync(c->S.X, xr4.data(), sizeof(float4) * xr4.size(), cudaMemcpyHostToDevice,
                                             c->stream), "rest positions");
        if (st == DLO_OK)
            st = cuda_err(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned) * c->B, c->stream), "status reset");
        if (st == DLO_OK) st = cuda_err(c, launch_init(P, c->stream), "state init");
        c->launches++;
    }
    c->from_set_state = true;
    if (st == DLO_OK) st = cuda_err(c, cudaStreamSynchronize(c->stream), "create");
    return st;
}

void runtime_release(dlo_ctx* c) {
    for (cudaStream_t s : c->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->joins) cudaEventDestroy(e);
    if (c->fork) cudaEventDestroy(c->fork);
    c->side.clear();
    c->joins.clear();
    c->fork = nullptr;
}

cudaStream_t class_stream(dlo_ctx* c, size_t k) { return c->side.empty() ? c->stream : c->side[k]; }

cudaError_t fork_classes(dlo_ctx* c) {
    if (c->side.empty()) return cudaSuccess;
    cudaError_t e = cudaEventRecord(c->fork, c->stream);
    for (size_t k = 0; k < c->side.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c->side[k], c->fork, 0);
    return e;
}

cudaError_t join_classes(dlo_ctx* c) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < c->side.size() && e == cudaSuccess; ++k) {
        e = cudaEventRecord(c->joins[k], c->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->joins[k], 0);
    }
    return e;
}

// ------------------------------------------------------------------ rollout recording
extern "C" dlo_status dlo_begin_rollout(dlo_ctx* c, int n_frames) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (n_frames <= 0) return set_err(c, DLO_ERR_INVALID_ARG, "n_frames must be positive");
    const size_t per = 16 * (3 * (size_t)c->V + 2 * (size_t)c->Et) + sizeof(float) * 24 * (size_t)c->B;
    const size_t abytes = sizeof(float) * 12 * (size_t)c->B * n_frames;
    int K = std::min(c->opt.checkpoint_every, n_frames);
    const size_t budget = c->opt.hbm_budget ? c->opt.hbm_budget : ((size_t)80 << 30);
    if (K <= 0) {
        // autotune: the shortest interval (the least recomputation in the backward) whose
        // checkpoint ring, action record and backward workspace fit the HBM budget; the
        // backward reruns at most K - 1 frames per segment to rebuild the frame-start states
        K = n_frames;
        for (int k = 1; k <= n_frames; ++k) {
            BwdPlan plan;
            if (bwd_plan(c, 0, k, plan) != DLO_OK) return DLO_ERR_INVALID_ARG;
            const size_t total = per * (size_t)((n_frames + k - 1) / k) + abytes + plan.bytes;
            if (total <= budget) {
                K = k;
                break;
            }
        }
    }
    const int count = (n_frames + K - 1) / K;
    // Frames per backward launch pair: the chunk records may take half of what the ring and the
    // action record leave of the budget (at most 24 GiB), and never less than the default the
    // interval was chosen with.  Longer chunks mean fewer launch pairs, each with its own tail.
    {
        const size_t used = per * (size_t)count + abytes;
        const size_t spare = budget > used ? budget - used : 0;
        const size_t dflt = std::min<size_t>((size_t)8 << 30, budget / 8);
        c->rec_budget = std::max(dflt, std::min<size_t>((size_t)24 << 30, spare / 2));
    }
    const size_t need = per * count + 256 * 8;
    if (need > c->ck_bytes) {
        dev_free(c, c->ck_mem);
        c->ck_mem = dev_alloc(c, need);
        c->ck_bytes = c->ck_mem ? need : 0;
        if (!c->ck_mem) return set_err(c, DLO_ERR_OOM, "checkpoint ring allocation failed");
    }
    char* p = reinterpret_cast<char*>(c->ck_mem);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    c->ck.X = reinterpret_cast<float4*>(take(16 * c->V * count));
    c->ck.Vl = reinterpret_cast<float4*>(take(16 * c->V * count));
    c->ck.HG = reinterpret_cast<float4*>(take(16 * c->V * count));
    c->ck.ED = reinterpret_cast<float4*>(take(16 * c->Et * count));
    c->ck.ET = reinterpret_cast<float4*>(take(16 * c->Et * count));
    c->ck.GP = reinterpret_cast<float*>(take(sizeof(float) * 24 * c->B * count));
    if (abytes > c->rec_bytes) {
        dev_free(c, c->rec_actions);
        c->rec_actions = reinterpret_cast<float*>(dev_alloc(c, abytes));
        c->rec_bytes = c->rec_actions ? abytes : 0;
        if (!c->rec_actions) return set_err(c, DLO_ERR_OOM, "action record allocation failed");
    }
    c->ck_every = K;
    c->ck_count = count;
    c->rec_frames = n_frames;
    c->rec_done = 0;
    c->rec_active = true;
    c->rec_from_set = c->from_set_state;
    c->rec_nsub = -1;
    return DLO_OK;
}

// ------------------------------------------------------------------ step
dlo_status launch_step(dlo_ctx* c, const float* actions, int frames, int substeps, float* x_frames, int frame0,
                       bool record) {
    cudaError_t fe = fork_classes(c);
    if (fe != cudaSuccess) return cuda_err(c, fe, "fork");
    for (size_t k = 0; k < c->buckets.size(); ++k) {
        const Bucket& bk = c->buckets[k];
        FwdParams P{};
        P.rods = c->d_rods;
        P.order = bk.d_order;
        P.n_order = bk.n;
        P.counter = c->d_counters + k;
        P.S = c->S;
        P.KIN = c->d_kin;
        P.ES = c->d_es;
        P.actions = actions;
        P.xframes = x_frames;
        P.frames = frames;
        P.B = c->B;
        P.force_nsub = substeps;
        P.frame0 = frame0;
        P.nvert_total = c->V;
        if (record) {
            P.ck = c->ck;
            P.ck_strideV = c->V;
            P.ck_strideE = c->Et;
            P.ck_strideB = 24LL * c->B;
            P.ck_every = c->ck_every;
            P.ck_count = c->ck_count;
        }
        P.status = c->d_status;
        P.residual = c->d_residual;
        P.npairs = c->d_npairs;
        P.reaction = c->d_reaction;
        P.pair_list = c->d_pair_list;
        P.scene = c->scene;
        cudaStream_t sk = class_stream(c, k);
        cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), sk);
        if (e == cudaSuccess) e = launch_forward(P, bk.nv_max, bk.contact, bk.grid, bk.warps, sk);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "forward launch");
    }
    fe = join_classes(c);
    if (fe != cudaSuccess) return cuda_err(c, fe, "join");
    return DLO_OK;
}

extern "C" dlo_status dlo_step(dlo_ctx* c, const float* actions, int frames, int substeps, float* x_frames) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (frames < 0 || substeps < 0 || substeps > 100000) return set_err(c, DLO_ERR_INVALID_ARG, "bad frames/substeps");
    if (x_frames && ((uintptr_t)x_frames & 15u)) return set_err(c, DLO_ERR_INVALID_ARG, "x_frames must be 16-byte aligned");
    if (frames == 0) return DLO_OK;
    const bool rec = c->rec_active && c->rec_done < c->rec_frames;
    int frame0 = 0;
    const float* acts = actions;
    if (rec) {
        if (c->rec_done + frames > c->rec_frames)
            return set_err(c, DLO_ERR_STATE, "step runs past the frames armed by dlo_begin_rollout");
        if (c->rec_nsub >= 0 && c->rec_nsub != substeps)
            return set_err(c, DLO_ERR_STATE, "substeps changed inside a recorded rollout");
        c->rec_nsub = substeps;
        float* dst = c->rec_actions + (size_t)12 * c->B * c->rec_done;
        cudaError_t e = actions ? cudaMemcpyAsync(dst, actions, sizeof(float) * 12 * c->B * frames,
                                                  cudaMemcpyDeviceToDevice, c->stream)
                                : cudaMemsetAsync(dst, 0, sizeof(float) * 12 * c->B * frames, c->stream);
        if (e != cudaSuccess) return cuda_err(c, e, "record actions");
        frame0 = c->rec_done;
        acts = dst;
    } else {
        c->rec_active = false;
    }
    dlo_status st = launch_step(c, acts, frames, substeps, x_frames, frame0, rec);
    if (st != DLO_OK) return st;
    if (rec) c->rec_done += frames;
    c->from_set_state = false;
    return DLO_OK;
}
