// dlo_noalloc.cu -- dlo_backward_noalloc: the rollout adjoint with no memory allocation.
//
// dlo_backward grows a workspace through the context's allocator whenever a rollout needs
// more recompute scratch than the last one did.  Some callers cannot allocate during the
// call: an optimisation loop that has already handed the rest of its device memory budget
// to other work (a torch caching-allocator pool at capacity, or memory partitioned between
// many simulation workers) would fail there with an out-of-memory error in the middle of a
// run, and a caller that holds its memory layout fixed for its whole lifetime wants no
// allocator activity at all.  This entry point serves them: every temporary it needs comes
// from one file-scope static device array of kStaticScratchBytes, and it runs the same
// backward kernels as dlo_backward with as many resident rod slots as that array holds.
//
// The array is shared by every context on a device, so calls on one device must not
// overlap: two calls in flight at once (from different host threads, or on different
// streams) would overwrite each other's scratch.  Each call synchronises its stream before
// it returns, so calls made one after the other from one thread never overlap.
#include <atomic>
#include <cstdio>

#include "dlo_kernels.h"
#include "dlo_runtime.h"
#include "dlo_vec.cuh"

namespace dlo {
cudaError_t launch_frames_adjoint(const RodInfo* rods, int B, const float4* X0, const float4* gtb0,
                                  const float4* gd1b0, float4* gx0, V3<double>* work, cudaStream_t st);
}
using namespace dlo;

// 256 MiB: enough for the 4096-rod x 128-vertex workload at 50-frame checkpoints (the
// frame-initialisation adjoint takes 67 MB, the rest holds ~170 resident rod slots of 1.1 MB).
static constexpr size_t kStaticScratchBytes = DLO_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch, looked up once per device with that device current.
static constexpr int kMaxDevices = 64;
static std::atomic<void*> g_scratch_ptr[kMaxDevices];

static dlo_status scratch_address(dlo_ctx* c, char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_err(c, DLO_ERR_INVALID_ARG, "device ordinal out of range");
    void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaGetSymbolAddress of the static scratch");
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = reinterpret_cast<char*>(p);
    return DLO_OK;
}

// The per-rod status words, read through a fixed stack buffer (no host allocation).
static dlo_status check_status_noalloc(dlo_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "stream");
    unsigned s[256];
    for (int b0 = 0; b0 < c->B; b0 += 256) {
        const int n = c->B - b0 < 256 ? c->B - b0 : 256;
        e = cudaMemcpy(s, c->d_status + b0, sizeof(unsigned) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(c, e, "status copy");
        for (int i = 0; i < n; ++i) {
            if (s[i] & 1u) return set_err(c, DLO_ERR_NONFINITE, "rod " + std::to_string(b0 + i) + " has a non-finite state");
            if (s[i] & 2u)
                return set_err(c, DLO_ERR_CAPACITY, "rod " + std::to_string(b0 + i) + " overflowed its self-contact pair list");
        }
    }
    return DLO_OK;
}


extern "C" dlo_status dlo_backward_noalloc(dlo_ctx* c, const float* dL_dx_T, const float* dL_dv_T,
                                           const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial,
                                           float* dL_dx0, float* dL_dv0, float* dL_dtheta0) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!c->rec_active || c->rec_done != c->rec_frames || c->rec_frames == 0)
        return set_err(c, DLO_ERR_STATE, "dlo_backward_noalloc needs a completed rollout armed by dlo_begin_rollout");
    for (const void* p : {(const void*)dL_dx_T, (const void*)dL_dv_T, (const void*)dL_dx0, (const void*)dL_dv0})
        if (p && ((uintptr_t)p & 15u)) return set_err(c, DLO_ERR_INVALID_ARG, "float4 arrays must be 16-byte aligned");
    if (c->opt.self_contact && c->opt.n_iter_pbd < 1)
        return set_err(c, DLO_ERR_INVALID_ARG, "self-contact gradients need at least one projection iteration");
    if (c->buckets.size() > (size_t)kNumSizeClasses) return set_err(c, DLO_ERR_INVALID_ARG, "more size classes than expected");
    char* base = nullptr;
    dlo_status st = scratch_address(c, &base);
    if (st != DLO_OK) return st;

    // fixed part: cotangents of the initial reference frames (gtb0, gd1b0) and, when the
    // gradient must reach x0 through the frame initialisation, its FP64 work array
    const bool frames_adj = c->rec_from_set && dL_dx0;
    const size_t fixed_raw = 2 * 16 * (size_t)c->Et + (frames_adj ? 4 * sizeof(V3<double>) * (size_t)c->V : 0);
    const size_t fixed = (fixed_raw + 255) & ~(size_t)255;
    const int force = c->rec_nsub > 0 ? c->rec_nsub : 0;
    size_t slot_b[kNumSizeClasses];
    int warps[kNumSizeClasses], grid[kNumSizeClasses], nsmax[kNumSizeClasses];
    for (size_t k = 0; k < c->buckets.size(); ++k) {
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
                if (size_class(c->rods_h[b].nv) == bk.nv_max) ns = std::max(ns, c->nsub[b]);
        nsmax[k] = ns;
        const size_t NV = bk.nv_max;
        slot_b[k] = 16 * ((size_t)c->ck_every * (5 * NV + 6) +
                          (size_t)ns * ((7 + 2 * kPairsPerVertex) * NV + (size_t)4 * c->opt.n_iter_pbd * NV));
        // reject what cannot run even one rod at a time
        if (fixed + slot_b[k] > kStaticScratchBytes) {
            char msg[256];
            snprintf(msg, sizeof msg,
                     "the backward needs %zu bytes of scratch for one rod of %d vertices plus %zu for the whole "
                     "batch; the static scratch holds %zu (use dlo_backward, or a shorter checkpoint interval)",
                     slot_b[k], bk.nv_max, fixed, kStaticScratchBytes);
            return set_err(c, DLO_ERR_CAPACITY, msg);
        }
        // as many resident rod slots as the array holds, at most the natural persistent grid
        const size_t slots = (kStaticScratchBytes - fixed) / slot_b[k];
        w = (int)std::min<size_t>((size_t)w, slots);
        const long long natural = std::min<long long>((long long)nb * c->sm_count, (bk.n + w - 1) / w);
        grid[k] = (int)std::min<long long>(natural, (long long)(slots / (size_t)w));
        warps[k] = w;
    }
    float4* gtb0 = reinterpret_cast<float4*>(base);
    float4* gd1b0 = gtb0 + c->Et;
    V3<double>* work = reinterpret_cast<V3<double>*>(gd1b0 + c->Et);
    char* scratch = base + fixed;
    // the buckets run one after the other on the stream, each over the whole slot area
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
        P.scratch = scratch;
        P.slot_bytes = slot_b[k];
        P.K = c->ck_every;
        P.nsub_max = nsmax[k];
        P.scene = c->scene;
        // the work-queue head (context memory from dlo_create) must start at zero
        cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = launch_backward(P, bk.nv_max, bk.contact, grid[k], warps[k], c->stream);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "backward launch");
    }
    if (frames_adj) {
        cudaError_t e = launch_frames_adjoint(c->d_rods, c->B, c->ck.X, gtb0, gd1b0,
                                              reinterpret_cast<float4*>(dL_dx0), work, c->stream);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "frames adjoint launch");
    }
    return check_status_noalloc(c);
}
