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
// backward kernels as dlo_backward, on as many rods at a time as that array holds: the rods
// of each size class are reversed in groups, one group after another, each with its own
// chunk records, frame-start states and carried cotangents in the array.
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
    char* base = nullptr;
    dlo_status st = scratch_address(c, &base);
    if (st != DLO_OK) return st;

    // fixed part: cotangents of the initial reference frames (gtb0, gd1b0) and, when the
    // gradient must reach x0 through the frame initialisation, its FP64 work array
    const bool frames_adj = c->rec_from_set && dL_dx0;
    const size_t fixed_raw = 2 * 16 * (size_t)c->Et + (frames_adj ? 4 * sizeof(V3<double>) * (size_t)c->V : 0);
    const size_t fixed = (fixed_raw + 255) & ~(size_t)255;
    const int force = c->rec_nsub > 0 ? c->rec_nsub : 0;
    BwdPlan plan;
    st = bwd_plan(c, force, c->ck_every, plan);
    if (st != DLO_OK) return st;
    const size_t avail = fixed < kStaticScratchBytes ? kStaticScratchBytes - fixed : 0;
    const int K = c->ck_every, F = c->rec_frames;
    float4* gtb0 = reinterpret_cast<float4*>(base);
    float4* gd1b0 = gtb0 + c->Et;
    V3<double>* work = reinterpret_cast<V3<double>*>(gd1b0 + c->Et);
    char* region = base + fixed;
    const BwdParams common = backward_common(c, force, dL_dx_T, dL_dv_T, dL_dtheta_T, dL_dactions, dL_dmaterial,
                                             dL_dx0, dL_dv0, dL_dtheta0, gtb0, gd1b0);
    // the classes one after the other on the stream, each over the whole array
    for (size_t k = 0; k < c->buckets.size(); ++k) {
        const int n = c->buckets[k].n;
        const int want = std::min(n, backward_resident_rods(c, k));
        // frames per chunk: the most (up to 16, a multiple of K from K on) with which the
        // array still holds as many rods as the reverse keeps resident; else one frame
        int C = 1, per_pass = 0;
        size_t r3, l2, cs;
        for (int cand = std::min(16, F); cand >= 1; --cand) {
            if (cand > K && cand % K) continue;
            backward_rod_f4(c, plan, k, cand, r3, l2, cs);
            const int fit = (int)std::min<size_t>((size_t)n, avail / (16 * (r3 + l2 + cs)));
            if (fit >= want || cand == 1) {
                C = cand;
                per_pass = fit;
                break;
            }
        }
        if (per_pass < 1) {
            char msg[256];
            snprintf(msg, sizeof msg,
                     "the backward needs %zu bytes of scratch for one rod of %d vertices plus %zu for the whole "
                     "batch; the static scratch holds %zu (use dlo_backward, or a shorter checkpoint interval)",
                     16 * (r3 + l2 + cs), c->buckets[k].nv_max, fixed, kStaticScratchBytes);
            return set_err(c, DLO_ERR_CAPACITY, msg);
        }
        backward_rod_f4(c, plan, k, C, r3, l2, cs);
        for (int i0 = 0; i0 < n; i0 += per_pass) {
            const int m = std::min(per_pass, n - i0);
            float4* R3 = reinterpret_cast<float4*>(region);
            float4* L2 = R3 + (size_t)m * r3;
            float4* CS = L2 + (size_t)m * l2;
            st = enqueue_backward_class(c, plan, k, c->stream, i0, m, R3, L2, CS, C, common);
            if (st != DLO_OK) return st;
        }
    }
    if (frames_adj) {
        cudaError_t e = launch_frames_adjoint(c->d_rods, c->B, c->ck.X, gtb0, gd1b0,
                                              reinterpret_cast<float4*>(dL_dx0), work, c->stream);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "frames adjoint launch");
    }
    return check_status_noalloc(c);
}
