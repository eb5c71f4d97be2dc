// dlo_runtime.h -- the context object behind the C ABI and the runtime's internal calls.
#pragma once
#include <string>
#include <vector>

#include "dlo.h"
#include "dlo_internal.h"

namespace dlo {
constexpr int kMaxVerts = 256;

// Rods of one shared-memory size class, launched together by the persistent kernels.
struct Bucket {
    int nv_max = 0;
    bool contact = false;
    int n = 0;              // rods in the bucket
    int* d_order = nullptr; // rod ids by decreasing cost (vertices x substeps)
    int warps = 0;          // rods in flight per CTA of the forward kernel
    int grid = 0;           // persistent CTAs
};
}  // namespace dlo

struct dlo_ctx {
    int B = 0;
    long long V = 0, Et = 0;
    cudaStream_t stream = nullptr;
    dlo_allocator alloc{};
    dlo_options opt{};
    dlo::SceneDev scene{};
    std::vector<void*> allocs;
    size_t bytes = 0;
    std::string err;
    std::vector<dlo::RodInfo> rods_h;
    std::vector<int> nsub;
    int sm_count = 0;
    // static device data
    dlo::RodInfo* d_rods = nullptr;
    float4* d_kin = nullptr;
    float2* d_mass = nullptr;
    float2* d_es = nullptr;
    float4* d_rest = nullptr;
    float* d_gp0 = nullptr;
    // live state and diagnostics
    dlo::StateRef S{};
    unsigned* d_status = nullptr;
    double* d_residual = nullptr;
    int* d_npairs = nullptr;
    int* d_counters = nullptr;   // one work-queue head per bucket
    float4* d_reaction = nullptr;  // [V][4] contact impulse slots when opt.reaction
    uint32_t* d_pair_list = nullptr;  // [B][1 + kPairListStride] last frame's candidates (self-contact)
    std::vector<dlo_material> mat_h;  // per-rod material as created (or last set)
    std::vector<double> lmin_h;       // per-rod shortest rest edge
    std::vector<dlo::Bucket> buckets;
    // with several size classes, each class's kernels run on its own stream, forked from and
    // joined back to `stream` with events, so that the classes' tails overlap
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    long long launches = 0;
    bool from_set_state = false;
    // rollout recording for dlo_backward
    bool rec_active = false;
    bool rec_from_set = false;
    int rec_frames = 0, rec_done = 0, rec_nsub = 0;
    int ck_every = 0, ck_count = 0;
    dlo::StateRef ck{};
    void* ck_mem = nullptr;
    size_t ck_bytes = 0;
    float* rec_actions = nullptr;
    size_t rec_bytes = 0;
    // backward workspace
    void* bw_mem = nullptr;
    size_t bw_bytes = 0;
    // plain comparator workspace
    void* pl_mem = nullptr;
    size_t pl_bytes = 0;
    // silhouette loss: per-pixel weights of one camera image per rod
    void* sil_mem = nullptr;
    size_t sil_bytes = 0;
};

// launch shape and workspace size of the backward for a checkpoint interval (dlo_adjoint.cu)
struct BwdPlan {
    std::vector<size_t> slot_b, offset;   // per class: bytes per resident rod, scratch offset
    std::vector<int> warps, grid, nsmax;
    size_t bytes = 0;
};
// the stream of size class k, and the fork / join around work issued on those streams
cudaStream_t class_stream(dlo_ctx* c, size_t k);
cudaError_t fork_classes(dlo_ctx* c);
cudaError_t join_classes(dlo_ctx* c);
dlo_status bwd_plan(dlo_ctx* c, int force, int K, BwdPlan& out);

dlo_status set_err(dlo_ctx* c, dlo_status s, const std::string& msg);
dlo_status cuda_err(dlo_ctx* c, cudaError_t e, const char* where);
dlo_status check_status(dlo_ctx* c);
void* dev_alloc(dlo_ctx* c, size_t bytes);
void dev_free(dlo_ctx* c, void* p);
dlo_status runtime_allocate(dlo_ctx* c, const std::vector<dlo::RodInfo>& rods, const std::vector<float4>& kin,
                            const std::vector<float2>& mass, const std::vector<float2>& es,
                            const std::vector<float4>& rest, const std::vector<float>& gp0,
                            const std::vector<float4>& xr4);
void runtime_release(dlo_ctx* c);
