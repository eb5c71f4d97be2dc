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
    size_t rec_budget = 0;   // chunk-record bytes the backward may use (set by dlo_begin_rollout)
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

// launch shapes and workspace of the chunked backward for a checkpoint interval (dlo_adjoint.cu)
struct BwdPlan {
    // per size class: substeps reserved per frame, frames per chunk, float4 per rod of the
    // chunk records (R3), of the segment's frame-start states (L2, empty when chunks start at
    // checkpoints) and of the carried cotangent state (CS); the class's region in the workspace
    std::vector<int> nsmax, C;
    std::vector<size_t> r3_rod, l2_rod, cs_rod, offset;
    size_t fixed = 0;    // initial-frame cotangents and the frame-initialisation adjoint's work
    size_t bytes = 0;    // everything, for all rods at once
};
// the stream of size class k, and the fork / join around work issued on those streams
cudaStream_t class_stream(dlo_ctx* c, size_t k);
cudaError_t fork_classes(dlo_ctx* c);
cudaError_t join_classes(dlo_ctx* c);
// rec_budget: bytes allowed for the chunk records of all classes (0 = the default)
dlo_status bwd_plan(dlo_ctx* c, int force, int K, BwdPlan& out, size_t rec_budget = 0);
// Enqueue the backward of size class k for the rods order[item0 .. item0 + n) on stream st,
// with that class's R3 / L2 / CS buffers sized for n rods; common holds the outputs and inputs.
dlo_status enqueue_backward_class(dlo_ctx* c, const BwdPlan& plan, size_t k, cudaStream_t st, int item0, int n,
                                  float4* R3, float4* L2, float4* CS, int C, const dlo::BwdParams& common);
// the launch inputs and outputs shared by every kernel of one backward
dlo::BwdParams backward_common(dlo_ctx* c, int force, const float* dL_dx_T, const float* dL_dv_T,
                               const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial, float* dL_dx0,
                               float* dL_dv0, float* dL_dtheta0, float4* gtb0, float4* gd1b0);
// float4 per rod of size class k with C frames per chunk: chunk records, segment frame-start
// states, carried cotangents; and the rods the reverse kernel keeps resident on the device
void backward_rod_f4(dlo_ctx* c, const BwdPlan& plan, size_t k, int C, size_t& r3, size_t& l2, size_t& cs);
int backward_resident_rods(dlo_ctx* c, size_t k);


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
