// dlo_internal.h -- device data layout shared by the C-ABI runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dlo {

enum RodFlags : int {
    ROD_INEXT = 1,       // stretching energy off, edges projected to rest length
    ROD_PLASTIC = 2,     // bending plasticity
    ROD_SLIMIT = 4,      // elastic stretching plus strain-limit projection
    ROD_SELF = 8,        // self-contact on
    ROD_CLOSED = 16,
    ROD_HASH = 32,       // self-contact candidates through the per-rod spatial hash
    ROD_STRANDS = 64     // several DLOs of one environment back to back; the edge between two
                         // of them ("break") has rest length 0 and carries no force (see below)
};

// An environment of several DLOs is one record whose vertices are the DLOs' vertices back to
// back ("strands", open only).  The edge that joins the last vertex of one strand to the
// first of the next is no part of the model: its rest length (ES.x, ET.w) is 0, its inverse
// axial inertia 0, it keeps the frame it was given (tangent z, d1 = x), it is no segment for
// self-contact, and the hinges at its two ends are inactive.  Everything else, self-contact
// between strands included, is the single-rod code path.

// One rod: offsets into the packed arrays and its per-rod constants (64 bytes).
struct RodInfo {
    int v0, nv, e0, ne;        // first vertex / edge, counts
    int nsub, flags, ngrip, excl;
    float h, kA, Bm, beta;     // substep, K A, E A r^2 / 4, G A r^2 / 2
    float sy, rc, cd, radius;  // yield curvature, creep rate, damping, radius
    float slim, contact_d, rsv, eps;    // strain limit, candidate distance, (reserved), eps_s
    int pair_cap, pair_off, pad0, pad1;
};

// Stride of the per-rod candidate list read back by DLO_Q_PAIR_LIST: 4 pairs per vertex of
// the largest size class (256 vertices).
constexpr int kPairListStride = 1024;

constexpr int kMaxPlanes = 4;
constexpr int kMaxBoxes = 4;

struct SceneDev {
    int n_planes, n_boxes, n_iter, self_contact;
    float4 planes[kMaxPlanes];     // (n, offset)
    float4 box_c[kMaxBoxes];       // centre
    float4 box_h[kMaxBoxes];       // half extents
    float grip_r, grip_hl, gravity, dt;
    float mu_self, mu_rigid, restitution, pad;
};

// State arrays of one snapshot (live state, or one checkpoint of the ring).
struct StateRef {
    float4* X;    // [V]    position, inverse mass
    float4* Vl;   // [V]    velocity, twist rate of edge starting here
    float4* ED;   // [Etot] reference d1 (base), theta
    float4* ET;   // [Etot] tangent the base frame is adapted to, unused
    float4* HG;   // [V]    rest curvature (2), rest twist, reference twist (hinge at vertex)
    float* GP;    // [B][2][12] gripper position + rotation (row major)
};

struct FwdParams {
    const RodInfo* rods;
    const int* order;         // rods in decreasing cost
    int n_order;
    int* counter;             // work queue head (zeroed before the launch)
    StateRef S;
    const float4* KIN;        // [V] grasp offset (xyz), kind (0 free, 1 pinned, 2/3 gripper)
    const float2* ES;         // [Etot] rest length, 1 / axial inertia
    const float* actions;     // [frames][B][2][6] or null
    float* xframes;           // [frames][V][4] or null
    int frames, B, force_nsub, frame0;
    long long nvert_total;
    // checkpoint ring: snapshot c holds the state at the start of rollout frame c * ck_every
    StateRef ck;
    long long ck_strideV, ck_strideE, ck_strideB;
    int ck_every, ck_count;
    unsigned* status;         // [B] bit 1 non-finite, bit 2 pair overflow, bit 4 moved past the margin
    double* residual;         // [B]
    int* npairs;              // [B]
    uint32_t* pair_list;      // [B][1 + kPairListStride]: the last frame's candidates (count, pairs) or null
    float4* reaction;         // [V][4] contact impulse slots (planes, boxes, gripper 0, 1) or null
    SceneDev scene;
};

struct BwdParams {
    const RodInfo* rods;
    const int* order;         // rods of the size class in decreasing cost
    int item0, n_items;       // this launch processes order[item0 .. item0 + n_items)
    int* counter;             // work-queue head (zeroed before each launch)
    StateRef ck;
    long long ck_strideV, ck_strideE, ck_strideB;
    int ck_every, ck_count;
    const float4* KIN;
    const float2* ES;
    const float* actions;     // recorded [F][B][12]
    int frames, B, force_nsub, nsub_max;
    int fa, fb;               // the chunk of frames [fa, fb) of this launch
    int mode;                 // recompute: 0 = the segment's frame-start states, 1 = the chunk's records
    int first_chunk, last_chunk;  // reverse: fb is the last frame / fa is frame 0
    float4* L2;               // [n_items][K][5 NV + 6] frame-start states of the current segment
    float4* R3;               // [n_items][fb - fa][frame record] the chunk's records
    float4* CS;               // [n_items][5 NV + 6] cotangent state carried between chunks
    size_t l2_rod, r3_rod, cs_rod;   // float4 per item of L2, R3, CS
    const float4* dLdx;       // [V] or null
    const float4* dLdv;       // [V] or null
    const float* dLdth;       // [Etot] or null
    float* gact;              // [F][B][12] or null
    float* gmat;              // [B][5] or null
    float4* gx0;              // [V] or null
    float4* gv0;              // [V] or null
    float* gth0;              // [Etot] or null
    float4* gtb0;             // [Etot] cotangent of the initial base tangents
    float4* gd1b0;            // [Etot] cotangent of the initial base d1
    unsigned* status;         // [B] status bits (debug builds: bit 8, a failed bounds check)
    SceneDev scene;
};

}  // namespace dlo
