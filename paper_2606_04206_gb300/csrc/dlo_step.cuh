// dlo_step.cuh -- one rod's frame and substep on one thread group, state in shared memory.
//
// Shared by the forward kernel and the backward kernel's recomputations.  Per substep
// (DLO-Lab Sec. 3.1 / 3.2 / App. A.1):
//   edge phase    each edge's reference frame by time-parallel transport and its material frame
//   hinge phase   curvature and twist, bending plasticity on the rest curvature, and the
//                 hinge's energy gradient back to its two edges' frames
//   edge phase    each edge's frame reversed once on the sum of its two hinges' seeds
//   vertex phase  gradient gather + stretching, gravity, damping, symplectic-Euler velocity,
//                 soft SDF contact (planes, boxes, capsule grippers), displacement predict,
//                 kinematic vertices, new reference-frame base
//   PBD phase     N_C x (red-black inextensibility / strain limit, Jacobi self-collision)
//   velocity      v = d/h, self-contact Coulomb friction, positions x + d
// Per frame: self-contact candidates (every edge pair behind a bounding-sphere filter),
// gripper pose update.
#pragma once
#include <type_traits>
#include "dlo_internal.h"
#include "dlo_kernels.h"
#include "dlo_physics.cuh"

namespace dlo {

// The per-rod constants as the persistent kernels hold them: a copy in registers, or (C) a
// reference to the record in global memory, read where used.
template <bool C>
using RodRef = typename std::conditional<C, const RodInfo&, const RodInfo>::type;

// A rod is stepped by a group of TPR threads (one or more whole warps); elements are spread
// over the group with stride TPR and phases are separated by the group's barrier (the warp's
// own for TPR = 32, else a named barrier of TPR threads).
template <int TPR>
struct Grp {
    int tid;      // thread index within the rod's group
    int bar;      // named barrier id (1..15) of the group
    float* red;   // 64 floats of the rod's shared header, for group reductions
    __device__ __forceinline__ void sync() const {
        if (TPR == 32)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TPR) : "memory");
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the group (deterministic order: warps' partial sums added in warp order).
template <int TPR>
__device__ __forceinline__ double grp_sum(double v, const Grp<TPR>& g) {
    v = warp_sum(v);
    if (TPR == 32) return v;
    double* r = reinterpret_cast<double*>(g.red);
    if ((g.tid & 31) == 0) r[g.tid >> 5] = v;
    g.sync();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < TPR / 32; ++k) s += r[k];
    g.sync();
    return s;
}

template <int TPR>
__device__ __forceinline__ bool grp_any(bool p, const Grp<TPR>& g) {
    const bool w = __any_sync(0xffffffffu, p);
    if (TPR == 32) return w;
    int* r = reinterpret_cast<int*>(g.red) + 32;
    if ((g.tid & 31) == 0) r[g.tid >> 5] = w ? 1 : 0;
    g.sync();
    bool s = false;
#pragma unroll
    for (int k = 0; k < TPR / 32; ++k) s |= r[k] != 0;
    g.sync();
    return s;
}

// Bitwise OR over the group.
template <int TPR>
__device__ __forceinline__ unsigned grp_or(unsigned v, const Grp<TPR>& g) {
    const unsigned w = __reduce_or_sync(0xffffffffu, v);
    if (TPR == 32) return w;
    unsigned* r = reinterpret_cast<unsigned*>(g.red) + 56;
    if ((g.tid & 31) == 0) r[g.tid >> 5] = w;
    g.sync();
    unsigned s = 0u;
#pragma unroll
    for (int k = 0; k < TPR / 32; ++k) s |= r[k];
    g.sync();
    return s;
}

// Largest value over the group (non-negative floats: their bit patterns order like the values).
template <int TPR>
__device__ __forceinline__ float grp_max_nonneg(float v, const Grp<TPR>& g) {
    const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (TPR == 32) return __uint_as_float(w);
    unsigned* r = reinterpret_cast<unsigned*>(g.red) + 60;
    if ((g.tid & 31) == 0) r[g.tid >> 5] = w;
    g.sync();
    unsigned m = 0u;
#pragma unroll
    for (int k = 0; k < TPR / 32; ++k) m = max(m, r[k]);
    g.sync();
    return __uint_as_float(m);
}

// Status bit of a failed bounds check.  Debug builds (-DDLO_DEBUG_BOUNDS) check every index
// the kernels take from data (candidate pairs, kinematic kinds, recorded pair counts, work-
// queue items) before using it: a failed check sets the bit in the rod's flag word (slot 40
// of its reduction scratch, folded into the rod's status when its work ends) and the access
// is skipped.  Release builds compile the checks away.
constexpr unsigned kStatusBounds = 8u;

__device__ __forceinline__ bool in_bounds(bool ok, float* red) {
#ifdef DLO_DEBUG_BOUNDS
    if (!ok) atomicOr(reinterpret_cast<unsigned*>(red) + 40, kStatusBounds);
    return ok;
#else
    (void)ok;
    (void)red;
    return true;
#endif
}

// Start of a rod's work: clear its flag word (debug builds).
template <int TPR>
__device__ __forceinline__ void bounds_begin(const Grp<TPR>& g) {
#ifdef DLO_DEBUG_BOUNDS
    if (g.tid == 0) reinterpret_cast<unsigned*>(g.red)[40] = 0u;
#else
    (void)g;
#endif
}

// End of a rod's work, after a group barrier: fold its flag word into status[rod].
template <int TPR>
__device__ __forceinline__ void bounds_end(const Grp<TPR>& g, unsigned* status, int rod) {
#ifdef DLO_DEBUG_BOUNDS
    if (g.tid == 0 && status) {
        const unsigned f = reinterpret_cast<unsigned*>(g.red)[40];
        if (f) atomicOr(&status[rod], f);
    }
#else
    (void)g;
    (void)status;
    (void)rod;
#endif
}

// Value held by thread 0 of the group.
template <int TPR>
__device__ __forceinline__ int grp_bcast0(int v, const Grp<TPR>& g) {
    if (TPR == 32) return __shfl_sync(0xffffffffu, v, 0);
    int* r = reinterpret_cast<int*>(g.red) + 48;
    if (g.tid == 0) *r = v;
    g.sync();
    const int out = *r;
    g.sync();
    return out;
}

// Exclusive prefix sum over the group.
template <int TPR>
__device__ __forceinline__ int grp_excl_scan(int v, const Grp<TPR>& g) {
    const int l = g.tid & 31, w = g.tid >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += y;
    }
    if (TPR == 32) return incl - v;
    int* r = reinterpret_cast<int*>(g.red) + 16;
    if (l == 31) r[w] = incl;
    g.sync();
    int off = 0;
    for (int k = 0; k < w; ++k) off += r[k];
    g.sync();
    return off + incl - v;
}

// Optional recording of a substep's intermediates for the adjoint (rec != nullptr): all in
// global memory, one record per substep of the frames being reversed.
struct Rec {
    float4* v1;     // [NV]: velocity after the force update, before rigid contact
    float4* dfin;   // [NV]: displacement after the PBD iterations, before friction
    float4* pbd;    // [n_iter][NV]: per edge, the unit direction and target / length of its
                    // inextensibility or strain-limit projection, (0, 0, 0, 1) where it did nothing
    float4* csnap;  // [n_iter][NV]: displacements before each self-contact sweep (frames with candidates)
    float4* fr0;    // [pair capacity]: first-iteration projection data of each pair
    float4* fr1;
    int nvmax;
};

constexpr float kFixPos = 1073741824.f;     // 2^30: fixed-point scale of position corrections
constexpr float kFixVel = 16777216.f;       // 2^24: fixed-point scale of velocity corrections

__device__ __forceinline__ int to_fix(float v, float scale) {
    float q = v * scale;
    q = fminf(fmaxf(q, -2147483520.f), 2147483520.f);
    return __float2int_rn(q);
}

// Impulse m (v_after - v_before) that one contact response gave the vertex, added to its slot.
__device__ __forceinline__ void add_impulse(float4* slot, float m, V3<float> vb, V3<float> va) {
    float4 a = *slot;
    *slot = make_float4(a.x + m * (va.x - vb.x), a.y + m * (va.y - vb.y), a.z + m * (va.z - vb.z), 0.f);
}

// Rigid contact of one vertex against the scene and the rod's grippers (Sec. 3.2).
// sp: the substep's gripper block (see Smem).  imp (optional): the vertex's four impulse
// slots (planes, boxes, gripper 0, gripper 1), to which each active response adds the
// impulse it gave the vertex of mass m; the rigid body receives the opposite.
__device__ __forceinline__ V3<float> rigid_contact(const SceneDev& sc, const RodInfo& R, V3<float> x,
                                                    V3<float> v, const float* sp, float4* imp = nullptr,
                                                    float m = 0.f) {
    bool on;
    for (int k = 0; k < sc.n_planes; ++k) {
        V3<float> n = f3(sc.planes[k]);
        float sdf = dot(x, n) - sc.planes[k].w;
        const V3<float> vb = v;
        v = contact_respond(v, sdf, n, zf3(), R.radius, R.eps, sc.mu_rigid, sc.restitution, on);
        if (imp && on) add_impulse(imp, m, vb, v);
    }
    for (int k = 0; k < sc.n_boxes; ++k) {
        V3<float> n;
        float sdf = sdf_box(x, f3(sc.box_c[k]), f3(sc.box_h[k]), n);
        const V3<float> vb = v;
        v = contact_respond(v, sdf, n, zf3(), R.radius, R.eps, sc.mu_rigid, sc.restitution, on);
        if (imp && on) add_impulse(imp + 1, m, vb, v);
    }
    for (int g = 0; g < R.ngrip; ++g) {
        const float* o = sp + 32 * g;
        V3<float> p = f3(o[0], o[1], o[2]);
        V3<float> ax = f3(o[8], o[11], o[14]);   // column 2 of R0: the capsule axis
        V3<float> a = p - sc.grip_hl * ax, b = p + sc.grip_hl * ax, n;
        if (capsule_far(x, a, b, sc.grip_r + R.radius + kContactReach * R.eps)) continue;
        float sdf = sdf_capsule(x, a, b, sc.grip_r, n);
        if (sdf > R.radius + kContactReach * R.eps) continue;
        V3<float> vp = f3(o[24], o[25], o[26]);
        V3<float> w = f3(o[27], o[28], o[29]);
        V3<float> vrig = vp + cross(w, x - p);
        const V3<float> vb = v;
        v = contact_respond(v, sdf, n, vrig, R.radius, R.eps, sc.mu_rigid, sc.restitution, on);
        if (imp && on) add_impulse(imp + 2 + g, m, vb, v);
    }
    return v;
}

template <int NV, bool CONTACT>
struct Smem {
    float4 *X, *X0, *V, *ED, *ET, *HG, *HB0, *HB1, *HB2, *ND;
    float4 *fr0, *fr1;
    int4* acc;
    uint32_t* pairs;
    float* red;
    // gripper block (read by every thread of the rod with broadcasts):
    //   fp  [24] pose at the start of the frame being stepped, per gripper p (3), R (9) row major
    //   f0  [24] a second frame-start pose (the frame the backward reverses)
    //   sp  [64] the current substep, per gripper (32): p0 (3), p1 (3), R0 (9), R1 (9), vp (3), w (3)
    //   act [12] the frame's actions
    float *fp, *f0, *sp, *act;
    __device__ Smem(float4* base) {
        red = reinterpret_cast<float*>(base + warp_smem_bytes(NV, CONTACT) / 16);
        fp = red + 64;
        f0 = fp + 24;
        sp = f0 + 24;
        act = sp + 64;
        X = base;
        X0 = base + NV;
        V = base + 2 * NV;
        ED = base + 3 * NV;
        ET = base + 4 * NV;
        HG = base + 5 * NV;
        HB0 = base + 6 * NV;
        HB1 = base + 7 * NV;
        HB2 = base + 8 * NV;
        ND = base + 9 * NV;
        fr0 = base + 10 * NV;
        fr1 = fr0 + kPairsPerVertex * NV;
        acc = reinterpret_cast<int4*>(fr1 + kPairsPerVertex * NV);
        pairs = reinterpret_cast<uint32_t*>(acc + NV);
    }
};

// ------------------------------------------------------------------ broad phase
// Whether an edge strictly between edges a < b is a break edge (rest length 0): a and b then
// lie on different strands, and the exclusion window does not apply to them.
__device__ __forceinline__ bool break_between(const float4* ET, int a, int b) {
    for (int k = a + 1; k < b; ++k)
        if (!(ET[k].w > 0.f)) return true;
    return false;
}

constexpr int kBpBlock = 8;   // edges per block of the broad phase's first level

// Candidates of one rod: the edge pairs outside the exclusion window whose segments are
// closer than R.contact_d.  A rod has at most 256 edges, so every pair is considered, in two
// levels of exact bounding-sphere tests before the closest-point distance:
//   - each block of kBpBlock consecutive edges lies in the sphere around the centre of its
//     vertices' bounding box, with the distance to its farthest vertex as radius;
//   - each edge's segment lies in the sphere around its midpoint with its half length.
// A segment distance below contact_d implies both sphere distances are below contact_d plus
// the radii.  Level 1 tests every pair of blocks (one pair per thread) and lists the near
// ones; level 2 spreads the edge pairs of the listed block pairs over the group, one edge
// pair per thread, and runs the edge-sphere test, the exclusion window and the exact
// distance.  Found pairs are appended with a shared-memory atomic (rare), so their order
// varies; every use of the list (the Jacobi projection and friction, summed in fixed point,
// the records of the backward's recompute, the pair-list query) is independent of it.
template <int NV, bool CONTACT, int TPR>
__device__ int broad_phase(const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, bool closed, bool& overflow) {
    float4* mid = s.HB0;                          // midpoint, half length of each edge (-1: a break edge)
    int* cnt = reinterpret_cast<int*>(s.HB1);     // [0] pairs found, [1] near block pairs
    uint32_t* nearb = reinterpret_cast<uint32_t*>(s.HB1) + 4;   // near block pairs kA | kB << 16, kA <= kB
    float4* blk = s.HB2;                          // centre, radius of each block of edges
    static_assert((NV / kBpBlock + 1) * (NV / kBpBlock + 2) / 2 + 4 <= 4 * NV, "block pairs fit in HB1");
    const int ne = R.ne, nv = R.nv;
    const bool strands = R.flags & ROD_STRANDS;
    for (int j = g.tid; j < ne; j += TPR) {
        const int j1 = (j + 1 == nv) ? 0 : j + 1;
        const V3<float> p0 = f3(s.X[j]), p1 = f3(s.X[j1]);
        const V3<float> e = p1 - p0;
        mid[j] = (strands && !(s.ET[j].w > 0.f)) ? make_float4(0.f, 0.f, 0.f, -1.f)
                                                 : f4(0.5f * (p0 + p1), 0.5f * sqrtf(dot(e, e)));
    }
    const int nblk = (ne + kBpBlock - 1) / kBpBlock;
    for (int k = g.tid; k < nblk; k += TPR) {
        // the vertices of edges k*B .. min(ne, (k+1)*B) - 1 (a loop's last edge ends at vertex 0)
        const int v0 = k * kBpBlock, v1 = min(ne, v0 + kBpBlock);
        V3<float> lo = f3(s.X[v0]), hi = lo;
        for (int v = v0 + 1; v <= v1; ++v) {
            const V3<float> x = f3(s.X[v == nv ? 0 : v]);
            lo = f3(fminf(lo.x, x.x), fminf(lo.y, x.y), fminf(lo.z, x.z));
            hi = f3(fmaxf(hi.x, x.x), fmaxf(hi.y, x.y), fmaxf(hi.z, x.z));
        }
        const V3<float> c = 0.5f * (lo + hi);
        float r2 = 0.f;
        for (int v = v0; v <= v1; ++v) {
            const V3<float> d = f3(s.X[v == nv ? 0 : v]) - c;
            r2 = fmaxf(r2, dot(d, d));
        }
        blk[k] = f4(c, sqrtf(r2));
    }
    if (g.tid == 0) {
        cnt[0] = 0;
        cnt[1] = 0;
    }
    g.sync();
    const float cd = R.contact_d;
    // level 1: pairs of blocks
    for (int q = g.tid; q < nblk * nblk; q += TPR) {
        const int ka = q / nblk, kb = q - ka * nblk;
        if (kb < ka) continue;
        const float4 A = blk[ka], B = blk[kb];
        const float dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
        const float rr = (cd + A.w + B.w) * 1.0001f;
        if (dx * dx + dy * dy + dz * dz < rr * rr) nearb[atomicAdd(&cnt[1], 1)] = (uint32_t)ka | ((uint32_t)kb << 16);
    }
    g.sync();
    // level 2: the edge pairs of the near block pairs
    const int nn = cnt[1], cap = R.pair_cap;
    bool ovf = false;
    constexpr int BB = kBpBlock * kBpBlock;
    for (int t = g.tid; t < nn * BB; t += TPR) {
        const uint32_t bp = nearb[t / BB];
        const int a = (int)(bp & 0xffffu) * kBpBlock + (t % BB) / kBpBlock;
        const int b = (int)(bp >> 16) * kBpBlock + t % kBpBlock;
        if (b <= a || b >= ne) continue;
        const float4 ma = mid[a], mb = mid[b];
        if (!(ma.w >= 0.f && mb.w >= 0.f)) continue;
        const float dx = ma.x - mb.x, dy = ma.y - mb.y, dz = ma.z - mb.z;
        const float rr = (cd + ma.w + mb.w) * 1.00001f;
        if (!(dx * dx + dy * dy + dz * dz < rr * rr)) continue;
        int sep = b - a;
        if (closed) sep = min(sep, ne - sep);
        if (!(sep > R.excl || (strands && break_between(s.ET, a, b)))) continue;
        const int a1 = (a + 1 == nv) ? 0 : a + 1, b1 = (b + 1 == nv) ? 0 : b + 1;
        const V3<float> pa0 = f3(s.X[a]), pa1 = f3(s.X[a1]), pb0 = f3(s.X[b]), pb1 = f3(s.X[b1]);
        float su, uu;
        closest_params(pa0, pa1, pb0, pb1, su, uu);
        const V3<float> dd = (pa0 + su * (pa1 - pa0)) - (pb0 + uu * (pb1 - pb0));
        if (!(sqrtf(dot(dd, dd)) < cd)) continue;
        const int idx = atomicAdd(&cnt[0], 1);
        if (idx < cap)
            s.pairs[idx] = (uint32_t)a | ((uint32_t)b << 16);
        else
            ovf = true;
    }
    g.sync();
    overflow = grp_any<TPR>(ovf, g);
    const int np = cnt[0];
    g.sync();
    return min(np, cap);
}

__device__ __forceinline__ unsigned cell_hash(int ix, int iy, int iz, int mask) {
    return ((unsigned)ix * 73856093u ^ (unsigned)iy * 19349663u ^ (unsigned)iz * 83492791u) & (unsigned)mask;
}

// The same candidates found through a per-rod spatial hash of the edge midpoints (the option
// ROD_HASH).  Cells are the candidate distance plus the frame's longest edge, so that the 27
// cells around an edge's cell hold every edge whose segment can come within the candidate
// distance of it (two midpoints are at most that far apart then).  Midpoints are counting-
// sorted into a table of buckets in shared memory (HB0 and HB1, free at this point); each
// edge then tests the edges of its 27 neighbouring cells.
template <int NV, bool CONTACT, int TPR>
__device__ int broad_phase_hash(const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, bool closed,
                                bool& overflow) {
    constexpr int TBL = NV <= 32 ? 64 : (NV <= 64 ? 128 : (NV <= 128 ? 256 : 512));
    static_assert(2 * NV + TBL + 1 <= 8 * NV, "the hash table fits in HB0 and HB1");
    int* keys = reinterpret_cast<int*>(s.HB0);
    int* cnt = keys + NV;            // TBL bucket counters, then the pair counter
    int* sorted = cnt + TBL + 1;
    const int ne = R.ne, nv = R.nv;
    const bool strands = R.flags & ROD_STRANDS;
    auto real = [&](int j) { return !strands || s.ET[j].w > 0.f; };   // break edges are no segments
    float lmax = 0.f;
    for (int j = g.tid; j < ne; j += TPR) {
        if (!real(j)) continue;
        const int j1 = (j + 1 == nv) ? 0 : j + 1;
        const V3<float> e = f3(s.X[j1]) - f3(s.X[j]);
        lmax = fmaxf(lmax, sqrtf(dot(e, e)));
    }
    for (int k = g.tid; k <= TBL; k += TPR) cnt[k] = 0;
    lmax = grp_max_nonneg<TPR>(lmax, g);
    const float inv_cell = 1.f / (R.contact_d + lmax);
    const V3<float> org = f3(s.X[0]);
    for (int j = g.tid; j < ne; j += TPR) {
        if (!real(j)) continue;
        const int j1 = (j + 1 == nv) ? 0 : j + 1;
        const V3<float> m = 0.5f * (f3(s.X[j]) + f3(s.X[j1])) - org;
        const int ix = min(max(__float2int_rd(m.x * inv_cell), -510), 510) + 512;
        const int iy = min(max(__float2int_rd(m.y * inv_cell), -510), 510) + 512;
        const int iz = min(max(__float2int_rd(m.z * inv_cell), -510), 510) + 512;
        keys[j] = (ix << 20) | (iy << 10) | iz;
        atomicAdd(&cnt[cell_hash(ix, iy, iz, TBL - 1)], 1);
    }
    g.sync();
    {   // exclusive scan of the bucket counts, TBL / TPR consecutive buckets per thread
        constexpr int PER = TBL / TPR;
        int loc[PER];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            loc[k] = cnt[g.tid * PER + k];
            sum += loc[k];
        }
        int run = grp_excl_scan<TPR>(sum, g);
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            cnt[g.tid * PER + k] = run;
            run += loc[k];
        }
    }
    g.sync();
    for (int j = g.tid; j < ne; j += TPR) {
        if (!real(j)) continue;
        const int key = keys[j];
        const int pos = atomicAdd(&cnt[cell_hash(key >> 20, (key >> 10) & 1023, key & 1023, TBL - 1)], 1);
        sorted[pos] = j;
    }
    g.sync();
    // after the scatter cnt[h] is the end of bucket h (and the start of bucket h + 1)
    const int cap = R.pair_cap;
    const float cd = R.contact_d;
    bool ovf = false;
    for (int a = g.tid; a < ne; a += TPR) {
        if (!real(a)) continue;
        const int key = keys[a];
        const int ix = key >> 20, iy = (key >> 10) & 1023, iz = key & 1023;
        const int a1 = (a + 1 == nv) ? 0 : a + 1;
        const V3<float> pa0 = f3(s.X[a]), pa1 = f3(s.X[a1]);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int cx = ix + dx, cy = iy + dy, cz = iz + dz;
                    const int nk = (cx << 20) | (cy << 10) | cz;
                    const unsigned hh = cell_hash(cx, cy, cz, TBL - 1);
                    const int beg = hh ? cnt[hh - 1] : 0, end = cnt[hh];
                    for (int q = beg; q < end; ++q) {
                        const int b = sorted[q];
                        if (b <= a || keys[b] != nk) continue;
                        int sep = b - a;
                        if (closed) sep = min(sep, ne - sep);
                        if (sep <= R.excl && !(strands && break_between(s.ET, a, b))) continue;
                        const int b1 = (b + 1 == nv) ? 0 : b + 1;
                        const V3<float> pb0 = f3(s.X[b]), pb1 = f3(s.X[b1]);
                        float su, uu;
                        closest_params(pa0, pa1, pb0, pb1, su, uu);
                        const V3<float> dd = (pa0 + su * (pa1 - pa0)) - (pb0 + uu * (pb1 - pb0));
                        if (!(sqrtf(dot(dd, dd)) < cd)) continue;
                        const int idx = atomicAdd(&cnt[TBL], 1);
                        if (idx < cap)
                            s.pairs[idx] = (uint32_t)a | ((uint32_t)b << 16);
                        else
                            ovf = true;
                    }
                }
    }
    g.sync();
    overflow = grp_any<TPR>(ovf, g);
    const int np = cnt[TBL];
    g.sync();
    return min(np, cap);
}

// ------------------------------------------------------------------ PBD pieces
// Edges first, first+2, ... < last of one colour of the red-black inextensibility sweep.
__device__ __forceinline__ void color_range(int ne, bool closed, int color, int& first, int& last) {
    const bool three = closed && (ne & 1);
    if (color == 2) {
        first = ne - 1;
        last = ne;
    } else {
        first = color;
        last = (color == 0 && three) ? ne - 1 : ne;
    }
}

// One colour of inextensibility / strain-limit projections (App. A.1) on displacements D
// from start positions X0: C = |x_{j+1} - x_j| - |ebar|, lambda = C / (w_j + w_{j+1}).
// prec (optional): receives each edge's projection record (see Rec::pbd).
template <int TPR>
__device__ __forceinline__ void inext_color_arr(const RodInfo& R, const float4* X0, float4* D, const float4* ET,
                                                const Grp<TPR>& g, int color, bool closed, float4* prec = nullptr) {
    const int ne = R.ne, nv = R.nv;
    int first, last;
    color_range(ne, closed, color, first, last);
    const bool inext = R.flags & ROD_INEXT;
    for (int j = first + 2 * g.tid; j < last; j += 2 * TPR) {
        int j1 = (j + 1 == nv) ? 0 : j + 1;
        float4 A = D[j], B = D[j1];              // displacements (w = inverse mass)
        V3<float> e = (f3(X0[j1]) - f3(X0[j])) + (f3(B) - f3(A));
        float ell, ie;
        len_inv(e, ell, ie);
        float eb = ET[j].w;
        float target;
        bool active;
        if (inext) {
            target = eb;
            active = true;
        } else {
            float hi = (1.f + R.slim) * eb, lo = (1.f - R.slim) * eb;
            active = (ell > hi) || (ell < lo);
            target = ell > hi ? hi : lo;
        }
        float ws = A.w + B.w;
        if (!active || !(ws > 0.f) || !(eb > 0.f)) {   // eb = 0: the edge between two strands
            if (prec) prec[j] = make_float4(0.f, 0.f, 0.f, 1.f);
            continue;
        }
        float lam = (ell - target) / ws;
        V3<float> t = ie * e;
        if (prec) prec[j] = f4(t, target * ie);
        V3<float> da = (lam * A.w) * t, db = (lam * B.w) * t;
        D[j] = make_float4(A.x + da.x, A.y + da.y, A.z + da.z, A.w);
        D[j1] = make_float4(B.x - db.x, B.y - db.y, B.z - db.z, B.w);
    }
    g.sync();
}

template <int NV, bool CONTACT, int TPR>
__device__ __forceinline__ void inext_color(const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, int color,
                                            bool closed, float4* prec = nullptr) {
    inext_color_arr<TPR>(R, s.X0, s.X, s.ET, g, color, closed, prec);
}

template <int NV, bool CONTACT, int TPR>
__device__ __forceinline__ void contact_sweep(const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, int np,
                                              bool first) {
    const int nv = R.nv;   // s.acc is zero on entry and is left zero
    const float rsum = 2.f * R.radius;
    for (int p = g.tid; p < np; p += TPR) {
        uint32_t pr = s.pairs[p];
        int a0 = pr & 0xffff, c0 = pr >> 16;
        if (!in_bounds(a0 < nv && c0 < nv && p < R.pair_cap, s.red)) continue;
        int a1 = (a0 + 1 == nv) ? 0 : a0 + 1, c1 = (c0 + 1 == nv) ? 0 : c0 + 1;
        // current positions in coordinates local to the start position of vertex a0
        const V3<float> o = f3(s.X0[a0]);
        float4 A0 = s.X[a0], A1 = s.X[a1], C0 = s.X[c0], C1 = s.X[c1];
        V3<float> pa0 = f3(A0), pa1 = (f3(s.X0[a1]) - o) + f3(A1);
        V3<float> pc0 = (f3(s.X0[c0]) - o) + f3(C0), pc1 = (f3(s.X0[c1]) - o) + f3(C1);
        V3<float> dx[4], n;
        float su, uu, d, W;
        bool on = pair_correction(pa0, pa1, pc0, pc1, A0.w, A1.w, C0.w, C1.w, rsum, dx, su, uu, n, d, W);
        if (first) {
            s.fr0[p] = f4(on ? n : zf3(), on ? d : 0.f);
            s.fr1[p] = make_float4(su, uu, W, on ? 1.f : 0.f);
        }
        if (on) {
            const int idx[4] = {a0, a1, c0, c1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                atomicAdd(&s.acc[idx[k]].x, to_fix(dx[k].x, kFixPos));
                atomicAdd(&s.acc[idx[k]].y, to_fix(dx[k].y, kFixPos));
                atomicAdd(&s.acc[idx[k]].z, to_fix(dx[k].z, kFixPos));
            }
        }
    }
    g.sync();
    for (int i = g.tid; i < nv; i += TPR) {
        int4 q = s.acc[i];
        if (q.x | q.y | q.z) {
            float4 x = s.X[i];
            const float inv = 1.f / kFixPos;
            s.X[i] = make_float4(x.x + q.x * inv, x.y + q.y * inv, x.z + q.z * inv, x.w);
            s.acc[i] = make_int4(0, 0, 0, 0);
        }
    }
    g.sync();
}

template <int NV, bool CONTACT, int TPR>
__device__ __forceinline__ void self_friction(const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, int np,
                                              float h, float mu) {
    const int nv = R.nv;   // s.acc is zero on entry and is left zero
    for (int p = g.tid; p < np; p += TPR) {
        float4 F1 = s.fr1[p];
        if (!(F1.w > 0.f)) continue;
        float4 F0 = s.fr0[p];
        uint32_t pr = s.pairs[p];
        int a0 = pr & 0xffff, c0 = pr >> 16;
        if (!in_bounds(a0 < nv && c0 < nv && p < R.pair_cap, s.red)) continue;
        int a1 = (a0 + 1 == nv) ? 0 : a0 + 1, c1 = (c0 + 1 == nv) ? 0 : c0 + 1;
        float su = F1.x, uu = F1.y, W = F1.z;
        V3<float> n = f3(F0);
        V3<float> vrel = (1.f - su) * f3(s.V[a0]) + su * f3(s.V[a1]) - (1.f - uu) * f3(s.V[c0]) - uu * f3(s.V[c1]);
        V3<float> vt = vrel - dot(vrel, n) * n;
        float vt2 = dot(vt, vt);
        if (!(vt2 > 1e-24f)) continue;
        float coef = fminf(mu * F0.w / (h * sqrtf(vt2)), 1.f);
        V3<float> dv = (-(coef / W)) * vt;
        const int idx[4] = {a0, a1, c0, c1};
        const float wt[4] = {s.X[a0].w * (1.f - su), s.X[a1].w * su, -s.X[c0].w * (1.f - uu), -s.X[c1].w * uu};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(&s.acc[idx[k]].x, to_fix(wt[k] * dv.x, kFixVel));
            atomicAdd(&s.acc[idx[k]].y, to_fix(wt[k] * dv.y, kFixVel));
            atomicAdd(&s.acc[idx[k]].z, to_fix(wt[k] * dv.z, kFixVel));
        }
    }
    g.sync();
    for (int i = g.tid; i < nv; i += TPR) {
        int4 q = s.acc[i];
        if (q.x | q.y | q.z) {
            float4 v = s.V[i];
            const float inv = 1.f / kFixVel;
            s.V[i] = make_float4(v.x + q.x * inv, v.y + q.y * inv, v.z + q.z * inv, v.w);
            s.acc[i] = make_int4(0, 0, 0, 0);
        }
    }
    g.sync();
}

// The contact sweep and friction as out-of-line calls.  They run only on frames with
// candidates; kept out of the substep's inlined code they add no registers, and no code, to
// the path every substep takes.  The rod's shared-memory view is rebuilt from its base
// inside (a view passed by reference would be read from memory at every use).
template <int NV, bool CONTACT, int TPR>
__device__ __noinline__ void contact_sweep_call(const RodInfo* R, float4* base, int gtid, int gbar, int np,
                                                bool first) {
    Smem<NV, CONTACT> s(base);
    const Grp<TPR> g{gtid, gbar, s.red};
    contact_sweep<NV, CONTACT, TPR>(*R, s, g, np, first);
}

template <int NV, bool CONTACT, int TPR>
__device__ __noinline__ void self_friction_call(const RodInfo* R, float4* base, int gtid, int gbar, int np,
                                                float h, float mu) {
    Smem<NV, CONTACT> s(base);
    const Grp<TPR> g{gtid, gbar, s.red};
    self_friction<NV, CONTACT, TPR>(*R, s, g, np, h, mu);
}

// An edge's frame for the hinge phase from its stored (t, |e|), (d1r, cos theta) and
// sin theta: d2r = t x d1r and the material frame, as edge_forward forms them.
__device__ __forceinline__ void load_frame(EdgeF<float>& E, float4 ta, float4 rc, float sn) {
    E.t = f3(ta);
    E.d1r = f3(rc);
    E.c = rc.w;
    E.s = sn;
    E.d2r = cross(E.t, E.d1r);
    E.d1 = E.c * E.d1r + E.s * E.d2r;
    E.d2 = E.c * E.d2r - E.s * E.d1r;
}

// A hinge's gradient seeds for one of its edges, added to the edge's sums (the other hinge of
// the edge adds to the same sums).
__device__ __forceinline__ void add_seeds(float4* sg, float4* sr, V3<float> gt, V3<float> gd1r, float gth) {
    atomicAdd(&sg->x, gt.x);
    atomicAdd(&sg->y, gt.y);
    atomicAdd(&sg->z, gt.z);
    atomicAdd(&sg->w, gth);
    atomicAdd(&sr->x, gd1r.x);
    atomicAdd(&sr->y, gd1r.y);
    atomicAdd(&sr->z, gd1r.z);
}

// ------------------------------------------------------------------ one substep
template <int NV, bool CONTACT, int TPR>
__device__ __forceinline__ void substep_body(const SceneDev& sc, const float4* __restrict__ KIN, const float2* __restrict__ ES,
                        const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, float h, int np,
                        const Rec* rec = nullptr, float4* imp = nullptr, float* mv = nullptr) {
    const int nv = R.nv, ne = R.ne, v0 = R.v0, e0 = R.e0;
    const bool closed = R.flags & ROD_CLOSED;
    const int nh = closed ? nv : nv - 2;
    const bool strands = R.flags & ROD_STRANDS;
    // --- edge frames, once per edge: (t, |e|) in EA, (w0, n1) in EW, (d1r, cos theta) in ND
    // (the vertex phase takes the new reference director from there), and per edge the seeds
    // its two hinges send back: (dU/dt, dU/dtheta) in SG, (dU/dd1r, sin theta) in SR.  The
    // displacement array SR = X is rewritten by the vertex phase before it is read.
    float4* const EA = s.HB0;
    float4* const EW = s.HB1;
    float4* const SG = s.HB2;
    float4* const SR = s.X;
    for (int j = g.tid; j < ne; j += TPR) {
        const int j1 = (j + 1 == nv) ? 0 : j + 1;
        const float4 ed = s.ED[j], et = s.ET[j];
        SG[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (strands && !(et.w > 0.f)) continue;   // a break edge: no frame, no hinge
        EdgeF<float> E;
        edge_forward(E, f3(s.X0[j]), f3(s.X0[j1]), f3(et), f3(ed), ed.w);
        EA[j] = f4(E.t, E.ell);
        EW[j] = f4(E.w0, E.n1);
        s.ND[j] = f4(E.d1r, E.c);
        SR[j] = make_float4(0.f, 0.f, 0.f, E.s);
    }
    g.sync();
    // --- hinge phase: the hinge's own part, from its edges' frames
    for (int k = g.tid; k < nh; k += TPR) {
        const int i = closed ? k : k + 1;
        const int a = (i == 0) ? ne - 1 : i - 1;
        const int b = i;
        const float4 ETa = s.ET[a], ETb = s.ET[b];
        float4 hg = s.HG[i];
        if (strands && !(ETa.w > 0.f && ETb.w > 0.f)) continue;   // a hinge at an end of a break edge
        HingeF<float> H;
        load_frame(H.a, EA[a], s.ND[a], SR[a].w);
        load_frame(H.b, EA[b], s.ND[b], SR[b].w);
        hinge_core_forward(H, s.ED[a].w, s.ED[b].w, hg.w);
        const float lbar = 0.5f * (ETa.w + ETb.w);
        if (R.flags & ROD_PLASTIC) plastic_update(H.k0, H.k1, hg.x, hg.y, R.sy * lbar, R.rc);
        const float il = 1.f / lbar;
        const float gk0 = R.Bm * il * (H.k0 - hg.x), gk1 = R.Bm * il * (H.k1 - hg.y);
        const float gm = R.beta * il * (H.m - hg.z);
        V3<float> gta, gd1ra, gtb, gd1rb;
        float ghta, ghtb;
        hinge_core_reverse(H, gk0, gk1, gm, 0.f, gta, gd1ra, gtb, gd1rb, ghta, ghtb);
        add_seeds(SG + a, SR + a, gta, gd1ra, ghta);
        add_seeds(SG + b, SR + b, gtb, gd1rb, ghtb);
        s.HG[i] = make_float4(hg.x, hg.y, hg.z, H.mref);
    }
    g.sync();
    // --- per edge, the reverse through its frame: the gradient on the edge vector (in SG, with
    // the edge's twist gradient; zero for a break edge)
    for (int j = g.tid; j < ne; j += TPR) {
        const float4 et = s.ET[j], sg = SG[j];
        if (strands && !(et.w > 0.f)) continue;   // SG[j] stays zero
        const float4 ea = EA[j], ew = EW[j], nd = s.ND[j];
        EdgeF<float> E;
        E.t = f3(ea);
        E.ell = ea.w;
        E.w0 = f3(ew);
        E.n1 = ew.w;
        E.d1r = f3(nd);
        const V3<float> ge =
            edge_reverse<float, false>(E, f3(et), f3(s.ED[j]), f3(sg), f3(SR[j]), 0.f, nullptr, nullptr);
        SG[j] = f4(ge, sg.w);
    }
    g.sync();
    // --- vertex phase
    for (int i = g.tid; i < nv; i += TPR) {
        const float4 xi4 = s.X0[i];
        const V3<float> xi = f3(xi4);
        V3<float> g = zf3();
        const int im = (i == 0) ? nv - 1 : i - 1;
        float gth = 0.f;
        const bool has_e = closed || i < nv - 1;          // edge i starts here
        const bool has_em = closed || i >= 1;             // edge i-1 ends here
        // bending and twisting: the gradients on the edge vectors of the edges at this vertex
        if (has_e) {
            const float4 q = SG[i];
            g -= f3(q);
            gth = q.w;
        }
        if (has_em) g += f3(SG[im]);
        V3<float> t_i = zf3();
        float ell_i = 0.f;
        // a break edge (between two strands) starts here: no tangent, no force, frame kept
        const bool brk = strands && has_e && !(ES[e0 + i].x > 0.f);
        // stretching: the strains with IEEE-rounded square roots and quotients (the strains of
        // nearly inextensible ropes are ~1e-4, so a few ulps of the length matter to them)
        if (has_e && !brk) {
            const float4 q = EA[i];
            ell_i = q.w;
            t_i = f3(q);
            if (R.kA > 0.f) g -= (R.kA * edge_strain(f3(s.X0[i + 1 == nv ? 0 : i + 1]) - xi, ES[e0 + i].x)) * t_i;
        }
        if (R.kA > 0.f && has_em && !(strands && !(ES[e0 + im].x > 0.f)))   // edge i-1 ends here
            g += (R.kA * edge_strain(xi - f3(s.X0[im]), ES[e0 + im].x)) * f3(EA[im]);
        float4 vi = s.V[i];
        const float4 kin = KIN[v0 + i];
        const int kind = (int)kin.w;
        // displacement d of this substep (positions are only formed at its end, so the rebuilt
        // velocity d/h carries no cancellation error from |x| >> |h v|)
        V3<float> v2 = zf3(), d = zf3();
        float4 nd_out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kind == 0) {
            V3<float> grav = f3(0.f, 0.f, -sc.gravity);
            V3<float> acc = (-xi4.w) * g + grav - R.cd * f3(vi);
            V3<float> v1 = f3(vi) + h * acc;
            if (rec) rec->v1[i] = f4(v1, 0.f);
            v2 = rigid_contact(sc, R, xi, v1, s.sp, imp ? imp + 4 * i : nullptr, 1.f / xi4.w);
            d = h * v2;
        } else if (kind >= 2 && in_bounds(kind - 2 < R.ngrip, s.red)) {
            const float* o = s.sp + 32 * (kind - 2);
            const V3<float> off = f3(kin);
            const V3<float> p1 = f3(o[3], o[4], o[5]);
            const V3<float> tgt = p1 + f3(o[15] * off.x + o[16] * off.y + o[17] * off.z,
                                          o[18] * off.x + o[19] * off.y + o[20] * off.z,
                                          o[21] * off.x + o[22] * off.y + o[23] * off.z);
            nd_out = f4(tgt, 1.f);      // absolute target at the substep end
            d = tgt - xi;               // a grasped vertex sits at the gripper target
            v2 = d / h;
        }
        float om1 = vi.w;
        if (has_e) {
            const float invI = ES[e0 + i].y;
            om1 = vi.w + h * (-gth * invI - R.cd * vi.w);
            float4 ed = s.ED[i];
            if (brk) {
                s.ED[i] = make_float4(ed.x, ed.y, ed.z, ed.w + h * om1);
            } else {
                s.ED[i] = f4(f3(s.ND[i]), ed.w + h * om1);   // the edge's new reference director
                s.ET[i] = f4(t_i, ES[e0 + i].x);
            }
        }
        s.ND[i] = nd_out;
        s.X[i] = f4(d, xi4.w);
        s.V[i] = f4(v2, om1);
    }
    g.sync();
    // --- PBD
    const bool lenc = R.flags & (ROD_INEXT | ROD_SLIMIT);
    if (lenc || np > 0) {
        for (int it = 0; it < sc.n_iter; ++it) {
            if (lenc) {
                const int ncol = (closed && (ne & 1)) ? 3 : 2;
                for (int k = 0; k < ncol; ++k)
                    inext_color<NV, CONTACT, TPR>(R, s, g, k, closed, rec ? rec->pbd + (size_t)it * rec->nvmax : nullptr);
            }
            if (CONTACT && np > 0) {
                // each thread stores its own vertices; the sweep reads s.X and writes only the
                // accumulators before its own barrier
                if (rec)
                    for (int i = g.tid; i < nv; i += TPR) rec->csnap[(size_t)it * rec->nvmax + i] = s.X[i];
                contact_sweep_call<NV, CONTACT, TPR>(&R, s.X, g.tid, g.bar, np, it == 0);
            }
        }
    }
    // --- velocity from the displacement, friction, new positions
    const float ih = 1.f / h;
    for (int i = g.tid; i < nv; i += TPR) {
        float4 d = s.X[i], v = s.V[i];
        if (rec) rec->dfin[i] = d;
        s.V[i] = make_float4(d.x * ih, d.y * ih, d.z * ih, v.w);
    }
    g.sync();
    if (CONTACT && rec)
        for (int p = g.tid; p < np; p += TPR) {
            rec->fr0[p] = s.fr0[p];
            rec->fr1[p] = s.fr1[p];
        }
    if (CONTACT && np > 0) self_friction_call<NV, CONTACT, TPR>(&R, s.X, g.tid, g.bar, np, h, sc.mu_self);
    float dm2 = 0.f;   // the largest squared displacement of this thread's vertices
    for (int i = g.tid; i < nv; i += TPR) {
        float4 x0 = s.X0[i], d = s.X[i], nd = s.ND[i];
        float4 x = nd.w > 0.5f ? make_float4(nd.x, nd.y, nd.z, x0.w)
                               : make_float4(x0.x + d.x, x0.y + d.y, x0.z + d.z, x0.w);
        if (mv) {
            const float dx = x.x - x0.x, dy = x.y - x0.y, dz = x.z - x0.z;
            dm2 = fmaxf(dm2, dx * dx + dy * dy + dz * dz);
        }
        s.X0[i] = x;
        s.X[i] = x;
    }
    if (mv) *mv += sqrtf(dm2);
    g.sync();
}


// The substep inlined (the forward kernel, and the backward's per-frame recompute with
// records, where a call costs more than the larger code) and as one out-of-line copy (the
// backward's replay of the frames between two checkpoints).
template <int NV, bool CONTACT, int TPR>
__device__ __noinline__ void substep_call(const SceneDev& sc, const float4* __restrict__ KIN,
                                          const float2* __restrict__ ES, const RodInfo& R, Smem<NV, CONTACT>& s,
                                          const Grp<TPR>& g, float h, int np, const Rec* rec) {
    substep_body<NV, CONTACT, TPR>(sc, KIN, ES, R, s, g, h, np, rec);
}

// Substep pose block of gripper q (32 floats at out + 32 q) from the frame-start pose F
// (per gripper p (3), R (9) row major) and the frame's actions: positions and rotations at
// the substep's start (c0) and end (c1) of the frame, p + c dp and exp(c dphi) R (the start
// rotation of the first substep is the frame's own), and the rigid velocities dp/dt, dphi/dt.
__device__ __forceinline__ void substep_pose(const float* F, const float* act, int q, float c0, float c1, bool first,
                                             float inv_dt, float* out) {
    const float* f = F + 12 * q;
    const float* a = act + 6 * q;
    M3 RF;
#pragma unroll
    for (int k = 0; k < 9; ++k) RF.m[k] = f[3 + k];
    const M3 R0 = first ? RF : matmul(expmap(f3(c0 * a[3], c0 * a[4], c0 * a[5])), RF);
    const M3 R1 = matmul(expmap(f3(c1 * a[3], c1 * a[4], c1 * a[5])), RF);
    float* o = out + 32 * q;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o[c] = f[c] + c0 * a[c];
        o[3 + c] = f[c] + c1 * a[c];
        o[24 + c] = a[c] * inv_dt;
        o[27 + c] = a[3 + c] * inv_dt;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        o[6 + k] = R0.m[k];
        o[15 + k] = R1.m[k];
    }
}

// Frame end for gripper q: p += dp, R = exp(dphi) R.
__device__ __forceinline__ void frame_advance(float* F, const float* act, int q) {
    float* f = F + 12 * q;
    const float* a = act + 6 * q;
    M3 RF;
#pragma unroll
    for (int k = 0; k < 9; ++k) RF.m[k] = f[3 + k];
    const M3 Rn = matmul(expmap(f3(a[3], a[4], a[5])), RF);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] += a[c];
#pragma unroll
    for (int k = 0; k < 9; ++k) f[3 + k] = Rn.m[k];
}

// One frame of one rod: candidates (if self-contact), nsub substeps, pose update.  The frame's
// start pose is s.fp and its actions s.act, both set (and synchronised) by the caller; s.fp
// holds the end pose on return.  pre(sb) runs before substep sb (after a group barrier), e.g.
// to store the substep state, and returns the substep's record (or nullptr).  imp: the rod's
// impulse slots (4 per vertex) when the contact impulses are being accumulated (inlined
// substeps only).  mv (inlined substeps only): adds, per thread, the sum over the frame's
// substeps of the largest displacement of the thread's vertices, a bound on how far any of
// them moved during the frame.
template <int NV, bool CONTACT, int TPR, bool INLINE, class PreSub>
__device__ __forceinline__ int run_frame(const SceneDev& sc, const float4* __restrict__ KIN, const float2* __restrict__ ES,
                         const RodInfo& R, Smem<NV, CONTACT>& s, const Grp<TPR>& g, int nsub, float h, bool& ovf,
                         PreSub pre, float4* imp = nullptr, float* mv = nullptr) {
    int np = 0;
    if (CONTACT && (R.flags & ROD_SELF))
        np = (R.flags & ROD_HASH) ? broad_phase_hash<NV, CONTACT, TPR>(R, s, g, (R.flags & ROD_CLOSED) != 0, ovf)
                                  : broad_phase<NV, CONTACT, TPR>(R, s, g, (R.flags & ROD_CLOSED) != 0, ovf);
    const float inv_dt = 1.f / sc.dt;
    for (int sb = 0; sb < nsub; ++sb) {
        const Rec* rec = pre(sb);
        // the substep's gripper block: written here, read after the hinge phase's barrier
        if (g.tid < R.ngrip)
            substep_pose(s.fp, s.act, g.tid, (float)sb / (float)nsub, (float)(sb + 1) / (float)nsub, sb == 0, inv_dt,
                         s.sp);
        if (INLINE)
            substep_body<NV, CONTACT, TPR>(sc, KIN, ES, R, s, g, h, np, rec, imp, mv);
        else
            substep_call<NV, CONTACT, TPR>(sc, KIN, ES, R, s, g, h, np, rec);
    }
    if (g.tid < R.ngrip) frame_advance(s.fp, s.act, g.tid);
    g.sync();
    return np;
}

}  // namespace dlo
