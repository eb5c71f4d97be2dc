// dlo_plain.cu -- dlo_step_plain: the same rollout written the plain way, the comparator
// for the persistent kernels.  One kernel launch per phase per substep, one thread per
// element (rod, hinge, vertex, edge or contact-pair slot) across every rod at once, and the
// whole state in HBM between phases; the element functions and the operation order are
// those of the fused substep (dlo_step.cuh), so both follow the same trajectory up to
// rounding.  Self-contact candidates are found once per frame by brute force over each
// rod's edge pairs (the same set the fused kernel's broad phase finds).  Armed by
// dlo_begin_rollout it records checkpoints and actions like dlo_step, and dlo_backward_plain
// then differentiates the rollout the same way: one kernel launch per phase of the reverse per
// substep, one thread per element, the records and cotangents in HBM.
#include <algorithm>
#include <vector>

#include "dlo_bwd_kernel.cuh"
#include "dlo_kernels.h"
#include "dlo_runtime.h"

namespace dlo {
namespace {

// workspace layout (one allocation, built on the first call)
struct PlainWs {
    int* vrod;        // [V] rod of each vertex
    int* erod;        // [Et] rod of each edge
    int* prod;        // [P] rod of each pair slot
    int* poff;        // [B] first pair slot of each rod
    int* npair;       // [B] candidates found this frame
    uint32_t* pairs;  // [P] (a | b << 16), local edge indices
    float4* D;        // [V] displacement of the substep (w = inverse mass)
    float4* TGT;      // [V] gripper target of a grasped vertex (w = 1), else 0
    float4* NDR;      // [Et] transported reference d1 of each edge
    float4* HB0;      // [V] hinge gradient on its previous vertex (w: on edge i-1's twist)
    float4* HB1;      // [V] on its own vertex (w: on edge i's twist)
    float4* HB2;      // [V] on its next vertex
    float4* FR0;      // [P] first-iteration contact normal, depth
    float4* FR1;      // [P] closest parameters, weight sum, active flag
    int4* ACC;        // [V] fixed-point accumulators (kept at zero between uses)
    float* POSE;      // [B][64]: the substep gripper block of each rod (layout of Smem::sp)
    float* ZACT;      // [B][12] zero actions (frames stepped without actions)
    long long P;      // pair slots
};

__device__ __forceinline__ int nsub_of(const RodInfo& R, int force) { return force > 0 ? force : R.nsub; }

// gripper block of substep s (positions, rotations and rigid velocities, Sec. 3.2)
__global__ void pl_pose(SceneDev sc, const RodInfo* rods, int B, const float* GP, const float* act, int s, int force,
                        float* POSE) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    for (int q = 0; q < R.ngrip; ++q)
        substep_pose(GP + 24LL * b, act + 12LL * b, q, (float)s / (float)n, (float)(s + 1) / (float)n, s == 0,
                     1.f / sc.dt, POSE + 64LL * b);
}

// frame end: p += dp, R = exp(dphi) R
__global__ void pl_pose_advance(const RodInfo* rods, int B, float* GP, const float* act) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    for (int q = 0; q < R.ngrip; ++q) frame_advance(GP + 24LL * b, act + 12LL * b, q);
}

// candidates of one frame: every edge pair of a rod outside the exclusion window whose
// segments are closer than the candidate distance (one thread per first edge)
__global__ void pl_broad(const RodInfo* rods, const int* erod, long long Et, const float2* ES, const float4* X,
                         const int* poff, int* npair, uint32_t* pairs, unsigned* status) {
    const long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ge >= Et) return;
    const int b = erod[ge];
    const RodInfo R = rods[b];
    if (!(R.flags & ROD_SELF)) return;
    const bool closed = R.flags & ROD_CLOSED, strands = R.flags & ROD_STRANDS;
    const int a = (int)(ge - R.e0), nv = R.nv, ne = R.ne;
    // break edges (between the strands of one record) are no segments
    auto real = [&](int j) { return !strands || ES[R.e0 + j].x > 0.f; };
    if (!real(a)) return;
    const int a1 = (a + 1 == nv) ? 0 : a + 1;
    const V3<float> pa0 = f3(X[R.v0 + a]), pa1 = f3(X[R.v0 + a1]);
    bool ovf = false;
    for (int c = a + 1; c < ne; ++c) {
        if (!real(c)) continue;
        int sep = c - a;
        if (closed) sep = min(sep, ne - sep);
        if (sep <= R.excl) {   // the window applies within one strand
            bool other = false;
            for (int k = a + 1; strands && k < c; ++k) other |= !real(k);
            if (!other) continue;
        }
        const int c1 = (c + 1 == nv) ? 0 : c + 1;
        const V3<float> pb0 = f3(X[R.v0 + c]), pb1 = f3(X[R.v0 + c1]);
        float su, uu;
        closest_params(pa0, pa1, pb0, pb1, su, uu);
        const V3<float> dd = (pa0 + su * (pa1 - pa0)) - (pb0 + uu * (pb1 - pb0));
        if (!(sqrtf(dot(dd, dd)) < R.contact_d)) continue;
        const int idx = atomicAdd(&npair[b], 1);
        if (idx < R.pair_cap)
            pairs[poff[b] + idx] = (uint32_t)a | ((uint32_t)c << 16);
        else
            ovf = true;
    }
    if (ovf) atomicOr(&status[b], 2u);
}

// hinge phase: frames, plasticity and the hinge's energy gradient (one thread per hinge)
__global__ void pl_hinge(const RodInfo* rods, const int* vrod, long long V, const float4* X, const float4* ED,
                         const float4* ET, float4* HG, float4* HB0, float4* HB1, float4* HB2, float4* NDR, int s,
                         int force) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    if (s >= nsub_of(R, force)) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int nv = R.nv, ne = R.ne, i = (int)(gv - R.v0);
    if (!closed && (i < 1 || i > nv - 2)) return;
    const int a = (i == 0) ? ne - 1 : i - 1;
    const int b = i;
    const int im = (i == 0) ? nv - 1 : i - 1;
    const int ip = (i + 1 == nv) ? 0 : i + 1;
    const float4 EDa = ED[R.e0 + a], EDb = ED[R.e0 + b], ETa = ET[R.e0 + a], ETb = ET[R.e0 + b];
    const bool strands = R.flags & ROD_STRANDS;
    if (strands && !(ETa.w > 0.f && ETb.w > 0.f)) {   // a hinge at an end of a break edge
        HB0[gv] = HB1[gv] = HB2[gv] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float4 hg = HG[gv];
    HingeF<float> H;
    hinge_forward(H, f3(X[R.v0 + im]), f3(X[gv]), f3(X[R.v0 + ip]), f3(ETa), f3(EDa), f3(ETb), f3(EDb), EDa.w,
                  EDb.w, hg.w);
    const float lbar = 0.5f * (ETa.w + ETb.w);
    if (R.flags & ROD_PLASTIC) plastic_update(H.k0, H.k1, hg.x, hg.y, R.sy * lbar, R.rc);
    const float il = 1.f / lbar;
    const float gk0 = R.Bm * il * (H.k0 - hg.x), gk1 = R.Bm * il * (H.k1 - hg.y);
    const float gm = R.beta * il * (H.m - hg.z);
    V3<float> gxm, gxi, gxp;
    float gta, gtb;
    hinge_reverse<float, false>(H, f3(ETa), f3(EDa), f3(ETb), f3(EDb), gk0, gk1, gm, 0.f, gxm, gxi, gxp, gta, gtb,
                                nullptr, nullptr, nullptr, nullptr);
    HB0[gv] = f4(gxm, gta);
    HB1[gv] = f4(gxi, gtb);
    HB2[gv] = f4(gxp, 0.f);
    NDR[R.e0 + b] = f4(H.b.d1r, 0.f);
    // the first edge of an open rod or strand gets its frame from its only hinge
    if (!closed && (i == 1 || (strands && !(ET[R.e0 + a - 1].w > 0.f)))) NDR[R.e0 + a] = f4(H.a.d1r, 0.f);
    HG[gv] = make_float4(hg.x, hg.y, hg.z, H.mref);
}

// vertex phase: forces, symplectic Euler, rigid contact, twist update (one thread per vertex)
__global__ void pl_vertex(SceneDev sc, const RodInfo* rods, const int* vrod, long long V, const float4* KIN,
                          const float2* ES, const float4* X, float4* Vl, float4* ED, float4* ET,
                          const float4* HB0, const float4* HB1, const float4* HB2, const float4* NDR, float4* D,
                          float4* TGT, const float* POSE, const float* act, int s, int force, float4* V1out) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const int rod = vrod[gv];
    const RodInfo R = rods[rod];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float h = sc.dt / (float)n;
    const bool closed = R.flags & ROD_CLOSED;
    const int nv = R.nv, v0 = R.v0, e0 = R.e0, i = (int)(gv - v0);
    const int nh = closed ? nv : nv - 2;
    auto has_h = [&](int j) { return closed || (j >= 1 && j <= nv - 2); };
    const int ip = (i + 1 == nv) ? 0 : i + 1;
    const int im = (i == 0) ? nv - 1 : i - 1;
    const float4 xi4 = X[gv];
    const V3<float> xi = f3(xi4);
    V3<float> g = zf3();
    float gth = 0.f;
    const bool has_e = closed || i < nv - 1;
    if (has_h(i)) {
        const float4 q = HB1[gv];
        g += f3(q);
        gth += q.w;
    }
    if ((closed || i + 1 <= nv - 2) && has_h(ip) && (closed || i + 1 < nv)) {
        const float4 q = HB0[v0 + ip];
        g += f3(q);
        if (has_e) gth += q.w;
    }
    if ((closed || i >= 2) && has_h(im)) g += f3(HB2[v0 + im]);
    V3<float> t_i = zf3();
    const bool strands = R.flags & ROD_STRANDS;
    const bool brk = strands && has_e && !(ES[e0 + i].x > 0.f);   // a break edge starts here
    if (has_e && !brk) {
        const V3<float> e = f3(X[v0 + ip]) - xi;
        const float ell_i = sqrtf(dot(e, e));
        t_i = e / ell_i;
        if (R.kA > 0.f) g -= (R.kA * edge_strain(e, ES[e0 + i].x)) * t_i;
    }
    if (R.kA > 0.f && (closed || i >= 1) && !(strands && !(ES[e0 + im].x > 0.f))) {
        const V3<float> e = xi - f3(X[v0 + im]);
        g += (R.kA * edge_strain(e, ES[e0 + im].x)) * (e / sqrtf(dot(e, e)));
    }
    const float4 vi = Vl[gv];
    const float4 kin = KIN[gv];
    const int kind = (int)kin.w;
    const float* pose = POSE + 64LL * rod;
    V3<float> v2 = zf3(), d = zf3();
    float4 tgt4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kind == 0) {
        const V3<float> grav = f3(0.f, 0.f, -sc.gravity);
        const V3<float> acc = (-xi4.w) * g + grav - R.cd * f3(vi);
        const V3<float> v1 = f3(vi) + h * acc;
        if (V1out) V1out[gv] = f4(v1, 0.f);
        v2 = rigid_contact(sc, R, xi, v1, pose);
        d = h * v2;
    } else if (kind >= 2) {
        const float* o = pose + 32 * (kind - 2);
        const V3<float> off = f3(kin);
        const V3<float> tgt = f3(o[3], o[4], o[5]) + f3(o[15] * off.x + o[16] * off.y + o[17] * off.z,
                                                        o[18] * off.x + o[19] * off.y + o[20] * off.z,
                                                        o[21] * off.x + o[22] * off.y + o[23] * off.z);
        tgt4 = f4(tgt, 1.f);
        d = tgt - xi;
        v2 = d / h;
    }
    float om1 = vi.w;
    if (has_e) {
        const float invI = ES[e0 + i].y;
        om1 = vi.w + h * (-gth * invI - R.cd * vi.w);
        const float4 ed = ED[e0 + i];
        if (brk) {
            ED[e0 + i] = make_float4(ed.x, ed.y, ed.z, ed.w + h * om1);
        } else {
            const int ne = R.ne;
            const bool solo = nh == 0 || (strands && (i == 0 || !(ES[e0 + i - 1].x > 0.f)) &&
                                          (i + 1 >= ne || !(ES[e0 + i + 1].x > 0.f)));
            V3<float> d1r = solo ? zf3() : f3(NDR[e0 + i]);
            if (solo) {
                EdgeF<float> E;
                edge_forward(E, xi, f3(X[v0 + ip]), f3(ET[e0 + i]), f3(ed), ed.w);
                d1r = E.d1r;
            }
            ED[e0 + i] = f4(d1r, ed.w + h * om1);
            ET[e0 + i] = f4(t_i, ES[e0 + i].x);
        }
    }
    TGT[gv] = tgt4;
    D[gv] = f4(d, xi4.w);
    Vl[gv] = f4(v2, om1);
}

// one colour of the inextensibility / strain-limit projection (one thread per edge)
__global__ void pl_inext(const RodInfo* rods, const int* erod, long long Et, const float4* X, float4* D, const float4* ET,
                         int color, int s, int force, float4* PBDout) {
    const long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ge >= Et) return;
    const RodInfo R = rods[erod[ge]];
    if (s >= nsub_of(R, force) || !(R.flags & (ROD_INEXT | ROD_SLIMIT))) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int nv = R.nv, ne = R.ne, j = (int)(ge - R.e0);
    if (color == 2 && !(closed && (ne & 1))) return;
    int first, last;
    color_range(ne, closed, color, first, last);
    if (j < first || j >= last || ((j - first) & 1)) return;
    const int j1 = (j + 1 == nv) ? 0 : j + 1;
    const float4 A = D[R.v0 + j], B = D[R.v0 + j1];
    const V3<float> e = (f3(X[R.v0 + j1]) - f3(X[R.v0 + j])) + (f3(B) - f3(A));
    float ell, ie;
    len_inv(e, ell, ie);
    const float eb = ET[R.e0 + j].w;
    float target;
    bool active;
    if (R.flags & ROD_INEXT) {
        target = eb;
        active = true;
    } else {
        const float hi = (1.f + R.slim) * eb, lo = (1.f - R.slim) * eb;
        active = (ell > hi) || (ell < lo);
        target = ell > hi ? hi : lo;
    }
    const float ws = A.w + B.w;
    if (!active || !(ws > 0.f) || !(eb > 0.f)) {   // eb = 0: the edge between two strands
        if (PBDout) PBDout[ge] = make_float4(0.f, 0.f, 0.f, 1.f);
        return;
    }
    const float lam = (ell - target) / ws;
    const V3<float> t = ie * e;
    if (PBDout) PBDout[ge] = f4(t, target * ie);
    const V3<float> da = (lam * A.w) * t, db = (lam * B.w) * t;
    D[R.v0 + j] = make_float4(A.x + da.x, A.y + da.y, A.z + da.z, A.w);
    D[R.v0 + j1] = make_float4(B.x - db.x, B.y - db.y, B.z - db.z, B.w);
}

// one Jacobi sweep of the self-collision projection (one thread per pair slot)
// Debug builds (-DDLO_DEBUG_BOUNDS): a pair index outside its rod sets status bit 8 of the rod
// and the pair is skipped.  Release builds compile the check away.
__device__ __forceinline__ bool pair_ok(int a0, int c0, int nv, unsigned* status, int b) {
#ifdef DLO_DEBUG_BOUNDS
    if (a0 < nv && c0 < nv) return true;
    atomicOr(&status[b], kStatusBounds);
    return false;
#else
    (void)a0;
    (void)c0;
    (void)nv;
    (void)status;
    (void)b;
    return true;
#endif
}

__global__ void pl_contact(const RodInfo* rods, const int* prod, long long P, const int* poff, const int* npair,
                           const uint32_t* pairs, const float4* X, const float4* D, int4* ACC, float4* FR0,
                           float4* FR1, int first, int s, int force, unsigned* status) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = prod[p];
    const RodInfo R = rods[b];
    if (s >= nsub_of(R, force) || p - poff[b] >= min(npair[b], R.pair_cap)) return;
    const int nv = R.nv, v0 = R.v0;
    const uint32_t pr = pairs[p];
    const int a0 = pr & 0xffff, c0 = pr >> 16;
    if (!pair_ok(a0, c0, R.nv, status, b)) return;
    const int a1 = (a0 + 1 == nv) ? 0 : a0 + 1, c1 = (c0 + 1 == nv) ? 0 : c0 + 1;
    const V3<float> o = f3(X[v0 + a0]);
    const float4 A0 = D[v0 + a0], A1 = D[v0 + a1], C0 = D[v0 + c0], C1 = D[v0 + c1];
    const V3<float> pa0 = f3(A0), pa1 = (f3(X[v0 + a1]) - o) + f3(A1);
    const V3<float> pc0 = (f3(X[v0 + c0]) - o) + f3(C0), pc1 = (f3(X[v0 + c1]) - o) + f3(C1);
    V3<float> dx[4], n;
    float su, uu, d, W;
    const bool on = pair_correction(pa0, pa1, pc0, pc1, A0.w, A1.w, C0.w, C1.w, 2.f * R.radius, dx, su, uu, n, d, W);
    if (first) {
        FR0[p] = f4(on ? n : zf3(), on ? d : 0.f);
        FR1[p] = make_float4(su, uu, W, on ? 1.f : 0.f);
    }
    if (on) {
        const int idx[4] = {v0 + a0, v0 + a1, v0 + c0, v0 + c1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(&ACC[idx[k]].x, to_fix(dx[k].x, kFixPos));
            atomicAdd(&ACC[idx[k]].y, to_fix(dx[k].y, kFixPos));
            atomicAdd(&ACC[idx[k]].z, to_fix(dx[k].z, kFixPos));
        }
    }
}

// add the fixed-point sums to a per-vertex array and clear them (one thread per vertex)
__global__ void pl_apply(long long V, int4* ACC, float4* T, float scale) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const int4 q = ACC[gv];
    if (q.x | q.y | q.z) {
        const float4 x = T[gv];
        const float inv = 1.f / scale;
        T[gv] = make_float4(x.x + q.x * inv, x.y + q.y * inv, x.z + q.z * inv, x.w);
        ACC[gv] = make_int4(0, 0, 0, 0);
    }
}

// velocity from the substep's displacement (one thread per vertex)
__global__ void pl_velocity(SceneDev sc, const RodInfo* rods, const int* vrod, long long V, const float4* D,
                            float4* Vl, int s, int force, float4* DFout) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float ih = 1.f / (sc.dt / (float)n);
    const float4 d = D[gv], v = Vl[gv];
    if (DFout) DFout[gv] = d;
    Vl[gv] = make_float4(d.x * ih, d.y * ih, d.z * ih, v.w);
}

// self-contact friction from the first iteration's contact set (one thread per pair slot)
__global__ void pl_friction(SceneDev sc, const RodInfo* rods, const int* prod, long long P, const int* poff,
                            const int* npair, const uint32_t* pairs, const float4* X, const float4* Vl,
                            const float4* FR0, const float4* FR1, int4* ACC, int s, int force, unsigned* status) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = prod[p];
    const RodInfo R = rods[b];
    const int n = nsub_of(R, force);
    if (s >= n || p - poff[b] >= min(npair[b], R.pair_cap)) return;
    const float h = sc.dt / (float)n;
    const float4 F1 = FR1[p];
    if (!(F1.w > 0.f)) return;
    const float4 F0 = FR0[p];
    const int nv = R.nv, v0 = R.v0;
    const uint32_t pr = pairs[p];
    const int a0 = pr & 0xffff, c0 = pr >> 16;
    if (!pair_ok(a0, c0, R.nv, status, b)) return;
    const int a1 = (a0 + 1 == nv) ? 0 : a0 + 1, c1 = (c0 + 1 == nv) ? 0 : c0 + 1;
    const float su = F1.x, uu = F1.y, W = F1.z;
    const V3<float> nn = f3(F0);
    const V3<float> vrel = (1.f - su) * f3(Vl[v0 + a0]) + su * f3(Vl[v0 + a1]) - (1.f - uu) * f3(Vl[v0 + c0]) -
                           uu * f3(Vl[v0 + c1]);
    const V3<float> vt = vrel - dot(vrel, nn) * nn;
    const float vt2 = dot(vt, vt);
    if (!(vt2 > 1e-24f)) return;
    const float coef = fminf(sc.mu_self * F0.w / (h * sqrtf(vt2)), 1.f);
    const V3<float> dv = (-(coef / W)) * vt;
    const int idx[4] = {v0 + a0, v0 + a1, v0 + c0, v0 + c1};
    const float wt[4] = {X[v0 + a0].w * (1.f - su), X[v0 + a1].w * su, -X[v0 + c0].w * (1.f - uu),
                         -X[v0 + c1].w * uu};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        atomicAdd(&ACC[idx[k]].x, to_fix(wt[k] * dv.x, kFixVel));
        atomicAdd(&ACC[idx[k]].y, to_fix(wt[k] * dv.y, kFixVel));
        atomicAdd(&ACC[idx[k]].z, to_fix(wt[k] * dv.z, kFixVel));
    }
}

// positions at the substep end (one thread per vertex)
__global__ void pl_finalize(const RodInfo* rods, const int* vrod, long long V, float4* X, const float4* D,
                            const float4* TGT, int s, int force) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    if (s >= nsub_of(R, force)) return;
    const float4 x0 = X[gv], d = D[gv], t = TGT[gv];
    X[gv] = t.w > 0.5f ? make_float4(t.x, t.y, t.z, x0.w) : make_float4(x0.x + d.x, x0.y + d.y, x0.z + d.z, x0.w);
}

// non-finite state check (one thread per rod)
__global__ void pl_status(const RodInfo* rods, int B, const float4* X, const float4* Vl, unsigned* status) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    bool nf = false;
    for (int i = 0; i < R.nv; ++i) {
        const float4 x = X[R.v0 + i], v = Vl[R.v0 + i];
        nf |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z) &&
                isfinite(v.w));
    }
    if (nf) atomicOr(&status[b], 1u);
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

dlo_status plain_workspace(dlo_ctx* c, PlainWs& w) {
    std::vector<int> vrod(c->V), erod(c->Et), poff(c->B);
    long long P = 0;
    for (int b = 0; b < c->B; ++b) {
        const RodInfo& R = c->rods_h[b];
        for (int i = 0; i < R.nv; ++i) vrod[R.v0 + i] = b;
        for (int j = 0; j < R.ne; ++j) erod[R.e0 + j] = b;
        poff[b] = (int)P;
        if (R.flags & ROD_SELF) P += R.pair_cap;
    }
    std::vector<int> prod(std::max<long long>(P, 1), 0);
    for (int b = 0; b < c->B; ++b)
        if (c->rods_h[b].flags & ROD_SELF)
            for (int k = 0; k < c->rods_h[b].pair_cap; ++k) prod[poff[b] + k] = b;
    const long long V = c->V, Et = c->Et, B = c->B, Pn = std::max<long long>(P, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_vrod = take(4 * V), o_erod = take(4 * Et), o_prod = take(4 * Pn), o_poff = take(4 * B),
                 o_npair = take(4 * B), o_pairs = take(4 * Pn), o_D = take(16 * V), o_TGT = take(16 * V),
                 o_NDR = take(16 * Et), o_HB0 = take(16 * V), o_HB1 = take(16 * V), o_HB2 = take(16 * V),
                 o_FR0 = take(16 * Pn), o_FR1 = take(16 * Pn), o_ACC = take(16 * V), o_POSE = take(4 * 64 * B),
                 o_ZACT = take(4 * 12 * B);
    if (off > c->pl_bytes) {
        dev_free(c, c->pl_mem);
        c->pl_mem = dev_alloc(c, off);
        c->pl_bytes = c->pl_mem ? off : 0;
        if (!c->pl_mem) return set_err(c, DLO_ERR_OOM, "plain comparator workspace allocation failed");
    }
    char* m = reinterpret_cast<char*>(c->pl_mem);
    w.vrod = reinterpret_cast<int*>(m + o_vrod);
    w.erod = reinterpret_cast<int*>(m + o_erod);
    w.prod = reinterpret_cast<int*>(m + o_prod);
    w.poff = reinterpret_cast<int*>(m + o_poff);
    w.npair = reinterpret_cast<int*>(m + o_npair);
    w.pairs = reinterpret_cast<uint32_t*>(m + o_pairs);
    w.D = reinterpret_cast<float4*>(m + o_D);
    w.TGT = reinterpret_cast<float4*>(m + o_TGT);
    w.NDR = reinterpret_cast<float4*>(m + o_NDR);
    w.HB0 = reinterpret_cast<float4*>(m + o_HB0);
    w.HB1 = reinterpret_cast<float4*>(m + o_HB1);
    w.HB2 = reinterpret_cast<float4*>(m + o_HB2);
    w.FR0 = reinterpret_cast<float4*>(m + o_FR0);
    w.FR1 = reinterpret_cast<float4*>(m + o_FR1);
    w.ACC = reinterpret_cast<int4*>(m + o_ACC);
    w.POSE = reinterpret_cast<float*>(m + o_POSE);
    w.ZACT = reinterpret_cast<float*>(m + o_ZACT);
    w.P = P;
    cudaError_t e = cudaMemcpyAsync(w.vrod, vrod.data(), 4 * V, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.erod, erod.data(), 4 * Et, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.prod, prod.data(), 4 * prod.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.poff, poff.data(), 4 * B, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ACC, 0, 16 * V, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.POSE, 0, 4 * 64 * B, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ZACT, 0, 4 * 12 * B, c->stream);
    // the host vectors die at return: finish the copies first
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(c, e, "plain comparator workspace");
}


// ------------------------------------------------------------------ one plain frame
// State arrays the plain kernels step (the context's live state, or the backward's copy).
struct PlainState {
    float4 *X, *Vl, *HG, *ED, *ET;
    float* GP;   // [B][24]
};
// Optional records of one frame's substeps for the plain backward: per substep the arrays of
// every rod, at stride sV (vertex arrays), sE (edge arrays) and sP (pair arrays) per substep.
struct PlainRec {
    float4 *X0, *V, *HG, *ED, *ET, *V1, *DF, *PBD, *CSN, *FR0, *FR1;
    long long sV, sE, sP;
};

// The kernels of one frame of every rod (candidates, then per substep: pose, hinges, vertices,
// N_C x (colours, contact sweep), velocities, friction, positions; then the frame's pose).
cudaError_t plain_frame(dlo_ctx* c, const PlainWs& w, const PlainState& S, const float* act, int substeps,
                        int nsub_max, const PlainRec* rec) {
    const bool contact = c->opt.self_contact != 0 && w.P > 0;
    const long long V = c->V, Et = c->Et, P = w.P;
    const int B = c->B, T = 128, n_iter = c->opt.n_iter_pbd;
    cudaStream_t sm = c->stream;
    cudaError_t e = cudaSuccess;
    if (contact) {
        e = cudaMemsetAsync(w.npair, 0, 4 * (size_t)B, sm);
        pl_broad<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, c->d_es, S.X, w.poff, w.npair, w.pairs,
                                              c->d_status);
        c->launches++;
    }
    for (int s = 0; s < nsub_max && e == cudaSuccess; ++s) {
        if (rec) {   // the substep's start state
            e = cudaMemcpyAsync(rec->X0 + s * rec->sV, S.X, 16 * V, cudaMemcpyDeviceToDevice, sm);
            if (e == cudaSuccess) e = cudaMemcpyAsync(rec->V + s * rec->sV, S.Vl, 16 * V, cudaMemcpyDeviceToDevice, sm);
            if (e == cudaSuccess) e = cudaMemcpyAsync(rec->HG + s * rec->sV, S.HG, 16 * V, cudaMemcpyDeviceToDevice, sm);
            if (e == cudaSuccess) e = cudaMemcpyAsync(rec->ED + s * rec->sE, S.ED, 16 * Et, cudaMemcpyDeviceToDevice, sm);
            if (e == cudaSuccess) e = cudaMemcpyAsync(rec->ET + s * rec->sE, S.ET, 16 * Et, cudaMemcpyDeviceToDevice, sm);
        }
        pl_pose<<<blocks(B, T), T, 0, sm>>>(c->scene, c->d_rods, B, S.GP, act, s, substeps, w.POSE);
        pl_hinge<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, S.X, S.ED, S.ET, S.HG, w.HB0, w.HB1, w.HB2, w.NDR,
                                             s, substeps);
        pl_vertex<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, c->d_kin, c->d_es, S.X, S.Vl, S.ED,
                                              S.ET, w.HB0, w.HB1, w.HB2, w.NDR, w.D, w.TGT, w.POSE, act, s, substeps,
                                              rec ? rec->V1 + s * rec->sV : nullptr);
        c->launches += 3;
        for (int it = 0; it < n_iter; ++it) {
            for (int k = 0; k < 3; ++k)
                pl_inext<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, S.X, w.D, S.ET, k, s, substeps,
                                                      rec ? rec->PBD + s * rec->sE * n_iter + it * rec->sE : nullptr);
            c->launches += 3;
            if (contact) {
                if (rec && e == cudaSuccess)
                    e = cudaMemcpyAsync(rec->CSN + s * rec->sV * n_iter + it * rec->sV, w.D, 16 * V,
                                        cudaMemcpyDeviceToDevice, sm);
                pl_contact<<<blocks(P, T), T, 0, sm>>>(c->d_rods, w.prod, P, w.poff, w.npair, w.pairs, S.X, w.D, w.ACC,
                                                       rec ? rec->FR0 + s * rec->sP : w.FR0,
                                                       rec ? rec->FR1 + s * rec->sP : w.FR1, it == 0, s, substeps,
                                                       c->d_status);
                pl_apply<<<blocks(V, T), T, 0, sm>>>(V, w.ACC, w.D, kFixPos);
                c->launches += 2;
            }
        }
        pl_velocity<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, w.D, S.Vl, s, substeps,
                                                rec ? rec->DF + s * rec->sV : nullptr);
        c->launches++;
        if (contact) {
            pl_friction<<<blocks(P, T), T, 0, sm>>>(c->scene, c->d_rods, w.prod, P, w.poff, w.npair, w.pairs, S.X,
                                                    S.Vl, rec ? rec->FR0 + s * rec->sP : w.FR0,
                                                    rec ? rec->FR1 + s * rec->sP : w.FR1, w.ACC, s, substeps,
                                                    c->d_status);
            pl_apply<<<blocks(V, T), T, 0, sm>>>(V, w.ACC, S.Vl, kFixVel);
            c->launches += 2;
        }
        pl_finalize<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, S.X, w.D, w.TGT, s, substeps);
        c->launches++;
    }
    pl_pose_advance<<<blocks(B, T), T, 0, sm>>>(c->d_rods, B, S.GP, act);
    c->launches++;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// ------------------------------------------------------------------ the plain backward
// Per-phase reverse kernels, one thread per element across every rod, all state in HBM; each
// phase is the one of reverse_substep (dlo_bwd_kernel.cuh) written out for global arrays.
// Per-rod sums (material, pose and action cotangents) are added atomically.
struct PlainAdj {
    float4 *LX, *LD, *LV, *LE, *LT, *LK, *LP0, *LG, *LTMP, *HBE;
    double* GM;      // [B][5]
    float* LPF;      // [B][12]: frame-start pose cotangents (position 6, rotation 6)
    float* GA;       // [B][12]: the frame's action cotangents
    float* PA;       // [B][36]: the substep's pose cotangents (ps0, phs0, ps1, phs1, vp, w; 6 each)
    float* PM;       // [B][72]: the substep's pose maps (pose_rev_mat, 36 per gripper)
    float* GPF;      // [B][24]: the frame's start pose
};

__device__ __forceinline__ void atomic_add3f(float* a, V3<float> v) {
    atomicAdd(a, v.x);
    atomicAdd(a + 1, v.y);
    atomicAdd(a + 2, v.z);
}

__global__ void prb_init(const RodInfo* rods, const int* vrod, const int* erod, long long V, long long Et,
                         const float4* dLdx, const float4* dLdv, const float* dLdth, PlainAdj A, int B) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < V) {
        const RodInfo R = rods[vrod[t]];
        float4 dx = dLdx ? dLdx[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 dv = dLdv ? dLdv[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(R.flags & ROD_CLOSED) && t - R.v0 == R.nv - 1) dv.w = 0.f;
        A.LX[t] = make_float4(dx.x, dx.y, dx.z, 0.f);
        A.LV[t] = dv;
        A.LK[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (t < Et) {
        A.LE[t] = make_float4(0.f, 0.f, 0.f, dLdth ? dLdth[t] : 0.f);
        A.LT[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (t < B) {
        for (int k = 0; k < 5; ++k) A.GM[5 * t + k] = 0.0;
        for (int k = 0; k < 12; ++k) A.LPF[12 * t + k] = 0.f;
    }
}

// frame start: the carried frame-end pose cotangents into this frame's actions (per rod)
__global__ void prb_frame_begin(const RodInfo* rods, int B, const float* act, PlainAdj A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    float* ga = A.GA + 12 * b;
    float* lp = A.LPF + 12 * b;
    for (int k = 0; k < 12; ++k) ga[k] = 0.f;
    for (int q = 0; q < R.ngrip; ++q) {
        const float* a = act + 12LL * b + 6 * q;
        const V3<float> dphi = f3(a[3], a[4], a[5]);
        const V3<float> lr = f3(lp[6 + 3 * q], lp[7 + 3 * q], lp[8 + 3 * q]);
        ga[6 * q] = lp[3 * q];
        ga[6 * q + 1] = lp[3 * q + 1];
        ga[6 * q + 2] = lp[3 * q + 2];
        const V3<float> jr = jl_t(dphi, lr);
        ga[6 * q + 3] = jr.x;
        ga[6 * q + 4] = jr.y;
        ga[6 * q + 5] = jr.z;
        const V3<float> nr = mulT(expmap(dphi), lr);
        lp[6 + 3 * q] = nr.x;
        lp[7 + 3 * q] = nr.y;
        lp[8 + 3 * q] = nr.z;
    }
}

// substep start: the gripper block, the pose maps, zero pose cotangents (per rod)
__global__ void prb_sub_begin(SceneDev sc, const RodInfo* rods, int B, const float* act, int s, int force,
                              float* POSE, PlainAdj A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    const int n = nsub_of(R, force);
    for (int k = 0; k < 36; ++k) A.PA[36 * b + k] = 0.f;
    if (s >= n) return;
    const float c0 = (float)s / (float)n, c1 = (float)(s + 1) / (float)n;
    for (int q = 0; q < R.ngrip; ++q) {
        substep_pose(A.GPF + 24LL * b, act + 12LL * b, q, c0, c1, s == 0, 1.f / sc.dt, POSE + 64LL * b);
        for (int m = 0; m < 4; ++m) pose_rev_mat(act + 12LL * b, 4 * q + m, c0, c1, A.PM + 72LL * b);
    }
}

// B1: positions at the substep end (per vertex)
__global__ void prb_b1(const RodInfo* rods, const int* vrod, long long V, const float4* KIN, const float* POSE, int s,
                       int force, PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const int rod = vrod[gv];
    const RodInfo R = rods[rod];
    if (s >= nsub_of(R, force)) return;
    const float4 kin = KIN[gv];
    const int kind = (int)kin.w;
    const float4 lx = A.LX[gv];
    if (kind >= 2) {
        const int q = kind - 2;
        const V3<float> y1 = mul_rm(POSE + 64LL * rod + 32 * q + 15, f3(kin));
        float* pa = A.PA + 36LL * rod;
        atomic_add3f(pa + 12 + 3 * q, f3(lx));                 // ps1
        atomic_add3f(pa + 18 + 3 * q, cross(y1, f3(lx)));      // phs1
        A.LX[gv] = make_float4(0.f, 0.f, 0.f, 0.f);
        A.LD[gv] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        A.LD[gv] = make_float4(lx.x, lx.y, lx.z, 0.f);
    }
}

// B2: self-contact friction (per pair slot), into LP0 (positions) and LTMP (velocities)
__global__ void prb_b2(SceneDev sc, const RodInfo* rods, const int* prod, long long P, const int* poff,
                       const int* npair, const uint32_t* pairs, const float4* X0, const float4* T0, const float4* DF,
                       const float4* FR1, int s, int force, PlainAdj A, unsigned* status) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = prod[p];
    const RodInfo R = rods[b];
    const int n = nsub_of(R, force);
    if (s >= n || p - poff[b] >= min(npair[b], R.pair_cap)) return;
    if (!(FR1[p].w > 0.f)) return;
    const float h = sc.dt / (float)n, ih = 1.f / h;
    const int nv = R.nv, v0 = R.v0;
    const uint32_t pr = pairs[p];
    const int a0 = pr & 0xffff, q0 = pr >> 16;
    if (!pair_ok(a0, q0, R.nv, status, b)) return;
    const int idx[4] = {v0 + a0, v0 + ((a0 + 1 == nv) ? 0 : a0 + 1), v0 + q0, v0 + ((q0 + 1 == nv) ? 0 : q0 + 1)};
    const V3<float> o = f3(X0[idx[0]]);
    V3<float> Pf[4], Vf[4], lo[4];
    float w[4];
    for (int k = 0; k < 4; ++k) {
        Pf[k] = (k == 0) ? f3(T0[idx[0]]) : (f3(X0[idx[k]]) - o) + f3(T0[idx[k]]);
        Vf[k] = ih * f3(DF[idx[k]]);
        w[k] = X0[idx[k]].w;
        lo[k] = f3(A.LV[idx[k]]);
    }
    V3<float> pb[4], vb[4];
    if (!fric_pair_vjp(Pf, Vf, w, 2.f * R.radius, sc.mu_self, h, lo, pb, vb)) return;
    for (int k = 0; k < 4; ++k) {
        atomic_add3(&A.LP0[idx[k]], pb[k]);
        atomic_add3(&A.LTMP[idx[k]], vb[k]);
    }
}

// B2 gather, then B3: the velocity rebuilt from the displacement (per vertex)
__global__ void prb_b3(SceneDev sc, const RodInfo* rods, const int* vrod, long long V, int s, int force, int fric,
                       PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float ih = (float)n / sc.dt;
    float4 l = A.LV[gv];
    if (fric) {
        const float4 t = A.LTMP[gv];
        l = make_float4(l.x + t.x, l.y + t.y, l.z + t.z, l.w);
    }
    const V3<float> lv = ih * f3(l);
    const float4 d = A.LD[gv];
    A.LD[gv] = make_float4(d.x + lv.x, d.y + lv.y, d.z + lv.z, 0.f);
    A.LV[gv] = make_float4(0.f, 0.f, 0.f, l.w);
}

// B4, contact sweep of iteration it (per pair slot), into LTMP
__global__ void prb_b4c(const RodInfo* rods, const int* prod, long long P, const int* poff, const int* npair,
                        const uint32_t* pairs, const float4* X0, const float4* Dc, int s, int force, PlainAdj A,
                        unsigned* status) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = prod[p];
    const RodInfo R = rods[b];
    if (s >= nsub_of(R, force) || p - poff[b] >= min(npair[b], R.pair_cap)) return;
    const int nv = R.nv, v0 = R.v0;
    const uint32_t pr = pairs[p];
    const int a0 = pr & 0xffff, q0 = pr >> 16;
    if (!pair_ok(a0, q0, R.nv, status, b)) return;
    const int idx[4] = {v0 + a0, v0 + ((a0 + 1 == nv) ? 0 : a0 + 1), v0 + q0, v0 + ((q0 + 1 == nv) ? 0 : q0 + 1)};
    const V3<float> o = f3(X0[idx[0]]);
    V3<float> Pf[4], lo[4];
    float w[4];
    for (int k = 0; k < 4; ++k) {
        Pf[k] = (k == 0) ? f3(Dc[idx[0]]) : (f3(X0[idx[k]]) - o) + f3(Dc[idx[k]]);
        w[k] = X0[idx[k]].w;
        lo[k] = f3(A.LD[idx[k]]);
    }
    V3<float> pb[4];
    if (!pair_correction_vjp(Pf, w, 2.f * R.radius, lo, pb)) return;
    for (int k = 0; k < 4; ++k) atomic_add3(&A.LTMP[idx[k]], pb[k]);
}

// B4, the contact sweep's cotangents added (per vertex), plus the friction's on iteration 0
__global__ void prb_b4a(const RodInfo* rods, const int* vrod, long long V, int s, int force, int with_p0, PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    if (s >= nsub_of(R, force)) return;
    float4 t = A.LTMP[gv];
    if (with_p0) {
        const float4 q = A.LP0[gv];
        t = make_float4(t.x + q.x, t.y + q.y, t.z + q.z, 0.f);
    }
    const float4 ld = A.LD[gv], lx = A.LX[gv];
    A.LD[gv] = make_float4(ld.x + t.x, ld.y + t.y, ld.z + t.z, 0.f);
    A.LX[gv] = make_float4(lx.x + t.x, lx.y + t.y, lx.z + t.z, 0.f);
}

// B4, colour k of the length projections of iteration it in reverse (per edge)
__global__ void prb_b4k(const RodInfo* rods, const int* erod, long long Et, const float4* X0, const float4* Q, int color,
                        int s, int force, PlainAdj A) {
    const long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ge >= Et) return;
    const RodInfo R = rods[erod[ge]];
    if (s >= nsub_of(R, force) || !(R.flags & (ROD_INEXT | ROD_SLIMIT))) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int nv = R.nv, ne = R.ne, j = (int)(ge - R.e0);
    if (color == 2 && !(closed && (ne & 1))) return;
    int first, last;
    color_range(ne, closed, color, first, last);
    if (j < first || j >= last || ((j - first) & 1)) return;
    const float4 q = Q[ge];
    if (q.x == 0.f && q.y == 0.f && q.z == 0.f) return;
    const long long a = R.v0 + j, b = R.v0 + ((j + 1 == nv) ? 0 : j + 1);
    const float wa = X0[a].w, wb = X0[b].w, ws = wa + wb;
    const V3<float> t = f3(q);
    const V3<float> la = f3(A.LD[a]), lb = f3(A.LD[b]);
    const V3<float> mu = (wa / ws) * la - (wb / ws) * lb;
    const V3<float> le = mu - q.w * (mu - dot(mu, t) * t);
    A.LD[a] = f4(la - le, 0.f);
    A.LD[b] = f4(lb + le, 0.f);
    A.LX[a] = f4(f3(A.LX[a]) - le, 0.f);
    A.LX[b] = f4(f3(A.LX[b]) + le, 0.f);
}

// B5: rigid contact, symplectic Euler, gravity, damping, twist rate (per vertex)
__global__ void prb_b5(SceneDev sc, const RodInfo* rods, const int* vrod, long long V, const float4* KIN,
                       const float2* ES, const float4* X0, const float4* Vn_, const float4* V1, const float* POSE,
                       int s, int force, PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const int rod = vrod[gv];
    const RodInfo R = rods[rod];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float h = sc.dt / (float)n;
    const bool closed = R.flags & ROD_CLOSED;
    const int i = (int)(gv - R.v0), nv = R.nv;
    const float4 kin = KIN[gv];
    const int kind = (int)kin.w;
    const float4 x4 = X0[gv], vn = Vn_[gv];
    const V3<float> ld0 = f3(A.LD[gv]);
    const float* sp = POSE + 64LL * rod;
    float* pa = A.PA + 36LL * rod;
    float4 lvn = make_float4(0.f, 0.f, 0.f, 0.f), lg = make_float4(0.f, 0.f, 0.f, 0.f);
    double gd = 0.0;
    if (kind == 0) {
        V3<float> lam = h * ld0;
        const int nprim = sc.n_planes + sc.n_boxes + R.ngrip;
        V3<float> vs[kMaxPlanes + kMaxBoxes + 2];
        vs[0] = f3(V1[gv]);
        const V3<float> x = f3(x4);
        unsigned onmask = 0;
        for (int k = 0; k < nprim; ++k) {
            const int q = k - sc.n_planes - sc.n_boxes;
            V3<float> gp = zf3(), gax = zf3(), vp = zf3(), w = zf3();
            if (q >= 0) {
                const float* o = sp + 32 * q;
                gp = f3(o[0], o[1], o[2]);
                gax = f3(o[8], o[11], o[14]);
                vp = f3(o[24], o[25], o[26]);
                w = f3(o[27], o[28], o[29]);
            }
            bool on;
            V3<float> nxt = prim_respond<float>(k, sc, R, x, vs[k], gp, gax, vp, w, on);
            if (on) onmask |= 1u << k;
            if (k + 1 < kMaxPlanes + kMaxBoxes + 2) vs[k + 1] = nxt;
        }
        V3<float> lx_acc = zf3();
        for (int k = nprim - 1; k >= 0; --k) {
            if (!((onmask >> k) & 1u)) continue;
            const int q = k - sc.n_planes - sc.n_boxes;
            V3<float> gp = zf3(), gax = zf3(), vp = zf3(), w = zf3();
            if (q >= 0) {
                const float* o = sp + 32 * q;
                gp = f3(o[0], o[1], o[2]);
                gax = f3(o[8], o[11], o[14]);
                vp = f3(o[24], o[25], o[26]);
                w = f3(o[27], o[28], o[29]);
            }
            V3<float> ntmp;
            if (q >= 0 && sdf_capsule(x, gp - sc.grip_hl * gax, gp + sc.grip_hl * gax, sc.grip_r, ntmp) > -sc.grip_r) {
                V3<float> lxk, lvk, lpk, lphik, lvpk, lwk;
                capsule_contact_rev(x, vs[k], gp, gax, sc.grip_hl, sc.grip_r, vp, w, R.radius, R.eps, sc.mu_rigid,
                                    sc.restitution, lam, lxk, lvk, lpk, lphik, lvpk, lwk);
                lx_acc += lxk;
                lam = lvk;
                atomic_add3f(pa + 3 * q, lpk);          // ps0
                atomic_add3f(pa + 6 + 3 * q, lphik);    // phs0
                atomic_add3f(pa + 24 + 3 * q, lvpk);    // vp
                atomic_add3f(pa + 30 + 3 * q, lwk);     // w
                continue;
            }
            if (k < sc.n_planes) {
                const V3<float> nn = f3(sc.planes[k]);
                V3<float> lv, ln, lvr;
                float lsdf;
                contact_respond_rev(vs[k], dot(x, nn) - sc.planes[k].w, nn, zf3(), R.radius, R.eps, sc.mu_rigid,
                                    sc.restitution, lam, lv, lsdf, ln, lvr);
                lx_acc += lsdf * nn;
                lam = lv;
                continue;
            }
            if (q < 0) {   // box: closed-form reverse
                const int bi = k - sc.n_planes;
                V3<float> lv;
                lx_acc += box_contact_rev(x, vs[k], f3(sc.box_c[bi]), f3(sc.box_h[bi]), R.radius, R.eps, sc.mu_rigid,
                                          sc.restitution, lam, lv);
                lam = lv;
                continue;
            }
            const int nin = 18;   // the degenerate on-axis gripper contact keeps dual numbers
            float lin[18];
            for (int d = 0; d < nin; ++d) {
                V3<float> e = zf3();
                (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
                const int gq = d / 3;
                V3<dualf> xd = lift(x, gq == 0 ? e : zf3()), vd = lift(vs[k], gq == 1 ? e : zf3());
                V3<dualf> gpd = lift(gp, gq == 2 ? e : zf3()), gaxd = lift(gax, gq == 3 ? cross(e, gax) : zf3());
                V3<dualf> vpd = lift(vp, gq == 4 ? e : zf3()), wd = lift(w, gq == 5 ? e : zf3());
                bool on2;
                V3<dualf> out = prim_respond<dualf>(k, sc, R, xd, vd, gpd, gaxd, vpd, wd, on2);
                lin[d] = dot(ders(out), lam);
            }
            lx_acc += f3(lin[0], lin[1], lin[2]);
            lam = f3(lin[3], lin[4], lin[5]);
            atomic_add3f(pa + 3 * q, f3(lin[6], lin[7], lin[8]));
            atomic_add3f(pa + 6 + 3 * q, f3(lin[9], lin[10], lin[11]));
            atomic_add3f(pa + 24 + 3 * q, f3(lin[12], lin[13], lin[14]));
            atomic_add3f(pa + 30 + 3 * q, f3(lin[15], lin[16], lin[17]));
        }
        lvn = f4((1.f - h * R.cd) * lam, 0.f);
        lg = f4((-h * x4.w) * lam, 0.f);
        gd += -(double)h * (double)dot(f3(vn), lam);
        A.LX[gv] = f4(f3(A.LX[gv]) + lx_acc, 0.f);
    } else if (kind >= 2) {
        const int q = kind - 2;
        atomic_add3f(pa + 12 + 3 * q, ld0);                                              // ps1
        atomic_add3f(pa + 18 + 3 * q, cross(mul_rm(sp + 32 * q + 15, f3(kin)), ld0));    // phs1
        A.LX[gv] = f4(f3(A.LX[gv]) - ld0, 0.f);
    }
    const bool has_e = closed || i < nv - 1;
    if (has_e) {
        const long long ge = R.e0 + i;
        const float lw1 = A.LV[gv].w + h * A.LE[ge].w;
        const float invI = ES[ge].y;
        lvn.w = (1.f - h * R.cd) * lw1;
        lg.w = -h * invI * lw1;
        gd += -(double)h * (double)vn.w * (double)lw1;
    }
    A.LV[gv] = lvn;
    A.LG[gv] = lg;
    if (gd != 0.0) atomicAdd(&A.GM[5 * rod + 4], gd);
}

// the substep's pose cotangents into the frame-start pose and the frame's actions (per rod)
__global__ void prb_pose(SceneDev sc, const RodInfo* rods, int B, int s, int force, PlainAdj A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const RodInfo R = rods[b];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float c0 = (float)s / (float)n, c1 = (float)(s + 1) / (float)n, idt = 1.f / sc.dt;
    const float* pa = A.PA + 36 * b;
    float* ga = A.GA + 12 * b;
    float* lp = A.LPF + 12 * b;
    for (int q = 0; q < R.ngrip; ++q) {
        const V3<float> ps0 = f3(pa[3 * q], pa[3 * q + 1], pa[3 * q + 2]);
        const V3<float> ph0 = f3(pa[6 + 3 * q], pa[7 + 3 * q], pa[8 + 3 * q]);
        const V3<float> ps1 = f3(pa[12 + 3 * q], pa[13 + 3 * q], pa[14 + 3 * q]);
        const V3<float> ph1 = f3(pa[18 + 3 * q], pa[19 + 3 * q], pa[20 + 3 * q]);
        const V3<float> vp = f3(pa[24 + 3 * q], pa[25 + 3 * q], pa[26 + 3 * q]);
        const V3<float> w = f3(pa[30 + 3 * q], pa[31 + 3 * q], pa[32 + 3 * q]);
        const float* pm = A.PM + 72 * b + 36 * q;
        const V3<float> lpf = ps0 + ps1;
        lp[3 * q] += lpf.x;
        lp[3 * q + 1] += lpf.y;
        lp[3 * q + 2] += lpf.z;
        const V3<float> gdp = c0 * ps0 + c1 * ps1 + idt * vp;
        const V3<float> gdr = mul_rm(pm + 18, ph0) + mul_rm(pm + 27, ph1) + idt * w;
        ga[6 * q] += gdp.x;
        ga[6 * q + 1] += gdp.y;
        ga[6 * q + 2] += gdp.z;
        ga[6 * q + 3] += gdr.x;
        ga[6 * q + 4] += gdr.y;
        ga[6 * q + 5] += gdr.z;
        const V3<float> m0 = f3(pm[0] * ph0.x + pm[3] * ph0.y + pm[6] * ph0.z, pm[1] * ph0.x + pm[4] * ph0.y + pm[7] * ph0.z,
                                pm[2] * ph0.x + pm[5] * ph0.y + pm[8] * ph0.z);
        const V3<float> m1 = f3(pm[9] * ph1.x + pm[12] * ph1.y + pm[15] * ph1.z,
                                pm[10] * ph1.x + pm[13] * ph1.y + pm[16] * ph1.z,
                                pm[11] * ph1.x + pm[14] * ph1.y + pm[17] * ph1.z);
        const V3<float> r = m0 + m1;
        lp[6 + 3 * q] += r.x;
        lp[7 + 3 * q] += r.y;
        lp[8 + 3 * q] += r.z;
    }
}

// B8: the new reference-frame base and the stretching force's second order (per edge)
__global__ void prb_b8(const RodInfo* rods, const int* erod, long long Et, const float2* ES, const float4* X0,
                       const float4* ED, const float4* ET, int s, int force, PlainAdj A) {
    const long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ge >= Et) return;
    const int rod = erod[ge];
    const RodInfo R = rods[rod];
    if (s >= nsub_of(R, force)) return;
    const int nv = R.nv, j = (int)(ge - R.e0);
    const long long a = R.v0 + j, b = R.v0 + ((j + 1 == nv) ? 0 : j + 1);
    const float4 ed = ED[ge], et = ET[ge];
    if ((R.flags & ROD_STRANDS) && !(et.w > 0.f)) {   // a break edge kept its base frame: identity reverse
        A.HBE[ge] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    EdgeF<float> E;
    edge_forward(E, f3(X0[a]), f3(X0[b]), f3(et), f3(ed), ed.w);
    V3<float> gtb, gd1b;
    V3<float> le = edge_reverse<float, true>(E, f3(et), f3(ed), f3(A.LT[ge]), f3(A.LE[ge]), 0.f, &gtb, &gd1b);
    if (R.kA > 0.f) {
        const V3<float> les = f3(A.LG[b]) - f3(A.LG[a]);
        const float eb = ES[ge].x;
        const float tl = dot(E.t, les);
        const float st = edge_strain(f3(X0[b]) - f3(X0[a]), eb);
        le += R.kA * ((tl / eb) * E.t + st / E.ell * (les - tl * E.t));
        atomicAdd(&A.GM[5 * rod + 0], (double)st * (double)tl);
    }
    A.HBE[ge] = f4(le, 0.f);
    A.LT[ge] = f4(gtb, 0.f);
    A.LE[ge] = f4(gd1b, A.LE[ge].w);
}

// B8 gather: each vertex takes the edge cotangents of the edges it ends (per vertex)
__global__ void prb_b8g(const RodInfo* rods, const int* vrod, long long V, int s, int force, PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    if (s >= nsub_of(R, force)) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int i = (int)(gv - R.v0), nv = R.nv, ne = R.ne;
    V3<float> l = f3(A.LX[gv]);
    if (closed || i < nv - 1) l -= f3(A.HBE[R.e0 + i]);
    if (closed || i > 0) l += f3(A.HBE[R.e0 + (i == 0 ? ne - 1 : i - 1)]);
    A.LX[gv] = f4(l, 0.f);
}

// B7: hinges, the elastic force's second order (dual numbers), plasticity and its reverse
// (per hinge, at its vertex)
__global__ void prb_b7(const RodInfo* rods, const int* vrod, long long V, const float4* X0, const float4* ED,
                       const float4* ET, const float4* HG, int s, int force, PlainAdj A) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const int rod = vrod[gv];
    const RodInfo R = rods[rod];
    if (s >= nsub_of(R, force)) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int nv = R.nv, ne = R.ne, i = (int)(gv - R.v0);
    if (!closed && (i < 1 || i > nv - 2)) return;
    const long long ea = R.e0 + ((i == 0) ? ne - 1 : i - 1), eb = R.e0 + i;
    const long long im = R.v0 + ((i == 0) ? nv - 1 : i - 1), ip = R.v0 + ((i + 1 == nv) ? 0 : i + 1);
    const float4 EDa = ED[ea], EDb = ED[eb], ETa = ET[ea], ETb = ET[eb], hg = HG[gv];
    if ((R.flags & ROD_STRANDS) && !(ETa.w > 0.f && ETb.w > 0.f)) return;   // at an end of a break edge
    const float lbar = 0.5f * (ETa.w + ETb.w), il = 1.f / lbar;
    HingeF<dualf> Hd;
    const float4 gm_ = A.LG[im], gi_ = A.LG[gv], gp_ = A.LG[ip];
    // the twist-rate cotangent of edge j sits with vertex j (the edge starting there)
    hinge_forward(Hd, lift(f3(X0[im]), f3(gm_)), lift(f3(X0[gv]), f3(gi_)), lift(f3(X0[ip]), f3(gp_)), lift(f3(ETa)),
                  lift(f3(EDa)), lift(f3(ETb)), lift(f3(EDb)), mkd(EDa.w, A.LG[R.v0 + (ea - R.e0)].w),
                  mkd(EDb.w, A.LG[R.v0 + (eb - R.e0)].w), mkd(hg.w));
    const float hk0 = Hd.k0.v, hk1 = Hd.k1.v;
    float kb0 = hg.x, kb1 = hg.y;
    const bool yielded = (R.flags & ROD_PLASTIC) && plastic_update(hk0, hk1, kb0, kb1, R.sy * lbar, R.rc);
    dualf e0d = Hd.k0 - kb0, e1d = Hd.k1 - kb1, emd = Hd.m - hg.z;
    dualf gk0 = (R.Bm * il) * e0d, gk1 = (R.Bm * il) * e1d, gmt = (R.beta * il) * emd;
    double g1 = (double)il * ((double)e0d.v * e0d.d + (double)e1d.v * e1d.d);
    double g2 = (double)il * (double)emd.v * (double)emd.d;
    double g3 = 0.0;
    float lk0 = A.LK[gv].x - gk0.d, lk1 = A.LK[gv].y - gk1.d;
    if (yielded) {
        const float el0 = hk0 - hg.x, el1 = hk1 - hg.y;
        const float nn = sqrtf(el0 * el0 + el1 * el1), thr = R.sy * lbar;
        const float g = R.rc * (nn - thr) / nn;
        const float kk = R.rc * thr / (nn * nn * nn) * (el0 * lk0 + el1 * lk1);
        const float le0 = g * lk0 + kk * el0, le1 = g * lk1 + kk * el1;
        g3 = -(double)R.rc * lbar * ((double)el0 * lk0 + (double)el1 * lk1) / nn;
        gk0.d += le0;
        gk1.d += le1;
        lk0 -= le0;
        lk1 -= le1;
    }
    V3<dualf> gxm, gxi, gxp, gtba, gd1ba, gtbb, gd1bb;
    dualf gta, gtb;
    hinge_reverse<dualf, true>(Hd, lift(f3(ETa)), lift(f3(EDa)), lift(f3(ETb)), lift(f3(EDb)), gk0, gk1, gmt, mkd(0.f),
                               gxm, gxi, gxp, gta, gtb, &gtba, &gd1ba, &gtbb, &gd1bb);
    atomic_add3(&A.LX[im], ders(gxm));
    atomic_add3(&A.LX[gv], ders(gxi));
    atomic_add3(&A.LX[ip], ders(gxp));
    atomicAdd(&A.LE[ea].w, gta.d);
    atomicAdd(&A.LE[eb].w, gtb.d);
    atomic_add3(&A.LT[ea], ders(gtba));
    atomic_add3(&A.LE[ea], ders(gd1ba));
    atomic_add3(&A.LT[eb], ders(gtbb));
    atomic_add3(&A.LE[eb], ders(gd1bb));
    A.LK[gv] = make_float4(lk0, lk1, 0.f, 0.f);
    atomicAdd(&A.GM[5 * rod + 1], g1);
    atomicAdd(&A.GM[5 * rod + 2], g2);
    if (g3 != 0.0) atomicAdd(&A.GM[5 * rod + 3], g3);
}

// the frame's action cotangents (per rod)
__global__ void prb_frame_end(const RodInfo* rods, int B, int f, float* gact, PlainAdj A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || !gact) return;
    const RodInfo R = rods[b];
    for (int k = 0; k < 12; ++k) gact[((size_t)f * B + b) * 12 + k] = k < 6 * R.ngrip ? A.GA[12 * b + k] : 0.f;
}

// outputs: the cotangents of the initial state and the material
__global__ void prb_out(const RodInfo* rods, long long V, long long Et, int B, PlainAdj A, float4* gx0, float4* gv0,
                        float* gth0, float4* gtb0, float4* gd1b0, float* gmat) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < V) {
        if (gx0) gx0[t] = A.LX[t];
        if (gv0) gv0[t] = A.LV[t];
    }
    if (t < Et) {
        if (gth0) gth0[t] = A.LE[t].w;
        gtb0[t] = A.LT[t];
        gd1b0[t] = make_float4(A.LE[t].x, A.LE[t].y, A.LE[t].z, 0.f);
    }
    if (t < B && gmat) {
        const RodInfo R = rods[t];
        const double r = R.radius, Ar = 3.14159265358979323846 * r * r, r2 = r * r;
        const double* gm = A.GM + 5 * t;
        gmat[5 * t + 0] = R.kA > 0.f ? (float)(gm[0] * Ar) : 0.f;
        gmat[5 * t + 1] = (float)(gm[1] * Ar * r2 / 4.0);
        gmat[5 * t + 2] = (float)(gm[2] * Ar * r2 / 2.0);
        gmat[5 * t + 3] = (float)gm[3];
        gmat[5 * t + 4] = (float)gm[4];
    }
}
}  // namespace
}  // namespace dlo

using namespace dlo;

namespace dlo {
cudaError_t launch_frames_adjoint(const RodInfo* rods, int B, const float4* X0, const float4* gtb0,
                                  const float4* gd1b0, float4* gx0, V3<double>* work, cudaStream_t st);
}

// Checkpoint c of the ring from the state arrays S (the layout dlo_step writes).
static cudaError_t plain_checkpoint(dlo_ctx* c, const PlainState& S, long long cidx) {
    cudaStream_t sm = c->stream;
    cudaError_t e = cudaMemcpyAsync(c->ck.X + cidx * c->V, S.X, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ck.Vl + cidx * c->V, S.Vl, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ck.HG + cidx * c->V, S.HG, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ck.ED + cidx * c->Et, S.ED, 16 * c->Et, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ck.ET + cidx * c->Et, S.ET, 16 * c->Et, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ck.GP + cidx * 24LL * c->B, S.GP, sizeof(float) * 24 * c->B, cudaMemcpyDeviceToDevice, sm);
    return e;
}

static cudaError_t plain_restore(dlo_ctx* c, const PlainState& S, long long cidx) {
    cudaStream_t sm = c->stream;
    cudaError_t e = cudaMemcpyAsync(S.X, c->ck.X + cidx * c->V, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.Vl, c->ck.Vl + cidx * c->V, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.HG, c->ck.HG + cidx * c->V, 16 * c->V, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.ED, c->ck.ED + cidx * c->Et, 16 * c->Et, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.ET, c->ck.ET + cidx * c->Et, 16 * c->Et, cudaMemcpyDeviceToDevice, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.GP, c->ck.GP + cidx * 24LL * c->B, sizeof(float) * 24 * c->B, cudaMemcpyDeviceToDevice, sm);
    return e;
}

extern "C" dlo_status dlo_step_plain(dlo_ctx* c, const float* actions, int frames, int substeps) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (frames < 0 || substeps < 0 || substeps > 100000) return set_err(c, DLO_ERR_INVALID_ARG, "bad frames/substeps");
    if (frames == 0) return DLO_OK;
    const bool rec = c->rec_active && c->rec_done < c->rec_frames;
    if (rec) {
        if (c->rec_done + frames > c->rec_frames)
            return set_err(c, DLO_ERR_STATE, "step runs past the frames armed by dlo_begin_rollout");
        if (c->rec_nsub >= 0 && c->rec_nsub != substeps)
            return set_err(c, DLO_ERR_STATE, "substeps changed inside a recorded rollout");
    } else {
        c->rec_active = false;
    }
    PlainWs w;
    dlo_status st = plain_workspace(c, w);
    if (st != DLO_OK) return st;
    int nsub_max = substeps;
    if (!nsub_max)
        for (int b = 0; b < c->B; ++b) nsub_max = std::max(nsub_max, c->nsub[b]);
    const int B = c->B, T = 128;
    const float* acts = actions;
    if (rec) {   // the actions are recorded for the backward, as by dlo_step
        c->rec_nsub = substeps;
        float* dst = c->rec_actions + (size_t)12 * B * c->rec_done;
        cudaError_t e = actions ? cudaMemcpyAsync(dst, actions, sizeof(float) * 12 * B * frames,
                                                  cudaMemcpyDeviceToDevice, c->stream)
                                : cudaMemsetAsync(dst, 0, sizeof(float) * 12 * B * frames, c->stream);
        if (e != cudaSuccess) return cuda_err(c, e, "record actions");
        acts = dst;
    }
    const PlainState S{c->S.X, c->S.Vl, c->S.HG, c->S.ED, c->S.ET, c->S.GP};
    for (int f = 0; f < frames; ++f) {
        const float* act = acts ? acts + 12LL * B * f : w.ZACT;
        cudaError_t e = cudaSuccess;
        if (rec) {
            const int gf = c->rec_done + f;
            if (gf % c->ck_every == 0 && gf / c->ck_every < c->ck_count) e = plain_checkpoint(c, S, gf / c->ck_every);
        }
        if (e == cudaSuccess) e = plain_frame(c, w, S, act, substeps, nsub_max, nullptr);
        if (e != cudaSuccess) return cuda_err(c, e, "plain comparator launch");
    }
    pl_status<<<blocks(B, T), T, 0, c->stream>>>(c->d_rods, B, c->S.X, c->S.Vl, c->d_status);
    c->launches++;
    if (rec) c->rec_done += frames;
    c->from_set_state = false;
    return cuda_err(c, cudaGetLastError(), "plain comparator launch");
}

extern "C" dlo_status dlo_backward_plain(dlo_ctx* c, const float* dL_dx_T, const float* dL_dv_T,
                                         const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial,
                                         float* dL_dx0, float* dL_dv0, float* dL_dtheta0) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!c->rec_active || c->rec_done != c->rec_frames || c->rec_frames == 0)
        return set_err(c, DLO_ERR_STATE, "dlo_backward_plain needs a completed rollout armed by dlo_begin_rollout");
    for (const void* p : {(const void*)dL_dx_T, (const void*)dL_dv_T, (const void*)dL_dx0, (const void*)dL_dv0})
        if (p && ((uintptr_t)p & 15u)) return set_err(c, DLO_ERR_INVALID_ARG, "float4 arrays must be 16-byte aligned");
    if (c->opt.self_contact && c->opt.n_iter_pbd < 1)
        return set_err(c, DLO_ERR_INVALID_ARG, "self-contact gradients need at least one projection iteration");
    PlainWs w;
    dlo_status st = plain_workspace(c, w);
    if (st != DLO_OK) return st;
    const int force = c->rec_nsub > 0 ? c->rec_nsub : 0;
    int nsub_max = force;
    if (!nsub_max)
        for (int b = 0; b < c->B; ++b) nsub_max = std::max(nsub_max, c->nsub[b]);
    const long long V = c->V, Et = c->Et, P = w.P, Pn = std::max<long long>(P, 1);
    const int B = c->B, T = 128, n_iter = c->opt.n_iter_pbd, F = c->rec_frames, K = c->ck_every;
    const bool contact = c->opt.self_contact != 0 && P > 0;
    // workspace: the working state, one frame's records, the cotangents, per-rod sums
    const size_t nV = (size_t)V, nE = (size_t)Et;
    const size_t rec_f4 = (size_t)nsub_max * (5 * nV + 2 * nE + (size_t)n_iter * (nE + nV) + 2 * (size_t)Pn);
    const size_t f4 = 3 * nV + 2 * nE + rec_f4 + 7 * nV + 3 * nE;
    const size_t bytes = 16 * f4 + sizeof(double) * 5 * B + sizeof(float) * (size_t)B * (12 + 12 + 36 + 72 + 24 + 24) +
                         2 * 16 * nE + 4 * sizeof(V3<double>) * nV + 4096;
    if (bytes > c->bw_bytes) {
        dev_free(c, c->bw_mem);
        c->bw_mem = dev_alloc(c, bytes);
        c->bw_bytes = c->bw_mem ? bytes : 0;
        if (!c->bw_mem) return set_err(c, DLO_ERR_OOM, "plain backward workspace allocation failed");
    }
    char* m = reinterpret_cast<char*>(c->bw_mem);
    auto take4 = [&](size_t n) {
        float4* q = reinterpret_cast<float4*>(m);
        m += 16 * n;
        return q;
    };
    const PlainState S{take4(nV), take4(nV), take4(nV), take4(nE), take4(nE), nullptr};
    PlainRec R{};
    R.sV = V;
    R.sE = Et;
    R.sP = Pn;
    R.X0 = take4(nsub_max * nV);
    R.V = take4(nsub_max * nV);
    R.HG = take4(nsub_max * nV);
    R.ED = take4(nsub_max * nE);
    R.ET = take4(nsub_max * nE);
    R.V1 = take4(nsub_max * nV);
    R.DF = take4(nsub_max * nV);
    R.PBD = take4((size_t)nsub_max * n_iter * nE);
    R.CSN = take4((size_t)nsub_max * n_iter * nV);
    R.FR0 = take4(nsub_max * (size_t)Pn);
    R.FR1 = take4(nsub_max * (size_t)Pn);
    PlainAdj A{};
    A.LX = take4(nV);
    A.LD = take4(nV);
    A.LV = take4(nV);
    A.LK = take4(nV);
    A.LP0 = take4(nV);
    A.LG = take4(nV);
    A.LTMP = take4(nV);
    A.LE = take4(nE);
    A.LT = take4(nE);
    A.HBE = take4(nE);
    float4* gtb0 = take4(nE);
    float4* gd1b0 = take4(nE);
    A.GM = reinterpret_cast<double*>(m);
    m += sizeof(double) * 5 * B;
    A.LPF = reinterpret_cast<float*>(m);
    A.GA = A.LPF + 12 * B;
    A.PA = A.GA + 12 * B;
    A.PM = A.PA + 36 * B;
    A.GPF = A.PM + 72 * B;
    float* GPW = A.GPF + 24 * B;   // the working state's gripper poses
    m = reinterpret_cast<char*>(GPW + 24 * B);
    m = reinterpret_cast<char*>(((uintptr_t)m + 255) & ~(uintptr_t)255);
    V3<double>* work = reinterpret_cast<V3<double>*>(m);
    PlainState SW = S;
    SW.GP = GPW;
    cudaStream_t sm = c->stream;
    const long long NT = std::max<long long>(std::max<long long>(V, Et), B);
    prb_init<<<blocks(NT, T), T, 0, sm>>>(c->d_rods, w.vrod, w.erod, V, Et, reinterpret_cast<const float4*>(dL_dx_T),
                                          reinterpret_cast<const float4*>(dL_dv_T), dL_dtheta_T, A, B);
    c->launches++;
    for (int f = F - 1; f >= 0; --f) {
        const float* act = c->rec_actions + 12LL * B * f;
        // the frame's start state: its segment's checkpoint, then the frames before it
        const int seg = f / K, f0 = seg * K;
        cudaError_t e = plain_restore(c, SW, seg);
        for (int g = f0; g < f && e == cudaSuccess; ++g)
            e = plain_frame(c, w, SW, c->rec_actions + 12LL * B * g, force, nsub_max, nullptr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(A.GPF, SW.GP, sizeof(float) * 24 * B, cudaMemcpyDeviceToDevice, sm);
        // the frame with every substep's records
        if (e == cudaSuccess) e = plain_frame(c, w, SW, act, force, nsub_max, &R);
        if (e != cudaSuccess) return cuda_err(c, e, "plain backward recompute");
        prb_frame_begin<<<blocks(B, T), T, 0, sm>>>(c->d_rods, B, act, A);
        c->launches++;
        for (int s = nsub_max - 1; s >= 0; --s) {
            const float4 *X0 = R.X0 + s * nV, *Vn = R.V + s * nV, *HG = R.HG + s * nV, *ED = R.ED + s * nE,
                         *ET = R.ET + s * nE, *V1 = R.V1 + s * nV, *DF = R.DF + s * nV;
            const float4 *PBD = R.PBD + (size_t)s * n_iter * nE, *CSN = R.CSN + (size_t)s * n_iter * nV;
            const float4* FR1 = R.FR1 + (size_t)s * Pn;
            prb_sub_begin<<<blocks(B, T), T, 0, sm>>>(c->scene, c->d_rods, B, act, s, force, w.POSE, A);
            prb_b1<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, c->d_kin, w.POSE, s, force, A);
            c->launches += 2;
            if (contact) {
                e = cudaMemsetAsync(A.LP0, 0, 16 * nV, sm);
                if (e == cudaSuccess) e = cudaMemsetAsync(A.LTMP, 0, 16 * nV, sm);
                prb_b2<<<blocks(P, T), T, 0, sm>>>(c->scene, c->d_rods, w.prod, P, w.poff, w.npair, w.pairs, X0, CSN, DF,
                                                   FR1, s, force, A, c->d_status);
                c->launches++;
            }
            prb_b3<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, s, force, contact ? 1 : 0, A);
            c->launches++;
            for (int it = n_iter - 1; it >= 0 && e == cudaSuccess; --it) {
                if (contact) {
                    e = cudaMemsetAsync(A.LTMP, 0, 16 * nV, sm);
                    prb_b4c<<<blocks(P, T), T, 0, sm>>>(c->d_rods, w.prod, P, w.poff, w.npair, w.pairs, X0,
                                                        CSN + (size_t)it * nV, s, force, A, c->d_status);
                    prb_b4a<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, s, force, it == 0 ? 1 : 0, A);
                    c->launches += 2;
                }
                for (int k = 2; k >= 0; --k)
                    prb_b4k<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, X0, PBD + (size_t)it * nE, k, s, force,
                                                         A);
                c->launches += 3;
            }
            prb_b5<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, c->d_kin, c->d_es, X0, Vn, V1, w.POSE, s,
                                               force, A);
            prb_pose<<<blocks(B, T), T, 0, sm>>>(c->scene, c->d_rods, B, s, force, A);
            prb_b8<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, c->d_es, X0, ED, ET, s, force, A);
            prb_b8g<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, s, force, A);
            prb_b7<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, X0, ED, ET, HG, s, force, A);
            c->launches += 5;
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_err(c, e, "plain backward launch");
        }
        prb_frame_end<<<blocks(B, T), T, 0, sm>>>(c->d_rods, B, f, dL_dactions, A);
        c->launches++;
    }
    prb_out<<<blocks(NT, T), T, 0, sm>>>(c->d_rods, V, Et, B, A, reinterpret_cast<float4*>(dL_dx0),
                                         reinterpret_cast<float4*>(dL_dv0), dL_dtheta0, gtb0, gd1b0, dL_dmaterial);
    c->launches++;
    if (c->rec_from_set && dL_dx0) {
        cudaError_t e = launch_frames_adjoint(c->d_rods, B, c->ck.X, gtb0, gd1b0, reinterpret_cast<float4*>(dL_dx0),
                                              work, sm);
        c->launches++;
        if (e != cudaSuccess) return cuda_err(c, e, "frames adjoint launch");
    }
    return check_status(c);
}
