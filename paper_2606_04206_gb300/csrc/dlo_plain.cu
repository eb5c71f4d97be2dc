// dlo_plain.cu -- dlo_step_plain: the same rollout written the plain way, the comparator
// for the persistent kernels.  One kernel launch per phase per substep, one thread per
// element (rod, hinge, vertex, edge or contact-pair slot) across every rod at once, and the
// whole state in HBM between phases; the element functions and the operation order are
// those of the fused substep (dlo_step.cuh), so both follow the same trajectory up to
// rounding.  Self-contact candidates are found once per frame by brute force over each
// rod's edge pairs (the same set the fused kernel's broad phase finds).  It does not record
// a rollout for dlo_backward.
#include <algorithm>
#include <vector>

#include "dlo_kernels.h"
#include "dlo_runtime.h"
#include "dlo_step.cuh"

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
__global__ void pl_broad(const RodInfo* rods, const int* erod, long long Et, const float4* X, const int* poff,
                         int* npair, uint32_t* pairs, unsigned* status) {
    const long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (ge >= Et) return;
    const int b = erod[ge];
    const RodInfo R = rods[b];
    if (!(R.flags & ROD_SELF)) return;
    const bool closed = R.flags & ROD_CLOSED;
    const int a = (int)(ge - R.e0), nv = R.nv, ne = R.ne;
    const int a1 = (a + 1 == nv) ? 0 : a + 1;
    const V3<float> pa0 = f3(X[R.v0 + a]), pa1 = f3(X[R.v0 + a1]);
    bool ovf = false;
    for (int c = a + 1; c < ne; ++c) {
        int sep = c - a;
        if (closed) sep = min(sep, ne - sep);
        if (sep <= R.excl) continue;
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
    if (!closed && i == 1) NDR[R.e0] = f4(H.a.d1r, 0.f);
    HG[gv] = make_float4(hg.x, hg.y, hg.z, H.mref);
}

// vertex phase: forces, symplectic Euler, rigid contact, twist update (one thread per vertex)
__global__ void pl_vertex(SceneDev sc, const RodInfo* rods, const int* vrod, long long V, const float4* KIN,
                          const float2* ES, const float4* X, float4* Vl, float4* ED, float4* ET,
                          const float4* HB0, const float4* HB1, const float4* HB2, const float4* NDR, float4* D,
                          float4* TGT, const float* POSE, const float* act, int s, int force) {
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
    if (has_e) {
        const V3<float> e = f3(X[v0 + ip]) - xi;
        const float ell_i = sqrtf(dot(e, e));
        t_i = e / ell_i;
        if (R.kA > 0.f) {
            const float eb = ES[e0 + i].x;
            g -= (R.kA * (ell_i / eb - 1.f)) * t_i;
        }
    }
    if (R.kA > 0.f && (closed || i >= 1)) {
        const V3<float> e = xi - f3(X[v0 + im]);
        const float ell = sqrtf(dot(e, e));
        const float eb = ES[e0 + im].x;
        g += (R.kA * (ell / eb - 1.f) / ell) * e;
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
        V3<float> d1r = nh > 0 ? f3(NDR[e0 + i]) : zf3();
        if (nh == 0) {
            EdgeF<float> E;
            edge_forward(E, xi, f3(X[v0 + ip]), f3(ET[e0 + i]), f3(ed), ed.w);
            d1r = E.d1r;
        }
        ED[e0 + i] = f4(d1r, ed.w + h * om1);
        ET[e0 + i] = f4(t_i, ES[e0 + i].x);
    }
    TGT[gv] = tgt4;
    D[gv] = f4(d, xi4.w);
    Vl[gv] = f4(v2, om1);
}

// one colour of the inextensibility / strain-limit projection (one thread per edge)
__global__ void pl_inext(const RodInfo* rods, const int* erod, long long Et, const float4* X, float4* D, const float4* ET,
                         int color, int s, int force) {
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
    const float ell = sqrtf(dot(e, e));
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
    if (!active || !(ws > 0.f)) return;
    const float lam = (ell - target) / ws;
    const V3<float> t = e / ell;
    const V3<float> da = (lam * A.w) * t, db = (lam * B.w) * t;
    D[R.v0 + j] = make_float4(A.x + da.x, A.y + da.y, A.z + da.z, A.w);
    D[R.v0 + j1] = make_float4(B.x - db.x, B.y - db.y, B.z - db.z, B.w);
}

// one Jacobi sweep of the self-collision projection (one thread per pair slot)
__global__ void pl_contact(const RodInfo* rods, const int* prod, long long P, const int* poff, const int* npair,
                           const uint32_t* pairs, const float4* X, const float4* D, int4* ACC, float4* FR0,
                           float4* FR1, int first, int s, int force) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = prod[p];
    const RodInfo R = rods[b];
    if (s >= nsub_of(R, force) || p - poff[b] >= min(npair[b], R.pair_cap)) return;
    const int nv = R.nv, v0 = R.v0;
    const uint32_t pr = pairs[p];
    const int a0 = pr & 0xffff, c0 = pr >> 16;
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
                            float4* Vl, int s, int force) {
    const long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gv >= V) return;
    const RodInfo R = rods[vrod[gv]];
    const int n = nsub_of(R, force);
    if (s >= n) return;
    const float ih = 1.f / (sc.dt / (float)n);
    const float4 d = D[gv], v = Vl[gv];
    Vl[gv] = make_float4(d.x * ih, d.y * ih, d.z * ih, v.w);
}

// self-contact friction from the first iteration's contact set (one thread per pair slot)
__global__ void pl_friction(SceneDev sc, const RodInfo* rods, const int* prod, long long P, const int* poff,
                            const int* npair, const uint32_t* pairs, const float4* X, const float4* Vl,
                            const float4* FR0, const float4* FR1, int4* ACC, int s, int force) {
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

}  // namespace
}  // namespace dlo

using namespace dlo;

extern "C" dlo_status dlo_step_plain(dlo_ctx* c, const float* actions, int frames, int substeps) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (frames < 0 || substeps < 0 || substeps > 100000) return set_err(c, DLO_ERR_INVALID_ARG, "bad frames/substeps");
    if (frames == 0) return DLO_OK;
    PlainWs w;
    dlo_status st = plain_workspace(c, w);
    if (st != DLO_OK) return st;
    c->rec_active = false;   // the plain comparator does not record a rollout
    int nsub_max = substeps;
    if (!nsub_max)
        for (int b = 0; b < c->B; ++b) nsub_max = std::max(nsub_max, c->nsub[b]);
    const bool contact = c->opt.self_contact != 0 && w.P > 0;
    const long long V = c->V, Et = c->Et, P = w.P;
    const int B = c->B, T = 128;
    cudaStream_t sm = c->stream;
    for (int f = 0; f < frames; ++f) {
        const float* act = actions ? actions + 12LL * B * f : w.ZACT;
        cudaError_t e = cudaSuccess;
        if (contact) {
            e = cudaMemsetAsync(w.npair, 0, 4 * (size_t)B, sm);
            pl_broad<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, c->S.X, w.poff, w.npair, w.pairs, c->d_status);
            c->launches++;
        }
        for (int s = 0; s < nsub_max; ++s) {
            pl_pose<<<blocks(B, T), T, 0, sm>>>(c->scene, c->d_rods, B, c->S.GP, act, s, substeps, w.POSE);
            pl_hinge<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, c->S.X, c->S.ED, c->S.ET, c->S.HG, w.HB0, w.HB1,
                                                 w.HB2, w.NDR, s, substeps);
            pl_vertex<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, c->d_kin, c->d_es, c->S.X, c->S.Vl,
                                                  c->S.ED, c->S.ET, w.HB0, w.HB1, w.HB2, w.NDR, w.D, w.TGT, w.POSE,
                                                  act, s, substeps);
            c->launches += 3;
            for (int it = 0; it < c->opt.n_iter_pbd; ++it) {
                for (int k = 0; k < 3; ++k)
                    pl_inext<<<blocks(Et, T), T, 0, sm>>>(c->d_rods, w.erod, Et, c->S.X, w.D, c->S.ET, k, s, substeps);
                c->launches += 3;
                if (contact) {
                    pl_contact<<<blocks(P, T), T, 0, sm>>>(c->d_rods, w.prod, P, w.poff, w.npair, w.pairs, c->S.X, w.D,
                                                           w.ACC, w.FR0, w.FR1, it == 0, s, substeps);
                    pl_apply<<<blocks(V, T), T, 0, sm>>>(V, w.ACC, w.D, kFixPos);
                    c->launches += 2;
                }
            }
            pl_velocity<<<blocks(V, T), T, 0, sm>>>(c->scene, c->d_rods, w.vrod, V, w.D, c->S.Vl, s, substeps);
            c->launches++;
            if (contact) {
                pl_friction<<<blocks(P, T), T, 0, sm>>>(c->scene, c->d_rods, w.prod, P, w.poff, w.npair, w.pairs,
                                                        c->S.X, c->S.Vl, w.FR0, w.FR1, w.ACC, s, substeps);
                pl_apply<<<blocks(V, T), T, 0, sm>>>(V, w.ACC, c->S.Vl, kFixVel);
                c->launches += 2;
            }
            pl_finalize<<<blocks(V, T), T, 0, sm>>>(c->d_rods, w.vrod, V, c->S.X, w.D, w.TGT, s, substeps);
            c->launches++;
        }
        pl_pose_advance<<<blocks(B, T), T, 0, sm>>>(c->d_rods, B, c->S.GP, act);
        c->launches++;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(c, e, "plain comparator launch");
    }
    pl_status<<<blocks(B, T), T, 0, sm>>>(c->d_rods, B, c->S.X, c->S.Vl, c->d_status);
    c->launches++;
    c->from_set_state = false;
    return cuda_err(c, cudaGetLastError(), "plain comparator launch");
}
