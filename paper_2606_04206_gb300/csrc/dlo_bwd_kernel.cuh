// dlo_bwd_kernel.cuh -- hand-written adjoint of the rod stepper with gradient checkpointing.
//
// DLO-Lab (Sec. 3.3) differentiates whole trajectories by caching one state per segment and,
// for each segment in reverse, re-running the forward simulation before back-propagating.
// Here the checkpoints live in HBM (written by the forward kernel every K frames) and the
// rollout is reversed in chunks of frames, last first, by two persistent kernels per chunk:
//   rec_kernel   forward-like (several rods per CTA): re-runs the chunk's frames from their
//                start state and stores every substep's records in HBM: its start state, the
//                velocity before rigid contact, the displacement before friction, one record
//                per edge and projection iteration (direction and target / length), the
//                displacements before each contact sweep and the first iteration's pair data;
//                for checkpoints more than a chunk apart it first stores the start state of
//                each of the segment's frames
//   rev_kernel   one group per rod: for each frame and substep, last first, loads the records
//                and applies the vector-Jacobian product of every phase in reverse order; the
//                cotangents of the rod's state are carried to the next chunk in HBM
// Second-order terms of the elastic forces are exact: the hinge gradient (a hand reverse pass)
// is re-run on dual numbers, giving d/de [dU/dz](x + e lambda) for every input z, which is
// the transpose-Jacobian product of the force (U's Hessian is symmetric).  Branches (contact
// on/off, yield, strain-limit activity, pair sets) follow the recomputed forward.
#pragma once
#include "dlo_fwd_kernel.cuh"

namespace dlo {

// Threads per CTA the reverse kernel is compiled for (its register budget).  Rods of up to 128
// vertices take at most 62.5 KB of shared memory each, so three fit an SM: 384 threads at 168
// registers.  Larger rods fit two per SM (one at 256 vertices), and keep 255 registers.
__host__ __device__ constexpr int rev_max_threads(int NV) { return NV <= 128 ? 384 : 256; }

__host__ __device__ constexpr size_t bwd_smem_bytes(int NV, bool contact) {
    return rod_smem_bytes(NV, contact) + (size_t)(10 * NV + 20) * 16;
}

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ void atomic_add3(float4* a, V3<float> v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
    atomicAdd(&a->z, v.z);
}

// J_l(phi)^T lam for the left Jacobian of the rotation exponential:
// exp([phi + d]x) ~ exp([J_l(phi) d]x) exp([phi]x),  J_l = I + A [phi]x + B [phi]x^2.
__device__ __forceinline__ V3<float> jl_t(V3<float> phi, V3<float> lam) {
    float t2 = dot(phi, phi), A, B;
    if (t2 < 1e-8f) {
        A = 0.5f - t2 / 24.f;
        B = 1.f / 6.f - t2 / 120.f;
    } else {
        float t = sqrtf(t2), sh = sinf(0.5f * t);
        A = 2.f * sh * sh / t2;
        B = (t - sinf(t)) / (t2 * t);
    }
    V3<float> c = cross(phi, lam);
    return lam - A * c + B * cross(phi, c);
}

// The linear maps that carry gripper q's substep pose cotangents to the frame's actions and
// start pose (see the pose block of reverse_substep), per gripper: M0 = exp(c0 dphi),
// M1 = exp(c1 dphi), c0 J_l(c0 dphi)^T and c1 J_l(c1 dphi)^T (row major, 9 floats each).  Thread
// t < 4 ngrip builds matrix t % 4 of gripper t / 4, so the eight run side by side.  With
// phi = c dphi: J_l(phi)^T = I - A [phi]x + B [phi]x^2, the coefficients of jl_t above.
__device__ __forceinline__ void pose_rev_mat(const float* act, int t, float c0, float c1, float* pm) {
    const int q = t >> 2, m = t & 3;
    const float c = (m & 1) ? c1 : c0;
    const V3<float> phi = c * f3(act[6 * q + 3], act[6 * q + 4], act[6 * q + 5]);
    float* o = pm + 36 * q + 9 * m;
    if (m < 2) {
        const M3 M = expmap(phi);
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = M.m[k];
        return;
    }
    const float t2 = dot(phi, phi);
    float A, B;
    if (t2 < 1e-8f) {
        A = 0.5f - t2 / 24.f;
        B = 1.f / 6.f - t2 / 120.f;
    } else {
        const float th = sqrtf(t2), sh = sinf(0.5f * th);
        A = 2.f * sh * sh / t2;
        B = (th - sinf(th)) / (t2 * th);
    }
    const float p[3] = {phi.x, phi.y, phi.z};
    const float d = 1.f - B * t2;
    // [phi]x = [[0, -z, y], [z, 0, -x], [-y, x, 0]]
    const float K[9] = {0.f, -phi.z, phi.y, phi.z, 0.f, -phi.x, -phi.y, phi.x, 0.f};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) o[3 * r + k] = c * ((r == k ? d : 0.f) - A * K[3 * r + k] + B * p[r] * p[k]);
}

// One rigid primitive acting on a vertex velocity (the k-th of planes, boxes, grippers).
template <class T>
__device__ __forceinline__ V3<T> prim_respond(int k, const SceneDev& sc, const RodInfo& R, V3<T> x, V3<T> v,
                                              V3<T> gp, V3<T> gax, V3<T> vp, V3<T> w, bool& act) {
    V3<T> n;
    T sdf;
    V3<T> vrig = zero3<T>();
    if (k < sc.n_planes) {
        n = mk3(cst<T>(sc.planes[k].x), cst<T>(sc.planes[k].y), cst<T>(sc.planes[k].z));
        sdf = dot(x, n) - sc.planes[k].w;
    } else if (k < sc.n_planes + sc.n_boxes) {
        const int b = k - sc.n_planes;
        sdf = sdf_box(x, f3(sc.box_c[b]), f3(sc.box_h[b]), n);
    } else {
        V3<T> a = gp - sc.grip_hl * gax, bb = gp + sc.grip_hl * gax;
        if (capsule_far(vals(x), vals(a), vals(bb), sc.grip_r + R.radius + kContactReach * R.eps)) {
            act = false;
            return v;
        }
        sdf = sdf_capsule(x, a, bb, sc.grip_r, n);
        vrig = vp + cross(w, x - gp);
    }
    return contact_respond(v, sdf, n, vrig, R.radius, R.eps, sc.mu_rigid, sc.restitution, act);
}

template <int NV, bool CONTACT>
struct AdjArrays {
    float4 *LX, *LD, *LV, *LE, *LT, *LK, *LP0, *LG, *V1, *DF;
    float* PM;   // per gripper (36): the substep's M0, M1, c0 J_l(c0 dphi)^T, c1 J_l(c1 dphi)^T (row major)
    __device__ AdjArrays(float4* a) {
        LX = a;
        LD = a + NV;
        LV = a + 2 * NV;
        LE = a + 3 * NV;
        LT = a + 4 * NV;
        LK = a + 5 * NV;
        LP0 = a + 6 * NV;
        LG = a + 7 * NV;
        V1 = a + 8 * NV;
        DF = a + 9 * NV;
        PM = reinterpret_cast<float*>(a + 10 * NV);
    }
};

// State snapshot layout in the per-rod scratch: X[NV], V[NV], HG[NV], ED[NV], ET[NV].
template <int NV, bool C, int TPR>
__device__ __forceinline__ void save_state(float4* dst, const RodInfo& R, const Grp<TPR>& g, const Smem<NV, C>& s) {
    for (int i = g.tid; i < R.nv; i += TPR) {
        dst[i] = s.X0[i];
        dst[NV + i] = s.V[i];
        dst[2 * NV + i] = s.HG[i];
    }
    for (int j = g.tid; j < R.ne; j += TPR) {
        dst[3 * NV + j] = s.ED[j];
        dst[4 * NV + j] = s.ET[j];
    }
}
template <int NV, bool C, int TPR>
__device__ __forceinline__ void load_state(const float4* src, const RodInfo& R, const Grp<TPR>& g, Smem<NV, C>& s) {
    for (int i = g.tid; i < R.nv; i += TPR) {
        float4 x = src[i];
        s.X0[i] = x;
        s.X[i] = x;
        s.V[i] = src[NV + i];
        s.HG[i] = src[2 * NV + i];
    }
    for (int j = g.tid; j < R.ne; j += TPR) {
        s.ED[j] = src[3 * NV + j];
        s.ET[j] = src[4 * NV + j];
    }
    g.sync();
}

// Per-g.tid pose cotangents of one substep (two grippers x 3).
struct PoseAdj {
    float ps0[6], phs0[6], ps1[6], phs1[6], vp[6], w[6];
    __device__ void zero() {
#pragma unroll
        for (int k = 0; k < 6; ++k) ps0[k] = phs0[k] = ps1[k] = phs1[k] = vp[k] = w[k] = 0.f;
    }
};
// gripper q in {0, 1}; both halves are addressed with constant indices so that the per-thread
// arrays stay in registers
__device__ __forceinline__ void add3(float* a, int q, V3<float> v) {
    if (q == 0) {
        a[0] += v.x;
        a[1] += v.y;
        a[2] += v.z;
    } else {
        a[3] += v.x;
        a[4] += v.y;
        a[5] += v.z;
    }
}
__device__ __forceinline__ V3<float> get3(const float* a, int q) {
    return q == 0 ? f3(a[0], a[1], a[2]) : f3(a[3], a[4], a[5]);
}
// row-major 3x3 at o times v
__device__ __forceinline__ V3<float> mul_rm(const float* o, V3<float> v) {
    return f3(o[0] * v.x + o[1] * v.y + o[2] * v.z, o[3] * v.x + o[4] * v.y + o[5] * v.z,
              o[6] * v.x + o[7] * v.y + o[8] * v.z);
}

// The dual-number frames of a rod's edges (7 float4 per edge) and the seeds the hinges send
// back to each edge (3 float4 per edge, accumulated with shared-memory atomics), kept in ten
// per-edge arrays that the substep's reverse no longer uses when it reaches its hinges.
struct EdgeDual {
    float4 *tv, *td, *wv, *wd, *rv, *rd, *cs;   // t | ell, w0 | n1, d1r | c (values, derivatives); s
    float4 *s0, *s1, *s2;                       // seeds: gt.v | gd1r.x.v, gt.d | gd1r.x.d, gd1r.yz (v, d)
    __device__ __forceinline__ void store(int j, const EdgeF<dualf>& E) const {
        tv[j] = make_float4(E.t.x.v, E.t.y.v, E.t.z.v, E.ell.v);
        td[j] = make_float4(E.t.x.d, E.t.y.d, E.t.z.d, E.ell.d);
        wv[j] = make_float4(E.w0.x.v, E.w0.y.v, E.w0.z.v, E.n1.v);
        wd[j] = make_float4(E.w0.x.d, E.w0.y.d, E.w0.z.d, E.n1.d);
        rv[j] = make_float4(E.d1r.x.v, E.d1r.y.v, E.d1r.z.v, E.c.v);
        rd[j] = make_float4(E.d1r.x.d, E.d1r.y.d, E.d1r.z.d, E.c.d);
        cs[j] = make_float4(E.s.v, E.s.d, 0.f, 0.f);
    }
    // what the hinge needs: t, d1r, d2r = t x d1r, the material frame (d1, d2) and (c, s)
    __device__ __forceinline__ void load_frame(int j, EdgeF<dualf>& E) const {
        const float4 a = tv[j], b = td[j], c = rv[j], d = rd[j], e = cs[j];
        E.t = mk3(mkd(a.x, b.x), mkd(a.y, b.y), mkd(a.z, b.z));
        E.d1r = mk3(mkd(c.x, d.x), mkd(c.y, d.y), mkd(c.z, d.z));
        E.c = mkd(c.w, d.w);
        E.s = mkd(e.x, e.y);
        E.d2r = cross(E.t, E.d1r);
        E.d1 = E.c * E.d1r + E.s * E.d2r;
        E.d2 = E.c * E.d2r - E.s * E.d1r;
    }
    // what edge_reverse needs: t, w0, d1r, n1, ell
    __device__ __forceinline__ void load_rev(int j, EdgeF<dualf>& E) const {
        const float4 a = tv[j], b = td[j], c = wv[j], d = wd[j], e = rv[j], f = rd[j];
        E.t = mk3(mkd(a.x, b.x), mkd(a.y, b.y), mkd(a.z, b.z));
        E.ell = mkd(a.w, b.w);
        E.w0 = mk3(mkd(c.x, d.x), mkd(c.y, d.y), mkd(c.z, d.z));
        E.n1 = mkd(c.w, d.w);
        E.d1r = mk3(mkd(e.x, f.x), mkd(e.y, f.y), mkd(e.z, f.z));
    }
    __device__ __forceinline__ void zero_seeds(int j) const {
        s0[j] = s1[j] = s2[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ __forceinline__ void add_seeds(int j, V3<dualf> gt, V3<dualf> gr) const {
        atomicAdd(&s0[j].x, gt.x.v);
        atomicAdd(&s0[j].y, gt.y.v);
        atomicAdd(&s0[j].z, gt.z.v);
        atomicAdd(&s0[j].w, gr.x.v);
        atomicAdd(&s1[j].x, gt.x.d);
        atomicAdd(&s1[j].y, gt.y.d);
        atomicAdd(&s1[j].z, gt.z.d);
        atomicAdd(&s1[j].w, gr.x.d);
        atomicAdd(&s2[j].x, gr.y.v);
        atomicAdd(&s2[j].y, gr.z.v);
        atomicAdd(&s2[j].z, gr.y.d);
        atomicAdd(&s2[j].w, gr.z.d);
    }
    __device__ __forceinline__ void load_seeds(int j, V3<dualf>& gt, V3<dualf>& gr) const {
        const float4 a = s0[j], b = s1[j], c = s2[j];
        gt = mk3(mkd(a.x, b.x), mkd(a.y, b.y), mkd(a.z, b.z));
        gr = mk3(mkd(a.w, b.w), mkd(c.x, c.z), mkd(c.y, c.w));
    }
};

// The values of a dual-number edge frame.
__device__ __forceinline__ EdgeF<float> edge_vals(const EdgeF<dualf>& D) {
    EdgeF<float> E;
    E.t = vals(D.t);
    E.w0 = vals(D.w0);
    E.d1r = vals(D.d1r);
    E.d2r = vals(D.d2r);
    E.d1 = vals(D.d1);
    E.d2 = vals(D.d2);
    E.ell = D.ell.v;
    E.n1 = D.n1.v;
    E.c = D.c.v;
    E.s = D.s.v;
    return E;
}

// ------------------------------------------------------------------ reverse of one substep
// On entry the shared state holds S_n (the substep's start), the recorded intermediates and,
// for a self-contact rod, the frame's pair list and the projection data of the first
// iteration; the cotangent arrays hold the cotangents of S_{n+1}.  On exit they hold those
// of S_n.  PBD: the substep's projection records ([n_iter][NV], see Rec::pbd); CSN: its
// displacements before each contact sweep ([n_iter][NV]).  gm accumulates (kA, Bm, beta,
// sigma_y, c_d) cotangents, lpf/lphif the frame-start pose cotangents and ga the frame's
// action cotangents (all per g.tid).
template <int NV, bool CONTACT, int TPR>
__device__ __noinline__ void reverse_substep(const BwdParams& P, const RodInfo& R, Smem<NV, CONTACT>& s,
                                AdjArrays<NV, CONTACT>& a, const float4* PBD, const float4* CSN, const Grp<TPR>& g,
                                float h, float c0, float c1, int np,
                                double* gm, float* lpf, float* lphif, float* ga) {
    const SceneDev& sc = P.scene;
    const int nv = R.nv, ne = R.ne, v0 = R.v0, e0 = R.e0;
    const bool closed = R.flags & ROD_CLOSED;
    const int nh = closed ? nv : nv - 2;
    const float ih = 1.f / h;
    const bool lenc = R.flags & (ROD_INEXT | ROD_SLIMIT);
    const float rsum = 2.f * R.radius;
    PoseAdj pa;
    pa.zero();
    // this substep's material terms, in registers (gm is the caller's memory), added to gm at
    // the end
    double gl[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = g.tid; i < nv; i += TPR) a.LP0[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    // ---- B1: positions at the substep end
    for (int i = g.tid; i < nv; i += TPR) {
        const float4 kin = P.KIN[v0 + i];
        const int kind = (int)kin.w;
        float4 lx = a.LX[i];
        if (kind >= 2 && in_bounds(kind - 2 < R.ngrip, s.red)) {
            const int q = kind - 2;
            V3<float> y1 = mul_rm(s.sp + 32 * q + 15, f3(kin));
            add3(pa.ps1, q, f3(lx));
            add3(pa.phs1, q, cross(y1, f3(lx)));
            a.LX[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.LD[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            a.LD[i] = make_float4(lx.x, lx.y, lx.z, 0.f);
        }
    }
    g.sync();
    // ---- B2: self-contact friction
    if (CONTACT && np > 0) {
        // displacements at the first contact sweep (after the colours of iteration 0)
        const float4* T0 = CSN;
        float4* LTMP = s.HB0;
        for (int i = g.tid; i < nv; i += TPR) LTMP[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        g.sync();
        for (int p = g.tid; p < np; p += TPR) {
            if (!(s.fr1[p].w > 0.f)) continue;
            uint32_t pr = s.pairs[p];
            const int a0 = pr & 0xffff, q0 = pr >> 16;
            if (!in_bounds(a0 < nv && q0 < nv, s.red)) continue;
            const int idx[4] = {a0, (a0 + 1 == nv) ? 0 : a0 + 1, q0, (q0 + 1 == nv) ? 0 : q0 + 1};
            const V3<float> o = f3(s.X0[a0]);
            V3<float> Pf[4], Vf[4], lo[4];
            float w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                Pf[k] = (k == 0) ? f3(T0[idx[0]]) : (f3(s.X0[idx[k]]) - o) + f3(T0[idx[k]]);
                Vf[k] = ih * f3(a.DF[idx[k]]);
                w[k] = s.X0[idx[k]].w;
                lo[k] = f3(a.LV[idx[k]]);
            }
            V3<float> pb[4], vb[4];
            if (fric_pair_vjp(Pf, Vf, w, rsum, sc.mu_self, h, lo, pb, vb))
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    atomic_add3(&a.LP0[idx[k]], pb[k]);
                    atomic_add3(&LTMP[idx[k]], vb[k]);
                }
        }
        g.sync();
        for (int i = g.tid; i < nv; i += TPR) {
            float4 l = a.LV[i], t = LTMP[i];
            a.LV[i] = make_float4(l.x + t.x, l.y + t.y, l.z + t.z, l.w);
        }
        g.sync();
    }
    // ---- B3: velocity rebuilt from the displacement
    for (int i = g.tid; i < nv; i += TPR) {
        const float4 kin = P.KIN[v0 + i];
        const int kind = (int)kin.w;
        (void)kin;
        (void)kind;
        float4 l = a.LV[i];
        V3<float> lv = ih * f3(l);
        float4 d = a.LD[i];
        a.LD[i] = make_float4(d.x + lv.x, d.y + lv.y, d.z + lv.z, 0.f);
        a.LV[i] = make_float4(0.f, 0.f, 0.f, l.w);
    }
    g.sync();
    // ---- B4: PBD iterations in reverse
    if (lenc || (CONTACT && np > 0)) {
        const int ncol = lenc ? ((closed && (ne & 1)) ? 3 : 2) : 0;
        for (int it = sc.n_iter - 1; it >= 0; --it) {
            if (CONTACT && np > 0) {
                const float4* Dc = CSN + (size_t)it * NV;   // displacements before the contact sweep
                float4* LTMP = a.LG;
                for (int i = g.tid; i < nv; i += TPR) LTMP[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                g.sync();
                for (int p = g.tid; p < np; p += TPR) {
                    uint32_t pr = s.pairs[p];
                    const int a0 = pr & 0xffff, q0 = pr >> 16;
                    if (!in_bounds(a0 < nv && q0 < nv, s.red)) continue;
                    const int idx[4] = {a0, (a0 + 1 == nv) ? 0 : a0 + 1, q0, (q0 + 1 == nv) ? 0 : q0 + 1};
                    const V3<float> o = f3(s.X0[a0]);
                    V3<float> Pf[4], lo[4];
                    float w[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        Pf[k] = (k == 0) ? f3(Dc[idx[0]]) : (f3(s.X0[idx[k]]) - o) + f3(Dc[idx[k]]);
                        w[k] = s.X0[idx[k]].w;
                        lo[k] = f3(a.LD[idx[k]]);
                    }
                    V3<float> pb[4];
                    if (pair_correction_vjp(Pf, w, rsum, lo, pb))
#pragma unroll
                        for (int k = 0; k < 4; ++k) atomic_add3(&LTMP[idx[k]], pb[k]);
                }
                g.sync();
                for (int i = g.tid; i < nv; i += TPR) {
                    float4 t = LTMP[i];
                    if (it == 0) {
                        float4 q = a.LP0[i];
                        t = make_float4(t.x + q.x, t.y + q.y, t.z + q.z, 0.f);
                    }
                    float4 ld = a.LD[i], lx = a.LX[i];
                    a.LD[i] = make_float4(ld.x + t.x, ld.y + t.y, ld.z + t.z, 0.f);
                    a.LX[i] = make_float4(lx.x + t.x, lx.y + t.y, lx.z + t.z, 0.f);
                }
                g.sync();
            }
            // colours in reverse, from each edge's record (unit direction t, ratio r = target /
            // length): the projection moved its ends by -+ w lambda t, lambda = (l - target) / ws
            const float4* Q = PBD + (size_t)it * NV;
            for (int k = ncol - 1; k >= 0; --k) {
                int first, last;
                color_range(ne, closed, k, first, last);
                for (int j = first + 2 * g.tid; j < last; j += 2 * TPR) {
                    const int j1 = (j + 1 == nv) ? 0 : j + 1;
                    const float4 q = Q[j];
                    if (q.x == 0.f && q.y == 0.f && q.z == 0.f) continue;   // the projection did nothing
                    const float wa = s.X0[j].w, wb = s.X0[j1].w, ws = wa + wb;
                    const V3<float> t = f3(q);
                    V3<float> la = f3(a.LD[j]), lb = f3(a.LD[j1]);
                    V3<float> mu = (wa / ws) * la - (wb / ws) * lb;
                    V3<float> le = mu - q.w * (mu - dot(mu, t) * t);
                    a.LD[j] = f4(la - le, 0.f);
                    a.LD[j1] = f4(lb + le, 0.f);
                    a.LX[j] = f4(f3(a.LX[j]) - le, 0.f);
                    a.LX[j1] = f4(f3(a.LX[j1]) + le, 0.f);
                }
                g.sync();
            }
        }
    }
    // ---- B5: vertex phase (rigid contact, symplectic Euler, gravity, damping, twist rate)
    for (int i = g.tid; i < nv; i += TPR) {
        const float4 kin = P.KIN[v0 + i];
        const int kind = (int)kin.w;
        const float4 x4 = s.X0[i];
        const float4 vn = s.V[i];
        V3<float> ld0 = f3(a.LD[i]);
        float4 lvn = make_float4(0.f, 0.f, 0.f, 0.f), lg = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kind == 0) {
            V3<float> lam = h * ld0;
            // forward sequence of the rigid primitives from the recorded pre-contact velocity
            const int nprim = sc.n_planes + sc.n_boxes + R.ngrip;
            V3<float> vs[kMaxPlanes + kMaxBoxes + 2];
            vs[0] = f3(a.V1[i]);
            const V3<float> x = f3(x4);
            unsigned onmask = 0;
            for (int k = 0; k < nprim; ++k) {
                const int q = k - sc.n_planes - sc.n_boxes;
                V3<float> gp = zf3(), gax = zf3(), vp = zf3(), w = zf3();
                if (q >= 0) {
                    const float* o = s.sp + 32 * q;
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
                    const float* o = s.sp + 32 * q;
                    gp = f3(o[0], o[1], o[2]);
                    gax = f3(o[8], o[11], o[14]);
                    vp = f3(o[24], o[25], o[26]);
                    w = f3(o[27], o[28], o[29]);
                }
                V3<float> ntmp;
                if (q >= 0 && sdf_capsule(x, gp - sc.grip_hl * gax, gp + sc.grip_hl * gax, sc.grip_r, ntmp) > -sc.grip_r) {
                    // capsule gripper: closed-form reverse (the degenerate on-axis case keeps dual numbers)
                    V3<float> lxk, lvk, lpk, lphik, lvpk, lwk;
                    capsule_contact_rev(x, vs[k], gp, gax, sc.grip_hl, sc.grip_r, vp, w, R.radius, R.eps,
                                        sc.mu_rigid, sc.restitution, lam, lxk, lvk, lpk, lphik, lvpk, lwk);
                    lx_acc += lxk;
                    lam = lvk;
                    add3(pa.ps0, q, lpk);
                    add3(pa.phs0, q, lphik);
                    add3(pa.vp, q, lvpk);
                    add3(pa.w, q, lwk);
                    continue;
                }
                if (k < sc.n_planes) {   // plane: closed-form reverse (sdf = n.x - o, constant n)
                    const V3<float> n = f3(sc.planes[k]);
                    V3<float> lv, ln, lvr;
                    float lsdf;
                    contact_respond_rev(vs[k], dot(x, n) - sc.planes[k].w, n, zf3(), R.radius, R.eps, sc.mu_rigid,
                                        sc.restitution, lam, lv, lsdf, ln, lvr);
                    lx_acc += lsdf * n;
                    lam = lv;
                    continue;
                }
                if (q < 0) {   // box: closed-form reverse
                    const int bi = k - sc.n_planes;
                    V3<float> lv;
                    lx_acc += box_contact_rev(x, vs[k], f3(sc.box_c[bi]), f3(sc.box_h[bi]), R.radius, R.eps,
                                              sc.mu_rigid, sc.restitution, lam, lv);
                    lam = lv;
                    continue;
                }
                const int nin = 18;   // the degenerate on-axis gripper contact keeps dual numbers
                float lin[18];
#pragma unroll 1
                for (int d = 0; d < nin; ++d) {
                    V3<float> e = zf3();
                    (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
                    const int g = d / 3;
                    V3<dualf> xd = lift(x, g == 0 ? e : zf3()), vd = lift(vs[k], g == 1 ? e : zf3());
                    V3<dualf> gpd = lift(gp, g == 2 ? e : zf3()), gaxd = lift(gax, g == 3 ? cross(e, gax) : zf3());
                    V3<dualf> vpd = lift(vp, g == 4 ? e : zf3()), wd = lift(w, g == 5 ? e : zf3());
                    bool on2;
                    V3<dualf> out = prim_respond<dualf>(k, sc, R, xd, vd, gpd, gaxd, vpd, wd, on2);
                    lin[d] = dot(ders(out), lam);
                }
                lx_acc += f3(lin[0], lin[1], lin[2]);
                lam = f3(lin[3], lin[4], lin[5]);
                add3(pa.ps0, q, f3(lin[6], lin[7], lin[8]));
                add3(pa.phs0, q, f3(lin[9], lin[10], lin[11]));
                add3(pa.vp, q, f3(lin[12], lin[13], lin[14]));
                add3(pa.w, q, f3(lin[15], lin[16], lin[17]));
            }
            // v1 = v + h (-w g + gravity - c_d v)
            const float wi = x4.w;
            lvn = f4((1.f - h * R.cd) * lam, 0.f);
            lg = f4((-h * wi) * lam, 0.f);
            gl[4] += (double)(-h * dot(f3(vn), lam));
            a.LX[i] = f4(f3(a.LX[i]) + lx_acc, 0.f);
        } else if (kind >= 2 && in_bounds(kind - 2 < R.ngrip, s.red)) {
            // d = target(pose at the substep end) - x0
            const int q = kind - 2;
            add3(pa.ps1, q, ld0);
            add3(pa.phs1, q, cross(mul_rm(s.sp + 32 * q + 15, f3(kin)), ld0));
            a.LX[i] = f4(f3(a.LX[i]) - ld0, 0.f);
        }
        const bool has_e = closed || i < nv - 1;
        if (has_e) {
            const float lw1 = a.LV[i].w + h * a.LE[i].w;     // d theta_{n+1} / d omega_1 = h
            const float invI = P.ES[e0 + i].y;
            lvn.w = (1.f - h * R.cd) * lw1;
            lg.w = -h * invI * lw1;
            gl[4] += (double)(-h * vn.w * lw1);
        }
        a.LV[i] = lvn;
        a.LG[i] = lg;
    }
    g.sync();
    // ---- pose cotangents of this substep -> frame-start pose and the frame's actions (pa is
    // complete after B5; folding it here ends its registers' life before B8 and B7).  Only
    // grasped vertices and vertices touching a gripper have any; the maps are a.PM's.
    const float idt = 1.f / sc.dt;
    for (int q = 0; q < R.ngrip; ++q) {
        const V3<float> ps0 = get3(pa.ps0, q), ps1 = get3(pa.ps1, q), vp = get3(pa.vp, q);
        const V3<float> ph0 = get3(pa.phs0, q), ph1 = get3(pa.phs1, q), w = get3(pa.w, q);
        const bool nz = ps0.x != 0.f || ps0.y != 0.f || ps0.z != 0.f || ps1.x != 0.f || ps1.y != 0.f ||
                        ps1.z != 0.f || vp.x != 0.f || vp.y != 0.f || vp.z != 0.f || ph0.x != 0.f ||
                        ph0.y != 0.f || ph0.z != 0.f || ph1.x != 0.f || ph1.y != 0.f || ph1.z != 0.f ||
                        w.x != 0.f || w.y != 0.f || w.z != 0.f;
        if (!nz) continue;
        const float* pm = a.PM + 36 * q;
        add3(lpf, q, ps0 + ps1);
        const V3<float> gdp = c0 * ps0 + c1 * ps1 + idt * vp;
        const V3<float> gdr = mul_rm(pm + 18, ph0) + mul_rm(pm + 27, ph1) + idt * w;
        ga[6 * q] += gdp.x;
        ga[6 * q + 1] += gdp.y;
        ga[6 * q + 2] += gdp.z;
        ga[6 * q + 3] += gdr.x;
        ga[6 * q + 4] += gdr.y;
        ga[6 * q + 5] += gdr.z;
        const V3<float> m0 = f3(pm[0] * ph0.x + pm[3] * ph0.y + pm[6] * ph0.z,
                                pm[1] * ph0.x + pm[4] * ph0.y + pm[7] * ph0.z,
                                pm[2] * ph0.x + pm[5] * ph0.y + pm[8] * ph0.z);
        const V3<float> m1 = f3(pm[9] * ph1.x + pm[12] * ph1.y + pm[15] * ph1.z,
                                pm[10] * ph1.x + pm[13] * ph1.y + pm[16] * ph1.z,
                                pm[11] * ph1.x + pm[14] * ph1.y + pm[17] * ph1.z);
        add3(lphif, q, m0 + m1);
    }
    // ---- B8: per edge, the reverse of the new reference-frame base and the stretching second
    // order; and the edge's frame as dual numbers in the direction of the force cotangents LG,
    // once per edge, for the hinge phase (B7).  Arrays dead after B5 hold the dual frames
    // (EdgeDual) and the seeds the two hinges of an edge send back to it (zeroed here).
    const bool strands = R.flags & ROD_STRANDS;
    const EdgeDual ES{a.LD, a.LP0, a.V1, a.DF, s.X, s.V, s.HB0, s.HB1, s.HB2, s.ND};
    // Each thread keeps its edges' position cotangents (this phase's and B7's) in registers and
    // adds them up per vertex in a fixed order at the end: no floating-point atomics, so the
    // reverse of a substep without contact candidates is bitwise reproducible.
    constexpr int EPT = (NV + TPR - 1) / TPR;   // edges per thread
    V3<float> le_keep[EPT];
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
        const int j = g.tid + m * TPR;
        le_keep[m] = zf3();
        if (j >= ne) continue;
        const int j1 = (j + 1 == nv) ? 0 : j + 1;
        const float4 ed = s.ED[j], et = s.ET[j];
        ES.zero_seeds(j);
        if (strands && !(et.w > 0.f)) continue;   // a break edge kept its base frame: identity reverse
        const float4 lga = a.LG[j], lgb = a.LG[j1];
        EdgeF<dualf> Ed;
        edge_forward(Ed, lift(f3(s.X0[j]), f3(lga)), lift(f3(s.X0[j1]), f3(lgb)), lift(f3(et)), lift(f3(ed)),
                     mkd(ed.w, lga.w));
        ES.store(j, Ed);
        const EdgeF<float> E = edge_vals(Ed);
        V3<float> gtb, gd1b;
        V3<float> le = edge_reverse<float, true>(E, f3(et), f3(ed), f3(a.LT[j]), f3(a.LE[j]), 0.f, &gtb, &gd1b);
        if (R.kA > 0.f) {
            const V3<float> les = f3(lgb) - f3(lga);
            const float eb = P.ES[e0 + j].x;
            const float tl = dot(E.t, les);
            const float st = edge_strain(f3(s.X0[j1]) - f3(s.X0[j]), eb);
            le += R.kA * ((tl / eb) * E.t + st / E.ell * (les - tl * E.t));
            gl[0] += (double)(st * tl);
        }
        le_keep[m] = le;
        a.LT[j] = f4(gtb, 0.f);
        a.LE[j] = f4(gd1b, a.LE[j].w);
    }
    g.sync();
    // ---- B7: hinges: force second order (dual numbers), plasticity, its first-order reverse.
    // The hinge's own part runs here; the reverse through its edges' frames runs per edge below
    // on the sum of the seeds of both hinges of the edge (the reverse is linear in them).
    for (int k = g.tid; k < nh; k += TPR) {
        const int i = closed ? k : k + 1;
        const int ea = (i == 0) ? ne - 1 : i - 1, eb = i;
        const float4 ETa = s.ET[ea], ETb = s.ET[eb], hg = s.HG[i];
        if (strands && !(ETa.w > 0.f && ETb.w > 0.f)) continue;   // inactive: at an end of a break edge
        const float lbar = 0.5f * (ETa.w + ETb.w), il = 1.f / lbar;
        // second order of the elastic force: tangents = cotangents of the gradient
        HingeF<dualf> Hd;
        ES.load_frame(ea, Hd.a);
        ES.load_frame(eb, Hd.b);
        hinge_core_forward(Hd, mkd(s.ED[ea].w, a.LG[ea].w), mkd(s.ED[eb].w, a.LG[eb].w), mkd(hg.w));
        const float hk0 = Hd.k0.v, hk1 = Hd.k1.v;   // the hinge's material curvature (for plasticity)
        float kb0 = hg.x, kb1 = hg.y;
        const bool plastic = R.flags & ROD_PLASTIC;
        const bool yielded = plastic && plastic_update(hk0, hk1, kb0, kb1, R.sy * lbar, R.rc);
        dualf e0d = Hd.k0 - kb0, e1d = Hd.k1 - kb1, emd = Hd.m - hg.z;
        dualf gk0 = (R.Bm * il) * e0d, gk1 = (R.Bm * il) * e1d, gmt = (R.beta * il) * emd;
        // each term in float, added to the FP64 sums (the cancellation is across terms)
        gl[1] += (double)(il * (e0d.v * e0d.d + e1d.v * e1d.d));
        gl[2] += (double)(il * emd.v * emd.d);
        // rest curvature: cotangent of the one used (-d gk / d .) plus the carried one
        float lk0 = a.LK[i].x - gk0.d, lk1 = a.LK[i].y - gk1.d;
        if (yielded) {
            const float el0 = hk0 - hg.x, el1 = hk1 - hg.y;
            const float n = sqrtf(el0 * el0 + el1 * el1), thr = R.sy * lbar;
            const float g = R.rc * (n - thr) / n;
            const float kk = R.rc * thr / (n * n * n) * (el0 * lk0 + el1 * lk1);
            const float le0 = g * lk0 + kk * el0, le1 = g * lk1 + kk * el1;     // cotangent of kappa_el
            gl[3] += (double)(-R.rc * lbar * (el0 * lk0 + el1 * lk1) / n);
            // The first-order reverse of kappa from seeds (le0, le1) is needed too.  The hinge
            // reverse is linear in its seeds, so adding them to the derivative part of the
            // dual seeds makes the reverse below return J^T le on top of the Hessian term.
            gk0.d += le0;
            gk1.d += le1;
            lk0 -= le0;
            lk1 -= le1;
        }
        V3<dualf> gta, gd1ra, gtb, gd1rb;
        dualf ghta, ghtb;
        hinge_core_reverse(Hd, gk0, gk1, gmt, mkd(0.f), gta, gd1ra, gtb, gd1rb, ghta, ghtb);
        ES.add_seeds(ea, gta, gd1ra);
        ES.add_seeds(eb, gtb, gd1rb);
        atomicAdd(&ES.cs[ea].z, ghta.d);   // two terms per edge, added to zero: order-free
        atomicAdd(&ES.cs[eb].z, ghtb.d);
        a.LK[i] = make_float4(lk0, lk1, 0.f, 0.f);
    }
    g.sync();
    // ---- B7, per edge: the reverse through the edge's frame (vertices and base frame); the
    // edge's total position cotangent goes to s0 (its own slot, after its seeds are read)
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
        const int j = g.tid + m * TPR;
        if (j >= ne) continue;
        const float4 et = s.ET[j];
        V3<float> tot = le_keep[m];
        if (!(strands && !(et.w > 0.f))) {
            V3<dualf> gt, gd1r;
            ES.load_seeds(j, gt, gd1r);
            EdgeF<dualf> Ed;
            ES.load_rev(j, Ed);
            V3<dualf> gtbd, gd1bd;
            tot += ders(edge_reverse<dualf, true>(Ed, lift(f3(et)), lift(f3(s.ED[j])), gt, gd1r, mkd(0.f), &gtbd,
                                                  &gd1bd));
            const float4 lt = a.LT[j], le = a.LE[j];
            a.LT[j] = f4(f3(lt) + ders(gtbd), 0.f);
            a.LE[j] = f4(f3(le) + ders(gd1bd), le.w + ES.cs[j].z);
        }
        ES.s0[j] = f4(tot, 0.f);
    }
    g.sync();
    for (int i = g.tid; i < nv; i += TPR) {
        V3<float> l = f3(a.LX[i]);
        if (closed || i < nv - 1) l -= f3(ES.s0[i]);                   // edge i starts here
        if (closed || i > 0) l += f3(ES.s0[i == 0 ? ne - 1 : i - 1]);  // edge i-1 ends here
        a.LX[i] = f4(l, 0.f);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) gm[c] += gl[c];
    g.sync();
}

// ------------------------------------------------------------------ record layout
// Records of one chunk of frames, per rod (float4 units; NV the size class, n the substeps
// reserved per frame, N the projection iterations):
//   per frame, kFrameHead + NV:  its start pose (24 floats) and candidate count (int at float 24),
//                                then its candidate pairs (4 NV uint32)
//   per substep, sub_rec(NV, N): start state (X0, V, HG, ED, ET; 5 NV), v1 (NV), dfin (NV),
//                                projection records (N NV), contact snapshots (N NV), first-
//                                iteration pair data fr0, fr1 (4 NV each)
// Only what a frame uses is written and read (projection records for length-constrained rods,
// snapshots and pair data for frames with candidates).
constexpr int kFrameHead = 8;
__host__ __device__ constexpr size_t sub_rec(int NV, int n_iter) {
    return (size_t)(7 + 2 * n_iter + 2 * kPairsPerVertex) * NV;
}
__host__ __device__ constexpr size_t frame_rec(int NV, int n_iter, int nsub) {
    return (size_t)(kFrameHead + NV) + (size_t)nsub * sub_rec(NV, n_iter);
}
// frame-start state of one frame of a segment: X0, V, HG, ED, ET and the pose (24 floats)
__host__ __device__ constexpr size_t seg_state(int NV) { return (size_t)5 * NV + 6; }
// cotangent state carried from one chunk's reverse to the next: LX, LV, LE, LT, LK, then the
// material sums (5 doubles) and the frame-start pose cotangents (12 floats)
__host__ __device__ constexpr size_t cot_state(int NV) { return (size_t)5 * NV + 6; }

// ------------------------------------------------------------------ the recompute kernel
// Persistent, forward-like (a group of threads per rod, state in shared memory, several rods
// per CTA).  mode 0: from the checkpoint of the segment that holds frame fa, store the start
// state of each of the segment's frames (L2).  mode 1: from the start state of frame fa (a
// checkpoint, or the segment's stored state), run frames fa .. fb-1 storing every substep's
// records (R3).
template <int NV, bool CONTACT>
__global__ void __launch_bounds__(kFwdMaxThreads) rec_kernel(BwdParams P) {
    constexpr int TPR = threads_per_rod(NV);
    extern __shared__ float4 dyn_smem[];
    const int slot = threadIdx.x / TPR;
    Smem<NV, CONTACT> s(dyn_smem + slot * (rod_smem_bytes(NV, CONTACT) / 16));
    const Grp<TPR> g{(int)(threadIdx.x % TPR), 1 + slot, s.red};
    const SceneDev& sc = P.scene;
    const int n_iter = sc.n_iter;
    const size_t SR = sub_rec(NV, n_iter), FR = frame_rec(NV, n_iter, P.nsub_max);
    if (CONTACT)   // the contact accumulators start at zero; every sweep leaves them at zero
        for (int i = g.tid; i < NV; i += TPR) s.acc[i] = make_int4(0, 0, 0, 0);
    for (;;) {
        const int k = grp_bcast0<TPR>(g.tid == 0 ? atomicAdd(P.counter, 1) : 0, g);
        if (k >= P.n_items) break;
        const int rod = P.order[P.item0 + k];
        bounds_begin<TPR>(g);
        if (!in_bounds(rod >= 0 && rod < P.B && P.rods[rod].nv <= NV, s.red)) {
            g.sync();
            bounds_end<TPR>(g, P.status, (rod >= 0 && rod < P.B) ? rod : 0);
            continue;
        }
        // with self-contact read from memory where used: a register copy spills the
        // contact variant of the kernel (its broad phase and sweeps) past the launch bound
        RodRef<CONTACT> R = P.rods[rod];
        const int nsub = P.force_nsub > 0 ? P.force_nsub : R.nsub;
        const float h = sc.dt / (float)nsub;
        const int seg = P.fa / P.ck_every, f0 = seg * P.ck_every;
        float4* L2 = P.L2 + (size_t)k * P.l2_rod;
        if (P.mode == 0 || P.fa == f0) {   // the segment's checkpoint
            const long long oV = seg * P.ck_strideV, oE = seg * P.ck_strideE;
            for (int i = g.tid; i < R.nv; i += TPR) {
                const float4 x = P.ck.X[oV + R.v0 + i];
                s.X0[i] = x;
                s.X[i] = x;
                s.V[i] = P.ck.Vl[oV + R.v0 + i];
                s.HG[i] = P.ck.HG[oV + R.v0 + i];
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                s.ED[j] = P.ck.ED[oE + R.e0 + j];
                s.ET[j] = P.ck.ET[oE + R.e0 + j];
            }
            if (g.tid < 24) s.fp[g.tid] = P.ck.GP[seg * P.ck_strideB + 24LL * rod + g.tid];
        } else {                            // the stored start state of frame fa
            const float4* e = L2 + (size_t)(P.fa - f0) * seg_state(NV);
            for (int i = g.tid; i < R.nv; i += TPR) {
                const float4 x = e[i];
                s.X0[i] = x;
                s.X[i] = x;
                s.V[i] = e[NV + i];
                s.HG[i] = e[2 * NV + i];
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                s.ED[j] = e[3 * NV + j];
                s.ET[j] = e[4 * NV + j];
            }
            if (g.tid < 24) s.fp[g.tid] = reinterpret_cast<const float*>(e + 5 * NV)[g.tid];
        }
        g.sync();
        bool ovf = false;
        if (P.mode == 0) {
            const int f1 = min(f0 + P.ck_every, P.frames);
            for (int f = f0; f < f1; ++f) {
                float4* e = L2 + (size_t)(f - f0) * seg_state(NV);
                save_state<NV, CONTACT, TPR>(e, R, g, s);
                if (g.tid < 24) reinterpret_cast<float*>(e + 5 * NV)[g.tid] = s.fp[g.tid];
                if (f + 1 == f1) break;   // the segment's last frame only needs its start state
                if (g.tid < 12) s.act[g.tid] = P.actions[((size_t)f * P.B + rod) * 12 + g.tid];
                g.sync();
                run_frame<NV, CONTACT, TPR, true>(sc, P.KIN, P.ES, R, s, g, nsub, h, ovf,
                                                  [](int) -> const Rec* { return nullptr; });
            }
        } else {
            float4* R3 = P.R3 + (size_t)k * P.r3_rod;
            for (int f = P.fa; f < P.fb; ++f) {
                float4* fb = R3 + (size_t)(f - P.fa) * FR;
                if (g.tid < 24) reinterpret_cast<float*>(fb)[g.tid] = s.fp[g.tid];
                if (g.tid < 12) s.act[g.tid] = P.actions[((size_t)f * P.B + rod) * 12 + g.tid];
                g.sync();
                Rec recs;
                const int np = run_frame<NV, CONTACT, TPR, true>(
                    sc, P.KIN, P.ES, R, s, g, nsub, h, ovf, [&](int sb) -> const Rec* {
                        float4* e3 = fb + kFrameHead + NV + (size_t)sb * SR;
                        save_state<NV, CONTACT, TPR>(e3, R, g, s);
                        recs = Rec{e3 + 5 * NV, e3 + 6 * NV, e3 + 7 * NV, e3 + (size_t)(7 + n_iter) * NV,
                                   e3 + (size_t)(7 + 2 * n_iter) * NV,
                                   e3 + (size_t)(7 + 2 * n_iter + kPairsPerVertex) * NV, NV};
                        g.sync();   // the substep overwrites what was just stored
                        return &recs;
                    });
                if (CONTACT) {
                    uint32_t* pl = reinterpret_cast<uint32_t*>(fb + kFrameHead);
                    for (int p = g.tid; p < np; p += TPR) pl[p] = s.pairs[p];
                    if (g.tid == 0) reinterpret_cast<int*>(fb)[24] = np;
                }
            }
        }
        g.sync();
        bounds_end<TPR>(g, P.status, rod);
    }
}

// ------------------------------------------------------------------ the reverse kernel
// Persistent, one group of threads per rod: for frames fb-1 .. fa, last first, and each
// frame's substeps, last first, load the substep's records and apply the reverse of every
// phase (reverse_substep).  The cotangents of the rod's state at frame fb come from dL/d(final
// state) on the first chunk (fb = F), else from the previous chunk's launch (CS); those at fa
// go to CS, or to the outputs on the last chunk (fa = 0).
template <int NV, bool CONTACT>
__global__ void __launch_bounds__(rev_max_threads(NV)) rev_kernel(BwdParams P) {
    constexpr int TPR = threads_per_rod(NV);
    extern __shared__ float4 dyn_smem[];
    const int rs = threadIdx.x / TPR;
    float4* base = dyn_smem + rs * (bwd_smem_bytes(NV, CONTACT) / 16);
    Smem<NV, CONTACT> s(base);
    AdjArrays<NV, CONTACT> a(base + rod_smem_bytes(NV, CONTACT) / 16);
    const Grp<TPR> g{(int)(threadIdx.x % TPR), 1 + rs, s.red};
    const SceneDev& sc = P.scene;
    const int n_iter = sc.n_iter;
    const size_t SR = sub_rec(NV, n_iter), FR = frame_rec(NV, n_iter, P.nsub_max);
    for (;;) {
        const int k = grp_bcast0<TPR>(g.tid == 0 ? atomicAdd(P.counter, 1) : 0, g);
        if (k >= P.n_items) break;
        const int rod = P.order[P.item0 + k];
        bounds_begin<TPR>(g);
        if (!in_bounds(rod >= 0 && rod < P.B && P.rods[rod].nv <= NV, s.red)) {
            g.sync();
            bounds_end<TPR>(g, P.status, (rod >= 0 && rod < P.B) ? rod : 0);
            continue;
        }
        const RodInfo R = P.rods[rod];
        const int nsub = P.force_nsub > 0 ? P.force_nsub : R.nsub;
        const float h = sc.dt / (float)nsub;
        float4* CS = P.CS + (size_t)k * P.cs_rod;
        double gm[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // FP64: these sums cancel strongly
        float lpf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, lphif[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (P.first_chunk) {
            for (int i = g.tid; i < R.nv; i += TPR) {
                float4 dx = P.dLdx ? P.dLdx[R.v0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 dv = P.dLdv ? P.dLdv[R.v0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
                if (!(R.flags & ROD_CLOSED) && i == R.nv - 1) dv.w = 0.f;
                a.LX[i] = make_float4(dx.x, dx.y, dx.z, 0.f);
                a.LV[i] = dv;
                a.LK[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                a.LE[j] = make_float4(0.f, 0.f, 0.f, P.dLdth ? P.dLdth[R.e0 + j] : 0.f);
                a.LT[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {   // the sums are carried by thread 0 of the group
            for (int i = g.tid; i < R.nv; i += TPR) {
                a.LX[i] = CS[i];
                a.LV[i] = CS[NV + i];
                a.LK[i] = CS[4 * NV + i];
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                a.LE[j] = CS[2 * NV + j];
                a.LT[j] = CS[3 * NV + j];
            }
            if (g.tid == 0) {
                const double* d = reinterpret_cast<const double*>(CS + 5 * NV);
                const float* q = reinterpret_cast<const float*>(CS + 5 * NV + 3);
#pragma unroll
                for (int c = 0; c < 5; ++c) gm[c] = d[c];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    lpf[c] = q[c];
                    lphif[c] = q[6 + c];
                }
            }
        }
        float ga[12];
        for (int f = P.fb - 1; f >= P.fa; --f) {
            const float4* fb = P.R3 + (size_t)k * P.r3_rod + (size_t)(f - P.fa) * FR;
            g.sync();   // the previous frame's reverse has finished reading s.act, s.f0 and the pairs
            if (g.tid < 12) s.act[g.tid] = P.actions[((size_t)f * P.B + rod) * 12 + g.tid];
            if (g.tid < 24) s.f0[g.tid] = reinterpret_cast<const float*>(fb)[g.tid];
            int np = 0;
            if (CONTACT) {
                np = reinterpret_cast<const int*>(fb)[24];
                if (!in_bounds(np >= 0 && np <= R.pair_cap, s.red)) np = 0;
                const uint32_t* pl = reinterpret_cast<const uint32_t*>(fb + kFrameHead);
                for (int p = g.tid; p < np; p += TPR) s.pairs[p] = pl[p];
            }
            g.sync();
            // carry the pose cotangent of frame f+1's start into this frame's actions
#pragma unroll
            for (int c = 0; c < 12; ++c) ga[c] = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q >= R.ngrip) break;
                const V3<float> dphi = f3(s.act[6 * q + 3], s.act[6 * q + 4], s.act[6 * q + 5]);
                const V3<float> lp = get3(lpf, q), lr = get3(lphif, q);
                ga[6 * q] = lp.x;
                ga[6 * q + 1] = lp.y;
                ga[6 * q + 2] = lp.z;
                const V3<float> jr = jl_t(dphi, lr);
                ga[6 * q + 3] = jr.x;
                ga[6 * q + 4] = jr.y;
                ga[6 * q + 5] = jr.z;
                const V3<float> nr = mulT(expmap(dphi), lr);
                lphif[3 * q] = nr.x;
                lphif[3 * q + 1] = nr.y;
                lphif[3 * q + 2] = nr.z;
            }
            for (int sb = nsub - 1; sb >= 0; --sb) {
                const float c0 = (float)sb / (float)nsub, c1 = (float)(sb + 1) / (float)nsub;
                // the substep's gripper block (read after the barrier below)
                if (g.tid < R.ngrip) substep_pose(s.f0, s.act, g.tid, c0, c1, sb == 0, 1.f / sc.dt, s.sp);
                // the reverse's pose maps, on other threads (another warp where there is one)
                constexpr int PT = TPR > 32 ? 32 : 2;
                if (g.tid >= PT && g.tid < PT + 4 * R.ngrip) pose_rev_mat(s.act, g.tid - PT, c0, c1, a.PM);
                // the substep's start state and recorded intermediates
                const float4* e3 = fb + kFrameHead + NV + (size_t)sb * SR;
                load_state<NV, CONTACT, TPR>(e3, R, g, s);
                for (int i = g.tid; i < R.nv; i += TPR) {
                    a.V1[i] = e3[5 * NV + i];
                    a.DF[i] = e3[6 * NV + i];
                }
                if (CONTACT)
                    for (int p = g.tid; p < np; p += TPR) {
                        s.fr0[p] = e3[(7 + 2 * n_iter) * NV + p];
                        s.fr1[p] = e3[(7 + 2 * n_iter + kPairsPerVertex) * NV + p];
                    }
                g.sync();
                reverse_substep<NV, CONTACT, TPR>(P, R, s, a, e3 + 7 * NV, e3 + (size_t)(7 + n_iter) * NV, g, h, c0,
                                                  c1, np, gm, lpf, lphif, ga);
            }
            if (P.gact) {
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    if (c >= 6 * R.ngrip) break;
                    const float v = (float)grp_sum<TPR>((double)ga[c], g);
                    if (g.tid == 0) P.gact[((size_t)f * P.B + rod) * 12 + c] = v;
                }
                if (g.tid == 0)
                    for (int c = 6 * R.ngrip; c < 12; ++c) P.gact[((size_t)f * P.B + rod) * 12 + c] = 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) gm[c] = grp_sum<TPR>(gm[c], g);
        if (P.last_chunk) {   // outputs: the cotangents of the initial state and the material
            for (int i = g.tid; i < R.nv; i += TPR) {
                if (P.gx0) P.gx0[R.v0 + i] = a.LX[i];
                if (P.gv0) P.gv0[R.v0 + i] = a.LV[i];
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                if (P.gth0) P.gth0[R.e0 + j] = a.LE[j].w;
                P.gtb0[R.e0 + j] = a.LT[j];
                P.gd1b0[R.e0 + j] = make_float4(a.LE[j].x, a.LE[j].y, a.LE[j].z, 0.f);
            }
            if (g.tid == 0 && P.gmat) {
                const double r = R.radius, A = 3.14159265358979323846 * r * r, r2 = r * r;
                P.gmat[5 * rod + 0] = R.kA > 0.f ? (float)(gm[0] * A) : 0.f;   // K_stretch
                P.gmat[5 * rod + 1] = (float)(gm[1] * A * r2 / 4.0);            // E_bend
                P.gmat[5 * rod + 2] = (float)(gm[2] * A * r2 / 2.0);            // G_twist
                P.gmat[5 * rod + 3] = (float)gm[3];                             // yield curvature
                P.gmat[5 * rod + 4] = (float)gm[4];                             // damping
            }
        } else {   // carry to the next chunk: arrays, and the group sums of gm, lpf, lphif
            for (int i = g.tid; i < R.nv; i += TPR) {
                CS[i] = a.LX[i];
                CS[NV + i] = a.LV[i];
                CS[4 * NV + i] = a.LK[i];
            }
            for (int j = g.tid; j < R.ne; j += TPR) {
                CS[2 * NV + j] = a.LE[j];
                CS[3 * NV + j] = a.LT[j];
            }
            float q[12];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                q[c] = (float)grp_sum<TPR>((double)lpf[c], g);
                q[6 + c] = (float)grp_sum<TPR>((double)lphif[c], g);
            }
            if (g.tid == 0) {
                double* d = reinterpret_cast<double*>(CS + 5 * NV);
                float* qq = reinterpret_cast<float*>(CS + 5 * NV + 3);
#pragma unroll
                for (int c = 0; c < 5; ++c) d[c] = gm[c];
#pragma unroll
                for (int c = 0; c < 12; ++c) qq[c] = q[c];
            }
        }
        g.sync();
        bounds_end<TPR>(g, P.status, rod);
    }
}

// ------------------------------------------------------------------ launch helpers
template <int NV, bool C>
static int rev_occ_t(int rpc) {
    if (rpc < 1 || rpc * threads_per_rod(NV) > rev_max_threads(NV)) return 0;
    size_t smem = bwd_smem_bytes(NV, C) * rpc;
    auto k = rev_kernel<NV, C>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads_per_rod(NV) * rpc, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
template <int NV, bool C>
static cudaError_t launch_rev_t(const BwdParams& P, int grid, int rpc, cudaStream_t st) {
    size_t smem = bwd_smem_bytes(NV, C) * rpc;
    auto k = rev_kernel<NV, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads_per_rod(NV) * rpc, smem, st>>>(P);
    return cudaGetLastError();
}
template <int NV, bool C>
static int rec_occ_t(int rpc) {
    if (rpc < 1 || rpc * threads_per_rod(NV) > kFwdMaxThreads) return 0;
    size_t smem = rod_smem_bytes(NV, C) * rpc;
    auto k = rec_kernel<NV, C>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads_per_rod(NV) * rpc, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
template <int NV, bool C>
static cudaError_t launch_rec_t(const BwdParams& P, int grid, int rpc, cudaStream_t st) {
    size_t smem = rod_smem_bytes(NV, C) * rpc;
    auto k = rec_kernel<NV, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads_per_rod(NV) * rpc, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace dlo
