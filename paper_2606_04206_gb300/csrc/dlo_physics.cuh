// dlo_physics.cuh -- element functions of the discrete-elastic-rod step (device side).
//
// Model: DLO-Lab (arXiv 2606.04206) Sec. 3.1 / App. A.1.  Each function is a template on the
// scalar type (float for the step, dualf for Jacobian-vector products in the adjoint).
//
// Energy of one hinge i (edges a = i-1, b = i), App. A.1:
//   (kappa b)_i = 2 t^a x t^b / (1 + t^a . t^b)
//   kappa_i     = 1/2 ( (kappa b).(d2^a + d2^b), (kappa b).(d1^a + d1^b) )
//   m_i         = theta^b - theta^a + (reference twist)
//   U_i = 1/2 (B/lbar) |kappa - kbar|^2 + 1/2 (beta/lbar) (m - mbar)^2
// Stretching of one edge: U_j = 1/2 K A (|e|/|ebar| - 1)^2 |ebar|.
// The reference frame of an edge is its stored base frame (t_base, d1_base) transported in
// time to the current tangent and re-orthonormalised; the material frame is that frame
// rotated by theta.  Forces are the exact gradient of U with respect to the vertex positions
// (including the dependence of the transported reference frame on them); it is computed by
// a hand-written reverse pass over the same expressions.
#pragma once
#include "dlo_vec.cuh"

namespace dlo {

constexpr float kTwoPi = 6.28318530717958647692f;

DLO_HD double dsqrt(double a) { return sqrt(a); }

// Parallel transport of d from unit tangent a to unit tangent b (rotation about a x b).
template <class T>
DLO_HD V3<T> transport(V3<T> a, V3<T> b, V3<T> d) {
    T c = dot(a, b);
    V3<T> k = cross(a, b);
    return c * d + cross(k, d) + (dot(k, d) / (1.f + c)) * k;
}
DLO_HD V3<double> transport_d(V3<double> a, V3<double> b, V3<double> d) {
    double c = dot(a, b);
    V3<double> k = cross(a, b);
    return c * d + cross(k, d) + (dot(k, d) / (1.0 + c)) * k;
}

// Length of e and its inverse from one reciprocal square root.
DLO_HD void len_inv(V3<float> e, float& ell, float& inv) {
    const float e2 = dot(e, e);
#ifdef __CUDA_ARCH__
    inv = rsqrtf(e2);
#else
    inv = 1.f / sqrtf(e2);
#endif
    ell = e2 * inv;
}

// Axial strain |e| / |ebar| - 1 with IEEE-rounded square root and quotient: the stretching
// sensitivity sums strains of nearly inextensible edges, so it keeps what float32 positions
// resolve rather than the approximate square root's extra ulps.
DLO_HD float edge_strain(V3<float> e, float eb) {
#ifdef __CUDA_ARCH__
    return __fdiv_rn(__fsqrt_rn(dot(e, e)), eb) - 1.f;
#else
    return sqrtf(dot(e, e)) / eb - 1.f;
#endif
}

// ------------------------------------------------------------------ edge frames
template <class T>
struct EdgeF {
    V3<T> t, w0, d1r, d2r, d1, d2;
    T ell, n1, c, s;
};

template <class T>
DLO_HD void edge_forward(EdgeF<T>& E, V3<T> xa, V3<T> xb, V3<T> tb, V3<T> d1b, T th) {
    V3<T> e = xb - xa;
    E.ell = norm(e);
    E.t = e / E.ell;
    E.w0 = transport(tb, E.t, d1b);
    V3<T> w1 = E.w0 - dot(E.w0, E.t) * E.t;
    E.n1 = norm(w1);
    E.d1r = w1 / E.n1;
    E.d2r = cross(E.t, E.d1r);
    E.c = dcos(th);
    E.s = dsin(th);
    E.d1 = E.c * E.d1r + E.s * E.d2r;
    E.d2 = E.c * E.d2r - E.s * E.d1r;
}

// Reverse of edge_forward: given adjoints of t and d1r (and of |e|), the adjoint of the edge
// vector e = xb - xa; with BASE also the adjoints of the base frame (tb, d1b).
template <class T, bool BASE>
DLO_HD V3<T> edge_reverse(const EdgeF<T>& E, V3<T> tb, V3<T> d1b, V3<T> gt, V3<T> gd1r, T gell,
                          V3<T>* gtb, V3<T>* gd1b) {
    V3<T> gw1 = (gd1r - dot(gd1r, E.d1r) * E.d1r) / E.n1;
    T w0t = dot(E.w0, E.t);
    T gw1t = dot(gw1, E.t);
    V3<T> gw0 = gw1 - gw1t * E.t;
    gt -= gw1t * E.w0 + w0t * gw1;
    T cp = dot(tb, E.t);
    V3<T> k = cross(tb, E.t);
    T kd = dot(k, d1b);
    T opc = 1.f + cp;
    T gkk = dot(gw0, k);
    T gcp = dot(gw0, d1b) - kd * gkk / (opc * opc);
    V3<T> gk = cross(d1b, gw0) + (kd / opc) * gw0 + (gkk / opc) * d1b;
    gt += gcp * tb + cross(gk, tb);
    if (BASE) {
        *gd1b = cp * gw0 + cross(gw0, k) + (gkk / opc) * k;
        *gtb = gcp * E.t + cross(E.t, gk);
    }
    return (gt - dot(gt, E.t) * E.t) / E.ell + gell * E.t;
}

// ------------------------------------------------------------------ hinge
template <class T>
struct HingeF {
    EdgeF<T> a, b;
    V3<T> X, kb, u;
    T cc, y, xq, mref, m, k0, k1;
};

// The hinge's own part, from its two edges' frames (H.a, H.b: t, d1r, d2r, d1, d2 set).
template <class T>
DLO_HD void hinge_core_forward(HingeF<T>& H, T tha, T thb, T mprev) {
    H.cc = 1.f + dot(H.a.t, H.b.t);
    H.X = cross(H.a.t, H.b.t);
    H.kb = (2.f / H.cc) * H.X;
    H.k0 = 0.5f * dot(H.kb, H.a.d2 + H.b.d2);
    H.k1 = 0.5f * dot(H.kb, H.a.d1 + H.b.d1);
    // reference twist: angle about t^b from the space-transported d1r^a to d1r^b
    H.u = (H.cc - 1.f) * H.a.d1r + cross(H.X, H.a.d1r) + (dot(H.X, H.a.d1r) / H.cc) * H.X;
    H.y = dot(cross(H.u, H.b.d1r), H.b.t);
    H.xq = dot(H.u, H.b.d1r);
    T ang = datan2(H.y, H.xq);
    float wr = rintf((vof(ang) - vof(mprev)) / kTwoPi);
    H.mref = mprev + ((ang - mprev) - kTwoPi * wr);
    H.m = thb - tha + H.mref;
}

template <class T>
DLO_HD void hinge_forward(HingeF<T>& H, V3<T> xm, V3<T> xi, V3<T> xp, V3<T> tba, V3<T> d1ba,
                          V3<T> tbb, V3<T> d1bb, T tha, T thb, T mprev) {
    edge_forward(H.a, xm, xi, tba, d1ba, tha);
    edge_forward(H.b, xi, xp, tbb, d1bb, thb);
    hinge_core_forward(H, tha, thb, mprev);
}

// Reverse of hinge_core_forward from seeds on kappa (gk0, gk1), on the total twist m (gmt,
// flows to theta and the reference twist) and on the reference twist alone (gmr): the adjoints
// of both edges' tangents and reference directors (gta, gd1ra, gtb, gd1rb) and of the two
// twist angles.
template <class T>
DLO_HD void hinge_core_reverse(const HingeF<T>& H, T gk0, T gk1, T gmt, T gmr, V3<T>& gta, V3<T>& gd1ra,
                               V3<T>& gtb_, V3<T>& gd1rb, T& gtha, T& gthb) {
    const EdgeF<T>& A = H.a;
    const EdgeF<T>& B = H.b;
    T hk0 = 0.5f * gk0, hk1 = 0.5f * gk1;
    V3<T> gkb = hk0 * (A.d2 + B.d2) + hk1 * (A.d1 + B.d1);
    V3<T> gd2 = hk0 * H.kb;      // same for both edges
    V3<T> gd1 = hk1 * H.kb;
    V3<T> gX = (2.f / H.cc) * gkb;
    T gcc = -dot(gkb, H.kb) / H.cc;
    // twist
    T gang = gmt + gmr;
    gtha = -gmt;
    gthb = gmt;
    T r2 = H.y * H.y + H.xq * H.xq;
    T gy = gang * H.xq / r2;
    T gxq = -(gang * H.y) / r2;
    V3<T> gu = gy * cross(B.d1r, B.t) + gxq * B.d1r;
    gd1rb = gy * cross(B.t, H.u) + gxq * H.u;
    gtb_ = gy * cross(H.u, B.d1r);
    T Xd = dot(H.X, A.d1r);
    T gux = dot(gu, H.X);
    gcc += dot(gu, A.d1r) - Xd * gux / (H.cc * H.cc);
    gd1ra = (H.cc - 1.f) * gu + cross(gu, H.X) + (gux / H.cc) * H.X;
    gX += cross(A.d1r, gu) + (Xd / H.cc) * gu + (gux / H.cc) * A.d1r;
    gta = gcc * B.t + cross(B.t, gX);
    gtb_ += gcc * A.t + cross(gX, A.t);
    // material frames -> reference frames and twist angles
    {
        gd1ra += A.c * gd1 - A.s * gd2;
        V3<T> gd2r = A.s * gd1 + A.c * gd2;
        gtha += dot(gd1, A.d2) - dot(gd2, A.d1);
        gta += cross(A.d1r, gd2r);
        gd1ra += cross(gd2r, A.t);
    }
    {
        gd1rb += B.c * gd1 - B.s * gd2;
        V3<T> gd2r = B.s * gd1 + B.c * gd2;
        gthb += dot(gd1, B.d2) - dot(gd2, B.d1);
        gtb_ += cross(B.d1r, gd2r);
        gd1rb += cross(gd2r, B.t);
    }
}

// Reverse of hinge_forward: the adjoints of the three vertices and the two twist angles; with
// BASE also of both base frames.
template <class T, bool BASE>
DLO_HD void hinge_reverse(const HingeF<T>& H, V3<T> tba, V3<T> d1ba, V3<T> tbb, V3<T> d1bb,
                          T gk0, T gk1, T gmt, T gmr, V3<T>& gxm, V3<T>& gxi, V3<T>& gxp,
                          T& gtha, T& gthb, V3<T>* gtba, V3<T>* gd1ba, V3<T>* gtbb,
                          V3<T>* gd1bb) {
    V3<T> gta, gd1ra, gtb_, gd1rb;
    hinge_core_reverse(H, gk0, gk1, gmt, gmr, gta, gd1ra, gtb_, gd1rb, gtha, gthb);
    const EdgeF<T>& A = H.a;
    const EdgeF<T>& B = H.b;
    T zero = cst<T>(0.f);
    V3<T> gea = edge_reverse<T, BASE>(A, tba, d1ba, gta, gd1ra, zero, gtba, gd1ba);
    V3<T> geb = edge_reverse<T, BASE>(B, tbb, d1bb, gtb_, gd1rb, zero, gtbb, gd1bb);
    gxm = -gea;
    gxi = gea - geb;
    gxp = geb;
}

// ------------------------------------------------------------------ plasticity (App. A.1)
// kappa_el = kappa - kbar; if |kappa_el| > sigma_y lbar: kbar += r_c (|k_el| - y)/|k_el| k_el.
DLO_HD bool plastic_update(float k0, float k1, float& kb0, float& kb1, float thr, float rc) {
    float e0 = k0 - kb0, e1 = k1 - kb1;
    float n2 = e0 * e0 + e1 * e1;
    if (!(n2 > 0.f)) return false;
    float n = sqrtf(n2);
    if (!(n > thr)) return false;
    float g = rc * (n - thr) / n;
    kb0 = kb0 + g * e0;
    kb1 = kb1 + g * e1;
    return true;
}

// ------------------------------------------------------------------ rigid SDF primitives
template <class T>
DLO_HD T sdf_box(V3<T> x, V3<float> c, V3<float> hl, V3<T>& n) {
    V3<T> p = x - mk3(cst<T>(c.x), cst<T>(c.y), cst<T>(c.z));
    float sx = vof(p.x) >= 0.f ? 1.f : -1.f, sy = vof(p.y) >= 0.f ? 1.f : -1.f,
          sz = vof(p.z) >= 0.f ? 1.f : -1.f;
    T qx = sx * p.x - hl.x, qy = sy * p.y - hl.y, qz = sz * p.z - hl.z;
    T ox = vof(qx) > 0.f ? qx : cst<T>(0.f), oy = vof(qy) > 0.f ? qy : cst<T>(0.f),
      oz = vof(qz) > 0.f ? qz : cst<T>(0.f);
    T ol2 = ox * ox + oy * oy + oz * oz;
    if (vof(ol2) > 0.f) {
        T ol = dsqrt(ol2);
        n = mk3(sx * ox / ol, sy * oy / ol, sz * oz / ol);
        return ol;
    }
    // inside: the largest (least negative) q, first index on ties
    int k = 0;
    T qm = qx;
    if (vof(qy) > vof(qm)) { k = 1; qm = qy; }
    if (vof(qz) > vof(qm)) { k = 2; qm = qz; }
    n = mk3(cst<T>(k == 0 ? sx : 0.f), cst<T>(k == 1 ? sy : 0.f), cst<T>(k == 2 ? sz : 0.f));
    return qm;
}

template <class T>
DLO_HD T sdf_capsule(V3<T> x, V3<T> a, V3<T> b, float rc, V3<T>& n) {
    V3<T> ab = b - a;
    T s = dclamp(dot(x - a, ab) / dot(ab, ab), 0.f, 1.f);
    V3<T> dv = x - (a + s * ab);
    T d2 = dot(dv, dv);
    if (!(vof(d2) > 0.f)) {
        n = zero3<T>();
        return cst<T>(-rc);
    }
    T d = dsqrt(d2);
    n = dv / d;
    return d - rc;
}

constexpr float kContactReach = 2.31f;   // -ln(0.1) = 2.3026 plus a margin

// Whether x lies farther than reach from the segment ab, by squared distances (no square root
// or quotient for the many vertices far from a gripper); a margin of 1e-3 reach keeps every
// point the exact test would take.
DLO_HD bool capsule_far(V3<float> x, V3<float> a, V3<float> b, float reach) {
    const V3<float> ab = b - a, xa = x - a;
    const float L2 = dot(ab, ab), q = dot(xa, ab);
    const float s = q <= 0.f ? 0.f : (q >= L2 ? 1.f : q / L2);
    const V3<float> dv = xa - s * ab;
    const float lim = 1.001f * reach;
    return dot(dv, dv) > lim * lim;
}

// Soft coupling (Sec. 3.2): d = r - SDF, f = min(exp(d / eps_s), 1); if f > 0.1 the relative
// velocity's normal part gets restitution and its tangential part Coulomb friction, and the
// result is blended in with weight f.
template <class T>
DLO_HD V3<T> contact_respond(V3<T> v, T sdf, V3<T> n, V3<T> vrig, float r, float eps_s,
                             float mu, float rest, bool& act) {
    // f < exp(-2.31) < 0.099 there: the contact is inactive (decided without the exponential)
    if (vof(sdf) > r + kContactReach * eps_s) {
        act = false;
        return v;
    }
    T f = dexp((r - sdf) / eps_s);
    if (vof(f) > 1.f) f = cst<T>(1.f);
    act = vof(f) > 0.1f;
    if (!act) return v;
    V3<T> vr = v - vrig;
    T vn = dot(vr, n);
    V3<T> vt = vr - vn * n;
    T vn2 = dmax(vn, (-rest) * vn);
    T dvn = vn2 - vn;
    T vt2 = dot(vt, vt);
    T sc = cst<T>(1.f);
    if (vof(vt2) > 1e-24f) sc = dmax(1.f - mu * dvn / dsqrt(vt2), cst<T>(0.f));
    V3<T> vr2 = vn2 * n + sc * vt;
    return v + f * (vr2 - vr);
}

// Reverse of contact_respond on its active branch (the caller has seen act == true): given the
// cotangent lo of the output velocity, the cotangents of v, sdf, the normal and the rigid
// velocity.  Branches (min / max selections) follow the forward values.
DLO_HD void contact_respond_rev(V3<float> v, float sdf, V3<float> n, V3<float> vrig, float r, float eps_s,
                                float mu, float rest, V3<float> lo, V3<float>& lv, float& lsdf, V3<float>& ln,
                                V3<float>& lvrig) {
    const float f0 = expf((r - sdf) / eps_s);
    const float f = f0 > 1.f ? 1.f : f0;
    const V3<float> vr = v - vrig;
    const float vn = dot(vr, n);
    const V3<float> vt = vr - vn * n;
    const bool keep = vn >= -rest * vn;
    const float vn2 = keep ? vn : -rest * vn;
    const float dvn = vn2 - vn;
    const float vt2 = dot(vt, vt);
    float sc = 1.f, s = 0.f, q = 1.f;
    const bool fr = vt2 > 1e-24f;
    if (fr) {
        s = sqrtf(vt2);
        q = 1.f - mu * dvn / s;
        sc = q >= 0.f ? q : 0.f;
    }
    const V3<float> vr2 = vn2 * n + sc * vt;
    // out = v + f (vr2 - vr)
    lv = lo;
    const float lf = dot(lo, vr2 - vr);
    const V3<float> lvr2 = f * lo;
    V3<float> lvr = -f * lo;
    float lvn2 = dot(lvr2, n);
    ln = vn2 * lvr2;
    const float lsc = dot(lvr2, vt);
    V3<float> lvt = sc * lvr2;
    float lvn = 0.f;
    if (fr && q >= 0.f) {
        const float ldvn = -mu * lsc / s;
        const float ls = mu * dvn * lsc / (s * s);
        lvt += (ls / s) * vt;
        lvn2 += ldvn;
        lvn -= ldvn;
    }
    lvn += keep ? lvn2 : -rest * lvn2;
    lvr += lvt;
    lvn -= dot(lvt, n);
    ln -= vn * lvt;
    lvr += lvn * n;
    ln += lvn * vr;
    lv += lvr;
    lvrig = -lvr;
    lsdf = f0 < 1.f ? -lf * f0 / eps_s : 0.f;
}

// Reverse of the soft contact of a vertex with a static box (centre c, half extents hl) on the
// active branch: from the cotangent lo of the output velocity, the cotangents of the position
// (returned) and of the velocity (lv).  Outside the box the SDF is |u|, u the offset from the
// nearest surface point (u_i = p_i - sign(p_i) hl_i on the axes where |p_i| > hl_i, else 0),
// and the normal u/|u| turns with x; inside, the SDF is the nearest face's |p_k| - hl_k and its
// normal is constant.
DLO_HD V3<float> box_contact_rev(V3<float> x, V3<float> v, V3<float> c, V3<float> hl, float r, float eps_s,
                                 float mu, float rest, V3<float> lo, V3<float>& lv) {
    V3<float> n;
    const float sdf = sdf_box(x, c, hl, n);
    V3<float> ln, lvr;
    float lsdf;
    contact_respond_rev(v, sdf, n, zf3(), r, eps_s, mu, rest, lo, lv, lsdf, ln, lvr);
    V3<float> lx = lsdf * n;
    const V3<float> p = x - c;
    const float qx = (p.x >= 0.f ? p.x : -p.x) - hl.x, qy = (p.y >= 0.f ? p.y : -p.y) - hl.y,
                qz = (p.z >= 0.f ? p.z : -p.z) - hl.z;
    if (qx > 0.f || qy > 0.f || qz > 0.f) {
        const V3<float> w = (ln - dot(ln, n) * n) / sdf;
        lx.x += qx > 0.f ? w.x : 0.f;
        lx.y += qy > 0.f ? w.y : 0.f;
        lx.z += qz > 0.f ? w.z : 0.f;
    }
    return lx;
}

// Reverse of the soft contact of a vertex with a capsule gripper (segment p +- hl * ax, radius
// rc, rigid velocity vp + w x (x - p)) on the active branch: from the cotangent lo of the output
// velocity, the cotangents of x, v, the capsule position p, its axis rotation (as a world-frame
// rotation vector), vp and w.
DLO_HD void capsule_contact_rev(V3<float> x, V3<float> v, V3<float> p, V3<float> ax, float hl, float rc,
                                V3<float> vp, V3<float> w, float r, float eps_s, float mu, float rest, V3<float> lo,
                                V3<float>& lx, V3<float>& lv, V3<float>& lp, V3<float>& lphi, V3<float>& lvp,
                                V3<float>& lw) {
    const V3<float> a = p - hl * ax, b = p + hl * ax, ab = b - a;
    const float L2 = dot(ab, ab);
    const float q = dot(x - a, ab) / L2;
    const float sc = q < 0.f ? 0.f : (q > 1.f ? 1.f : q);
    const V3<float> c = a + sc * ab, dv = x - c;
    const float d = sqrtf(dot(dv, dv));
    const V3<float> n = dv / d;
    const V3<float> y = x - p;
    const V3<float> vrig = vp + cross(w, y);
    V3<float> ln, lvrig;
    float lsdf;
    contact_respond_rev(v, d - rc, n, vrig, r, eps_s, mu, rest, lo, lv, lsdf, ln, lvrig);
    lvp = lvrig;
    lw = cross(y, lvrig);
    lx = cross(lvrig, w);
    lp = -lx;
    const V3<float> ldv = (ln - dot(ln, n) * n) / d + lsdf * n;
    lx += ldv;
    const V3<float> lc = -ldv;
    V3<float> la = lc, lab = sc * lc;
    if (q > 0.f && q < 1.f) {
        const float lq = dot(lc, ab);
        lx += (lq / L2) * ab;
        la -= (lq / L2) * ab;
        lab += lq * ((x - a) / L2 - (2.f * q / L2) * ab);
    }
    const V3<float> lb = lab;
    la -= lab;
    lp += la + lb;
    const V3<float> lax = hl * (lb - la);
    lphi = cross(ax, lax);
}

// ------------------------------------------------------------------ segment closest points
// Clamped closed-form closest points of segments p1q1 and p2q2 (Ericson, Real-Time Collision
// Detection, Sec. 5.1.9); near-parallel segments take s = 0 and u clamped.
template <class T>
DLO_HD void closest_params(V3<T> p1, V3<T> q1, V3<T> p2, V3<T> q2, T& s, T& u) {
    V3<T> d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
    T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r), c = dot(d1, r), b = dot(d1, d2);
    T den = a * e - b * b;
    if (vof(den) <= 1e-6f * vof(a) * vof(e))
        s = cst<T>(0.f);
    else
        s = dclamp((b * f - c * e) / den, 0.f, 1.f);
    T uu = (b * s + f) / e;
    if (vof(uu) < 0.f) {
        s = dclamp((-c) / a, 0.f, 1.f);
        u = cst<T>(0.f);
    } else if (vof(uu) > 1.f) {
        s = dclamp((b - c) / a, 0.f, 1.f);
        u = cst<T>(1.f);
    } else {
        u = uu;
    }
}

// One self-collision projection for an edge pair (App. A.1): the four position corrections.
template <class T>
DLO_HD bool pair_correction(V3<T> xa0, V3<T> xa1, V3<T> xb0, V3<T> xb1, float wa0, float wa1,
                            float wb0, float wb1, float rsum, V3<T>* dx, T& s, T& u, V3<T>& n,
                            T& d, T& W) {
    closest_params(xa0, xa1, xb0, xb1, s, u);
    V3<T> ca = xa0 + s * (xa1 - xa0);
    V3<T> cb = xb0 + u * (xb1 - xb0);
    V3<T> dv = ca - cb;
    T d2 = dot(dv, dv);
    T os = 1.f - s, ou = 1.f - u;
    W = wa0 * os * os + wa1 * s * s + wb0 * ou * ou + wb1 * u * u;
    if (!(vof(d2) > 1e-24f) || !(vof(W) > 0.f)) return false;
    T dist = dsqrt(d2);
    d = rsum - dist;
    if (!(vof(d) > 0.f)) return false;
    n = dv / dist;
    T k = d / W;
    dx[0] = (k * (wa0 * os)) * n;
    dx[1] = (k * (wa1 * s)) * n;
    dx[2] = (-(k * (wb0 * ou))) * n;
    dx[3] = (-(k * (wb1 * u))) * n;
    return true;
}

// Friction of one pair (App. A.1), as a function of the four positions at the first
// projection and the four rebuilt velocities; returns whether the pair acts.  This is the
// definition the closed-form reverse fric_pair_vjp differentiates (and is checked against
// with dual numbers); the kernels' forward applies the same formula from the first sweep's
// stored pair data (self_friction).
template <class T>
DLO_HD bool fric_pair(const V3<T>* P, const V3<T>* Vv, const float* w, float rsum, float mu, float h, V3<T>* dv) {
    T s, u, d, W;
    V3<T> n, dx[4];
    if (!pair_correction(P[0], P[1], P[2], P[3], w[0], w[1], w[2], w[3], rsum, dx, s, u, n, d, W)) return false;
    V3<T> vrel = (1.f - s) * Vv[0] + s * Vv[1] - (1.f - u) * Vv[2] - u * Vv[3];
    V3<T> vt = vrel - dot(vrel, n) * n;
    T vt2 = dot(vt, vt);
    if (!(vof(vt2) > 1e-24f)) return false;
    T coef = dmin(mu * d / (h * dsqrt(vt2)), cst<T>(1.f));
    V3<T> dd = (-(coef / W)) * vt;
    dv[0] = (w[0] * (1.f - s)) * dd;
    dv[1] = (w[1] * s) * dd;
    dv[2] = (-(w[2] * (1.f - u))) * dd;
    dv[3] = (-(w[3] * u)) * dd;
    return true;
}

// ------------------------------------------------------------------ closed-form pair reverses
// The forward of pair_correction (segments P0P1 and P2P3) with what its reverse needs: the
// closest-point solve's scalars and how s and u were formed (the branch taken), the normal,
// depth and weight sum.  The expressions are those of closest_params and pair_correction.
struct PairFwd {
    V3<float> d1, d2, r, n;
    float a, b, c, e, f, den, s0, s, u, dist, d, W;
    int sb;   // s: 0 constant (parallel or clamped), 1 (b f - c e) / den, 2 -c / a, 3 (b - c) / a
    bool uf;  // u = (b s0 + f) / e (else constant)
};

DLO_HD bool pair_fwd(const V3<float>* P, const float* w, float rsum, PairFwd& F) {
    F.d1 = P[1] - P[0];
    F.d2 = P[3] - P[2];
    F.r = P[0] - P[2];
    F.a = dot(F.d1, F.d1);
    F.e = dot(F.d2, F.d2);
    F.f = dot(F.d2, F.r);
    F.c = dot(F.d1, F.r);
    F.b = dot(F.d1, F.d2);
    F.den = F.a * F.e - F.b * F.b;
    float s = 0.f;
    F.sb = 0;
    if (!(F.den <= 1e-6f * F.a * F.e)) {
        const float q = (F.b * F.f - F.c * F.e) / F.den;
        s = q < 0.f ? 0.f : (q > 1.f ? 1.f : q);
        F.sb = (q < 0.f || q > 1.f) ? 0 : 1;
    }
    F.s0 = s;
    const float uu = (F.b * s + F.f) / F.e;
    F.uf = false;
    if (uu < 0.f) {
        const float q = (-F.c) / F.a;
        s = q < 0.f ? 0.f : (q > 1.f ? 1.f : q);
        F.sb = (q < 0.f || q > 1.f) ? 0 : 2;
        F.u = 0.f;
    } else if (uu > 1.f) {
        const float q = (F.b - F.c) / F.a;
        s = q < 0.f ? 0.f : (q > 1.f ? 1.f : q);
        F.sb = (q < 0.f || q > 1.f) ? 0 : 3;
        F.u = 1.f;
    } else {
        F.u = uu;
        F.uf = true;
    }
    F.s = s;
    const float u = F.u;
    const V3<float> ca = P[0] + s * (P[1] - P[0]);
    const V3<float> cb = P[2] + u * (P[3] - P[2]);
    const V3<float> dv = ca - cb;
    const float d2 = dot(dv, dv);
    const float os = 1.f - s, ou = 1.f - u;
    F.W = w[0] * os * os + w[1] * s * s + w[2] * ou * ou + w[3] * u * u;
    if (!(d2 > 1e-24f) || !(F.W > 0.f)) return false;
    F.dist = dsqrt(d2);
    F.d = rsum - F.dist;
    if (!(F.d > 0.f)) return false;
    F.n = dv / F.dist;
    return true;
}

// Reverse of pair_fwd: from the cotangents of s, u, the normal, the depth and the weight sum,
// the cotangents of the four points (Pb, overwritten).  Branches follow the forward's.
DLO_HD void pair_fwd_rev(const PairFwd& F, const V3<float>* P, const float* w, float sb_, float ub_, V3<float> nb,
                         float db, float Wb, V3<float>* Pb) {
    const float s = F.s, u = F.u, os = 1.f - s, ou = 1.f - u;
    sb_ += Wb * (2.f * w[1] * s - 2.f * w[0] * os);
    ub_ += Wb * (2.f * w[3] * u - 2.f * w[2] * ou);
    // n = dv / |dv|, d = rsum - |dv|
    const V3<float> dvb = (nb - dot(nb, F.n) * F.n) / F.dist - db * F.n;
    // dv = P0 + s (P1 - P0) - P2 - u (P3 - P2)
    Pb[0] = os * dvb;
    Pb[1] = s * dvb;
    Pb[2] = (-ou) * dvb;
    Pb[3] = (-u) * dvb;
    sb_ += dot(dvb, P[1] - P[0]);
    ub_ -= dot(dvb, P[3] - P[2]);
    // the closest-point solve
    float ab = 0.f, bb = 0.f, cb = 0.f, eb = 0.f, fb = 0.f;
    if (F.uf) {   // u = (b s0 + f) / e with s = s0
        bb += ub_ * F.s0 / F.e;
        sb_ += ub_ * F.b / F.e;
        fb += ub_ / F.e;
        eb -= ub_ * u / F.e;
    }
    if (F.sb == 1) {   // s = (b f - c e) / den, den = a e - b^2
        const float numb = sb_ / F.den, denb = -sb_ * s / F.den;
        bb += numb * F.f - 2.f * F.b * denb;
        fb += numb * F.b;
        cb -= numb * F.e;
        eb += denb * F.a - numb * F.c;
        ab += denb * F.e;
    } else if (F.sb == 2) {   // s = -c / a
        cb -= sb_ / F.a;
        ab -= sb_ * s / F.a;
    } else if (F.sb == 3) {   // s = (b - c) / a
        bb += sb_ / F.a;
        cb -= sb_ / F.a;
        ab -= sb_ * s / F.a;
    }
    const V3<float> d1b = (2.f * ab) * F.d1 + cb * F.r + bb * F.d2;
    const V3<float> d2b = (2.f * eb) * F.d2 + fb * F.r + bb * F.d1;
    const V3<float> rb = fb * F.d2 + cb * F.d1;
    Pb[0] += rb - d1b;
    Pb[1] += d1b;
    Pb[2] -= rb + d2b;
    Pb[3] += d2b;
}

// Vector-Jacobian product of the self-collision projection (pair_correction): with lo the
// cotangents of the four corrections, the cotangents of the four points.  False where the pair
// makes no correction (then Pb is untouched).
DLO_HD bool pair_correction_vjp(const V3<float>* P, const float* w, float rsum, const V3<float>* lo, V3<float>* Pb) {
    PairFwd F;
    if (!pair_fwd(P, w, rsum, F)) return false;
    const float s = F.s, u = F.u, os = 1.f - s, ou = 1.f - u;
    const float k = F.d / F.W;
    // sum_k lo_k . dx_k = k (n . Lam)
    const V3<float> Lam = (w[0] * os) * lo[0] + (w[1] * s) * lo[1] - (w[2] * ou) * lo[2] - (w[3] * u) * lo[3];
    const float m = dot(F.n, Lam);
    const V3<float> Lamb = k * F.n;
    const float sb_ = dot(Lamb, w[1] * lo[1] - w[0] * lo[0]);
    const float ub_ = dot(Lamb, w[2] * lo[2] - w[3] * lo[3]);
    pair_fwd_rev(F, P, w, sb_, ub_, k * Lam, m / F.W, -m * k / F.W, Pb);
    return true;
}

// Vector-Jacobian product of one pair's self-contact friction (the velocity corrections of
// fric_pair): with lo the cotangents of the four velocity corrections, the cotangents of the
// four points (Pb) and velocities (Vb).  False where the pair makes no correction.
DLO_HD bool fric_pair_vjp(const V3<float>* P, const V3<float>* Vv, const float* w, float rsum, float mu, float h,
                          const V3<float>* lo, V3<float>* Pb, V3<float>* Vb) {
    PairFwd F;
    if (!pair_fwd(P, w, rsum, F)) return false;
    const float s = F.s, u = F.u, os = 1.f - s, ou = 1.f - u;
    const V3<float> vrel = os * Vv[0] + s * Vv[1] - ou * Vv[2] - u * Vv[3];
    const float vn = dot(vrel, F.n);
    const V3<float> vt = vrel - vn * F.n;
    const float vt2 = dot(vt, vt);
    if (!(vt2 > 1e-24f)) return false;
    const float sv = dsqrt(vt2);
    const float c0 = mu * F.d / (h * sv);
    const bool free = c0 <= 1.f;
    const float coef = free ? c0 : 1.f;
    const float q = coef / F.W;
    // sum_k lo_k . dv_k = -q (vt . Gam)
    const V3<float> Gam = (w[0] * os) * lo[0] + (w[1] * s) * lo[1] - (w[2] * ou) * lo[2] - (w[3] * u) * lo[3];
    const float m = dot(vt, Gam);
    V3<float> vtb = (-q) * Gam;
    const V3<float> Gamb = (-q) * vt;
    float sb_ = dot(Gamb, w[1] * lo[1] - w[0] * lo[0]);
    float ub_ = dot(Gamb, w[2] * lo[2] - w[3] * lo[3]);
    const float coefb = -m / F.W, Wb = m * q / F.W;
    float db = 0.f;
    if (free) {   // coef = mu d / (h |vt|)
        db = coefb * coef / F.d;
        vtb += (-coefb * coef / (sv * sv)) * vt;
    }
    // vt = vrel - (vrel . n) n
    const float vnb = -dot(vtb, F.n);
    const V3<float> vrelb = vtb + vnb * F.n;
    const V3<float> nb = vnb * vrel - vn * vtb;
    Vb[0] = os * vrelb;
    Vb[1] = s * vrelb;
    Vb[2] = (-ou) * vrelb;
    Vb[3] = (-u) * vrelb;
    sb_ += dot(vrelb, Vv[1] - Vv[0]);
    ub_ += dot(vrelb, Vv[2] - Vv[3]);
    pair_fwd_rev(F, P, w, sb_, ub_, nb, db, Wb, Pb);
    return true;
}

}  // namespace dlo
