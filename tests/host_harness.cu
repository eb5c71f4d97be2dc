// Host-side harness: compiles the device element functions of the stepper as host code so
// the CPU test suite can check them against the FP64 oracle without a GPU.
#include "dlo_physics.cuh"

using namespace dlo;

static V3<float> ld3(const float* p) { return V3<float>{p[0], p[1], p[2]}; }
static void st3(float* p, V3<float> a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

// in: xm xi xp tba d1ba tbb d1bb (21) tha thb mprev kbar0 kbar1 mbar lbar Bm beta (9)
// out: U, gxm(3), gxi(3), gxp(3), gtha, gthb, mref, k0, k1, m, d1ra(3), d1rb(3)
extern "C" void hinge_grad_host(const float* in, float* out) {
    HingeF<float> H;
    V3<float> tba = ld3(in + 9), d1ba = ld3(in + 12), tbb = ld3(in + 15), d1bb = ld3(in + 18);
    hinge_forward(H, ld3(in), ld3(in + 3), ld3(in + 6), tba, d1ba, tbb, d1bb, in[21], in[22], in[23]);
    const float il = 1.f / in[27];
    const float gk0 = in[28] * il * (H.k0 - in[24]), gk1 = in[28] * il * (H.k1 - in[25]);
    const float gm = in[29] * il * (H.m - in[26]);
    V3<float> gxm, gxi, gxp;
    float gta, gtb;
    hinge_reverse<float, false>(H, tba, d1ba, tbb, d1bb, gk0, gk1, gm, 0.f, gxm, gxi, gxp, gta, gtb, nullptr,
                                nullptr, nullptr, nullptr);
    out[0] = 0.5f * in[28] * il * ((H.k0 - in[24]) * (H.k0 - in[24]) + (H.k1 - in[25]) * (H.k1 - in[25])) +
             0.5f * in[29] * il * (H.m - in[26]) * (H.m - in[26]);
    st3(out + 1, gxm);
    st3(out + 4, gxi);
    st3(out + 7, gxp);
    out[10] = gta;
    out[11] = gtb;
    out[12] = H.mref;
    out[13] = H.k0;
    out[14] = H.k1;
    out[15] = H.m;
    st3(out + 16, H.a.d1r);
    st3(out + 19, H.b.d1r);
}

// Directional derivative of the full hinge gradient (all 30 inputs) along `dir` (30), by
// running the same reverse pass on dual numbers.  out: 30 tangents of dU/d(input).
extern "C" void hinge_hvp_host(const float* in, const float* dir, float* out) {
    auto D3 = [&](int k) { return V3<dualf>{mkd(in[k], dir[k]), mkd(in[k + 1], dir[k + 1]), mkd(in[k + 2], dir[k + 2])}; };
    auto D1 = [&](int k) { return mkd(in[k], dir[k]); };
    HingeF<dualf> H;
    V3<dualf> tba = D3(9), d1ba = D3(12), tbb = D3(15), d1bb = D3(18);
    hinge_forward(H, D3(0), D3(3), D3(6), tba, d1ba, tbb, d1bb, D1(21), D1(22), D1(23));
    dualf il = 1.f / D1(27);
    dualf e0 = H.k0 - D1(24), e1 = H.k1 - D1(25), em = H.m - D1(26);
    dualf gk0 = D1(28) * il * e0, gk1 = D1(28) * il * e1, gm = D1(29) * il * em;
    V3<dualf> gxm, gxi, gxp, gtba, gd1ba, gtbb, gd1bb;
    dualf gta, gtb;
    hinge_reverse<dualf, true>(H, tba, d1ba, tbb, d1bb, gk0, gk1, gm, mkd(0.f), gxm, gxi, gxp, gta, gtb, &gtba, &gd1ba,
                               &gtbb, &gd1bb);
    V3<float> t;
    t = ders(gxm); out[0] = t.x; out[1] = t.y; out[2] = t.z;
    t = ders(gxi); out[3] = t.x; out[4] = t.y; out[5] = t.z;
    t = ders(gxp); out[6] = t.x; out[7] = t.y; out[8] = t.z;
    t = ders(gtba); out[9] = t.x; out[10] = t.y; out[11] = t.z;
    t = ders(gd1ba); out[12] = t.x; out[13] = t.y; out[14] = t.z;
    t = ders(gtbb); out[15] = t.x; out[16] = t.y; out[17] = t.z;
    t = ders(gd1bb); out[18] = t.x; out[19] = t.y; out[20] = t.z;
    out[21] = gta.d;
    out[22] = gtb.d;
    out[23] = 0.f;                                  // mprev: only through the wrap branch
    out[24] = -gk0.d;                               // dU/dkbar = -gk
    out[25] = -gk1.d;
    out[26] = -gm.d;                                // dU/dmbar = -gm
    dualf gl = -0.5f * (D1(28) * (e0 * e0 + e1 * e1) + D1(29) * em * em) * il * il;
    out[27] = gl.d;
    out[28] = (0.5f * il * (e0 * e0 + e1 * e1)).d;  // dU/dBm
    out[29] = (0.5f * il * em * em).d;              // dU/dbeta
}

// The backward reverses a yielded hinge in one dual pass: the plastic cotangent (le0, le1) of
// the material curvature is added to the derivative part of the curvature seeds, which relies
// on the hinge reverse being linear in its seeds.  in: the 24 hinge inputs of hinge_grad_host,
// dir: their 24 tangents, seeds: gk0, gk1, gm (value, derivative) and le0, le1.
// out[0..22]: derivative parts of the folded dual reverse (gxm gxi gxp gtba gd1ba gtbb gd1bb,
// gta gtb); out[23..45]: the unfolded dual reverse plus the float reverse from (le0, le1).
extern "C" void hinge_fold_host(const float* in, const float* dir, const float* seeds, float* out) {
    auto D3 = [&](int k) { return V3<dualf>{mkd(in[k], dir[k]), mkd(in[k + 1], dir[k + 1]), mkd(in[k + 2], dir[k + 2])}; };
    auto D1 = [&](int k) { return mkd(in[k], dir[k]); };
    HingeF<dualf> Hd;
    V3<dualf> tba = D3(9), d1ba = D3(12), tbb = D3(15), d1bb = D3(18);
    hinge_forward(Hd, D3(0), D3(3), D3(6), tba, d1ba, tbb, d1bb, D1(21), D1(22), D1(23));
    HingeF<float> Hf;
    const V3<float> ftba = ld3(in + 9), fd1ba = ld3(in + 12), ftbb = ld3(in + 15), fd1bb = ld3(in + 18);
    hinge_forward(Hf, ld3(in), ld3(in + 3), ld3(in + 6), ftba, fd1ba, ftbb, fd1bb, in[21], in[22], in[23]);
    const dualf gk0 = mkd(seeds[0], seeds[1]), gk1 = mkd(seeds[2], seeds[3]), gm = mkd(seeds[4], seeds[5]);
    const float le0 = seeds[6], le1 = seeds[7];
    V3<dualf> A[7], B[7];
    dualf a0, a1, b0, b1;
    hinge_reverse<dualf, true>(Hd, tba, d1ba, tbb, d1bb, gk0, gk1, gm, mkd(0.f), A[0], A[1], A[2], a0, a1, &A[3], &A[4],
                               &A[5], &A[6]);
    dualf f0 = gk0, f1 = gk1;
    f0.d += le0;
    f1.d += le1;
    hinge_reverse<dualf, true>(Hd, tba, d1ba, tbb, d1bb, f0, f1, gm, mkd(0.f), B[0], B[1], B[2], b0, b1, &B[3], &B[4],
                               &B[5], &B[6]);
    V3<float> C[7];
    float c0, c1;
    hinge_reverse<float, true>(Hf, ftba, fd1ba, ftbb, fd1bb, le0, le1, 0.f, 0.f, C[0], C[1], C[2], c0, c1, &C[3], &C[4],
                               &C[5], &C[6]);
    for (int k = 0; k < 7; ++k) {
        st3(out + 3 * k, ders(B[k]));
        st3(out + 23 + 3 * k, ders(A[k]) + C[k]);
    }
    out[21] = b0.d;
    out[22] = b1.d;
    out[44] = a0.d + c0;
    out[45] = a1.d + c1;
}

// in: x(3) v(3) vrig(3) sdf_kind (0 plane, 1 box, 2 capsule) params(9) r eps mu rest  out: v'(3), active
extern "C" void contact_host(const float* in, float* out) {
    V3<float> x = ld3(in), v = ld3(in + 3), vr = ld3(in + 6), n;
    int kind = (int)in[9];
    float sdf;
    if (kind == 0) {
        n = ld3(in + 10);
        sdf = dot(x, n) - in[13];
    } else if (kind == 1) {
        sdf = sdf_box(x, ld3(in + 10), ld3(in + 13), n);
    } else {
        sdf = sdf_capsule(x, ld3(in + 10), ld3(in + 13), in[16], n);
    }
    bool act;
    V3<float> o = contact_respond(v, sdf, n, vr, in[19], in[20], in[21], in[22], act);
    st3(out, o);
    out[3] = act ? 1.f : 0.f;
    out[4] = sdf;
}

extern "C" void closest_host(const float* in, float* out) {
    float s, u;
    closest_params(ld3(in), ld3(in + 3), ld3(in + 6), ld3(in + 9), s, u);
    out[0] = s;
    out[1] = u;
}

extern "C" void expmap_host(const float* phi, float* R) {
    M3 m = expmap(ld3(phi));
    for (int k = 0; k < 9; ++k) R[k] = m.m[k];
}

// Capsule-gripper contact: closed-form reverse against dual-number directional derivatives.
// in: x(3) v(3) p(3) ax(3) hl rc vp(3) w(3) r eps mu rest lo(3)  (29)
// out: closed-form (lx, lv, lp, lphi, lvp, lw) then the same from dual numbers (36), active (1)
template <class T>
static V3<T> capsule_eval(V3<T> x, V3<T> v, V3<T> p, V3<T> ax, float hl, float rc, V3<T> vp, V3<T> w, float r,
                          float eps, float mu, float rest, bool& act) {
    V3<T> n;
    T sdf = sdf_capsule(x, p - hl * ax, p + hl * ax, rc, n);
    V3<T> vr = vp + cross(w, x - p);
    return contact_respond(v, sdf, n, vr, r, eps, mu, rest, act);
}
extern "C" void capsule_rev_check(const float* in, float* out) {
    V3<float> x = ld3(in), v = ld3(in + 3), p = ld3(in + 6), ax = ld3(in + 9), vp = ld3(in + 14), w = ld3(in + 17);
    float hl = in[12], rc = in[13], r = in[20], eps = in[21], mu = in[22], rest = in[23];
    V3<float> lo = ld3(in + 24);
    bool on;
    capsule_eval<float>(x, v, p, ax, hl, rc, vp, w, r, eps, mu, rest, on);
    out[36] = on ? 1.f : 0.f;
    V3<float> o[6];
    capsule_contact_rev(x, v, p, ax, hl, rc, vp, w, r, eps, mu, rest, lo, o[0], o[1], o[2], o[3], o[4], o[5]);
    for (int k = 0; k < 6; ++k) st3(out + 3 * k, o[k]);
    for (int d = 0; d < 18; ++d) {
        V3<float> e = zf3();
        (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
        int gi = d / 3;
        bool act;
        V3<dualf> res = capsule_eval<dualf>(lift(x, gi == 0 ? e : zf3()), lift(v, gi == 1 ? e : zf3()),
                                            lift(p, gi == 2 ? e : zf3()), lift(ax, gi == 3 ? cross(e, ax) : zf3()),
                                            hl, rc, lift(vp, gi == 4 ? e : zf3()), lift(w, gi == 5 ? e : zf3()), r,
                                            eps, mu, rest, act);
        out[18 + d] = dot(ders(res), lo);
    }
}

// Plane contact: closed-form reverse against dual numbers.  in: x(3) v(3) n(3) off r eps mu rest lo(3)
// out: lx(3) lv(3) then the dual-number ones (12), active (1)
extern "C" void plane_rev_check(const float* in, float* out) {
    V3<float> x = ld3(in), v = ld3(in + 3), n = ld3(in + 6), lo = ld3(in + 14);
    float off = in[9], r = in[10], eps = in[11], mu = in[12], rest = in[13];
    V3<float> lv, ln, lvr;
    float lsdf;
    bool on;
    contact_respond(v, dot(x, n) - off, n, zf3(), r, eps, mu, rest, on);
    out[12] = on ? 1.f : 0.f;
    contact_respond_rev(v, dot(x, n) - off, n, zf3(), r, eps, mu, rest, lo, lv, lsdf, ln, lvr);
    st3(out, lsdf * n);
    st3(out + 3, lv);
    for (int d = 0; d < 6; ++d) {
        V3<float> e = zf3();
        (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
        V3<dualf> xd = lift(x, d < 3 ? e : zf3()), vd = lift(v, d >= 3 ? e : zf3());
        V3<dualf> nd = lift(n);
        dualf sdf = dot(xd, nd) - off;
        bool act;
        V3<dualf> res = contact_respond(vd, sdf, nd, lift(zf3()), r, eps, mu, rest, act);
        out[6 + d] = dot(ders(res), lo);
    }
}

// Self-contact projection and friction of one segment pair: closed-form vector-Jacobian products
// against dual-number directional derivatives through the forward code.
// in: P(12) V(12) w(4) rsum mu h lo_x(12) lo_v(12)  (55)
// out: projection Pb (12) then dual (12); friction Pb (12), Vb (12) then dual (24); flags (2)
extern "C" void pair_vjp_check(const float* in, float* out) {
    V3<float> P[4], Vv[4], lx[4], lv[4];
    float w[4];
    for (int k = 0; k < 4; ++k) {
        P[k] = ld3(in + 3 * k);
        Vv[k] = ld3(in + 12 + 3 * k);
        w[k] = in[24 + k];
        lx[k] = ld3(in + 31 + 3 * k);
        lv[k] = ld3(in + 43 + 3 * k);
    }
    const float rsum = in[28], mu = in[29], h = in[30];
    for (int i = 0; i < 74; ++i) out[i] = 0.f;
    V3<float> pb[4], vb[4];
    const bool on = pair_correction_vjp(P, w, rsum, lx, pb);
    out[72] = on ? 1.f : 0.f;
    if (on)
        for (int k = 0; k < 4; ++k) st3(out + 3 * k, pb[k]);
    for (int d = 0; d < 12; ++d) {
        V3<dualf> Pd[4], dx[4], n;
        dualf s, u, dd, W;
        for (int k = 0; k < 4; ++k) {
            V3<float> e = zf3();
            if (d / 3 == k) (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
            Pd[k] = lift(P[k], e);
        }
        float acc = 0.f;
        if (pair_correction(Pd[0], Pd[1], Pd[2], Pd[3], w[0], w[1], w[2], w[3], rsum, dx, s, u, n, dd, W))
            for (int k = 0; k < 4; ++k) acc += dot(ders(dx[k]), lx[k]);
        out[12 + d] = acc;
    }
    const bool fon = fric_pair_vjp(P, Vv, w, rsum, mu, h, lv, pb, vb);
    out[73] = fon ? 1.f : 0.f;
    if (fon)
        for (int k = 0; k < 4; ++k) {
            st3(out + 24 + 3 * k, pb[k]);
            st3(out + 36 + 3 * k, vb[k]);
        }
    for (int d = 0; d < 24; ++d) {
        V3<dualf> Pd[4], Vd[4], dv[4];
        for (int k = 0; k < 4; ++k) {
            V3<float> ep = zf3(), ev = zf3();
            if (d / 3 == k) (d % 3 == 0 ? ep.x : d % 3 == 1 ? ep.y : ep.z) = 1.f;
            if (d / 3 == 4 + k) (d % 3 == 0 ? ev.x : d % 3 == 1 ? ev.y : ev.z) = 1.f;
            Pd[k] = lift(P[k], ep);
            Vd[k] = lift(Vv[k], ev);
        }
        float acc = 0.f;
        if (fric_pair(Pd, Vd, w, rsum, mu, h, dv))
            for (int k = 0; k < 4; ++k) acc += dot(ders(dv[k]), lv[k]);
        out[48 + d] = acc;
    }
}

// Box contact: closed-form reverse against dual numbers.  in: x(3) v(3) c(3) hl(3) r eps mu rest lo(3)
// out: lx(3) lv(3) then the dual-number ones (12), active (1)
extern "C" void box_rev_check(const float* in, float* out) {
    V3<float> x = ld3(in), v = ld3(in + 3), c = ld3(in + 6), hl = ld3(in + 9), lo = ld3(in + 16);
    float r = in[12], eps = in[13], mu = in[14], rest = in[15];
    V3<float> n;
    bool on;
    contact_respond(v, sdf_box(x, c, hl, n), n, zf3(), r, eps, mu, rest, on);
    out[12] = on ? 1.f : 0.f;
    for (int i = 0; i < 12; ++i) out[i] = 0.f;
    if (!on) return;
    V3<float> lv;
    st3(out, box_contact_rev(x, v, c, hl, r, eps, mu, rest, lo, lv));
    st3(out + 3, lv);
    for (int d = 0; d < 6; ++d) {
        V3<float> e = zf3();
        (d % 3 == 0 ? e.x : d % 3 == 1 ? e.y : e.z) = 1.f;
        V3<dualf> xd = lift(x, d < 3 ? e : zf3()), vd = lift(v, d >= 3 ? e : zf3()), nd;
        dualf sdf = sdf_box(xd, c, hl, nd);
        bool act;
        V3<dualf> res = contact_respond(vd, sdf, nd, lift(zf3()), r, eps, mu, rest, act);
        out[6 + d] = dot(ders(res), lo);
    }
}
