// Operation count of one rod-vertex-substep of the stepper, taken by running the device
// element functions (compiled for the host) on a counting scalar.  Each edge's reference
// frame and its reverse are counted once (the hinge-local kernel evaluates them for both of
// an edge's hinges; that duplication is not part of the algorithm).
#include <cstdio>

#include "dlo_vec.cuh"

namespace dlo {
struct CountF;
}
static long long g_add = 0, g_mul = 0, g_div = 0, g_sqrt = 0, g_special = 0;

namespace dlo {
struct CountF {
    float v;
};
inline CountF operator+(CountF a, CountF b) { ++g_add; return {a.v + b.v}; }
inline CountF operator-(CountF a, CountF b) { ++g_add; return {a.v - b.v}; }
inline CountF operator*(CountF a, CountF b) { ++g_mul; return {a.v * b.v}; }
inline CountF operator/(CountF a, CountF b) { ++g_div; return {a.v / b.v}; }
inline CountF operator-(CountF a) { return {-a.v}; }
inline CountF operator+(CountF a, float b) { ++g_add; return {a.v + b}; }
inline CountF operator+(float a, CountF b) { ++g_add; return {a + b.v}; }
inline CountF operator-(CountF a, float b) { ++g_add; return {a.v - b}; }
inline CountF operator-(float a, CountF b) { ++g_add; return {a - b.v}; }
inline CountF operator*(CountF a, float b) { ++g_mul; return {a.v * b}; }
inline CountF operator*(float a, CountF b) { ++g_mul; return {a * b.v}; }
inline CountF operator/(CountF a, float b) { ++g_div; return {a.v / b}; }
inline CountF operator/(float a, CountF b) { ++g_div; return {a / b.v}; }
inline CountF& operator+=(CountF& a, CountF b) { a = a + b; return a; }
inline CountF& operator-=(CountF& a, CountF b) { a = a - b; return a; }
inline float vof(CountF a) { return a.v; }
inline CountF dsqrt(CountF a) { ++g_sqrt; return {sqrtf(a.v)}; }
inline CountF dsin(CountF a) { ++g_special; return {sinf(a.v)}; }
inline CountF dcos(CountF a) { ++g_special; return {cosf(a.v)}; }
inline CountF dexp(CountF a) { ++g_special; return {expf(a.v)}; }
inline CountF datan2(CountF y, CountF x) { ++g_special; return {atan2f(y.v, x.v)}; }
template <> inline CountF cst<CountF>(float a) { return {a}; }

// forward-mode dual number over the counting scalar: each dual operation costs the float
// operations it needs (value and one derivative)
struct DC {
    CountF v, d;
};
inline DC operator+(DC a, DC b) { return {a.v + b.v, a.d + b.d}; }
inline DC operator-(DC a, DC b) { return {a.v - b.v, a.d - b.d}; }
inline DC operator*(DC a, DC b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline DC operator/(DC a, DC b) {
    CountF q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
inline DC operator-(DC a) { return {-a.v, -a.d}; }
inline DC operator+(DC a, float b) { return {a.v + b, a.d}; }
inline DC operator+(float a, DC b) { return {a + b.v, b.d}; }
inline DC operator-(DC a, float b) { return {a.v - b, a.d}; }
inline DC operator-(float a, DC b) { return {a - b.v, -b.d}; }
inline DC operator*(DC a, float b) { return {a.v * b, a.d * b}; }
inline DC operator*(float a, DC b) { return {a * b.v, a * b.d}; }
inline DC operator/(DC a, float b) { return {a.v / b, a.d / b}; }
inline DC operator/(float a, DC b) {
    CountF q = a / b.v;
    return {q, (-q) * b.d / b.v};
}
inline DC& operator+=(DC& a, DC b) { a = a + b; return a; }
inline DC& operator-=(DC& a, DC b) { a = a - b; return a; }
inline float vof(DC a) { return a.v.v; }
inline DC dsqrt(DC a) {
    CountF s = dsqrt(a.v);
    return {s, 0.5f * a.d / s};
}
inline DC dsin(DC a) { return {dsin(a.v), dcos(a.v) * a.d}; }
inline DC dcos(DC a) { return {dcos(a.v), -(dsin(a.v) * a.d)}; }
inline DC dexp(DC a) {
    CountF e = dexp(a.v);
    return {e, e * a.d};
}
inline DC datan2(DC y, DC x) {
    CountF r2 = x.v * x.v + y.v * y.v;
    return {datan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2};
}
template <> inline DC cst<DC>(float a) { return {{a}, {0.f}}; }
// a vector over a scalar is three quotients, however the kernels form them (one reciprocal
// and three products)
inline V3<CountF> operator/(V3<CountF> a, CountF s) { return {a.x / s, a.y / s, a.z / s}; }
inline V3<DC> operator/(V3<DC> a, DC s) { return {a.x / s, a.y / s, a.z / s}; }
}  // namespace dlo

#include "dlo_physics.cuh"

using namespace dlo;
using T = CountF;

static void reset() { g_add = g_mul = g_div = g_sqrt = g_special = 0; }
static long long flops() { return g_add + g_mul + g_div + g_sqrt + g_special; }
static V3<T> c3(float x, float y, float z) { return V3<T>{{x}, {y}, {z}}; }

int main() {
    V3<T> xm = c3(0.f, 0.f, 0.f), xi = c3(0.01f, 0.001f, 0.f), xp = c3(0.02f, 0.f, 0.001f);
    V3<T> tb = c3(1.f, 0.f, 0.f), d1 = c3(0.f, 0.f, 1.f);
    T th{0.1f}, mp{0.f};
    // edge frame (once per edge) and its reverse (once per edge)
    reset();
    EdgeF<T> E;
    edge_forward(E, xm, xi, tb, d1, th);
    const long long edge_f = flops();
    reset();
    edge_reverse<T, false>(E, tb, d1, c3(1, 2, 3), c3(1, 1, 1), T{0.f}, nullptr, nullptr);
    const long long edge_r = flops();
    // hinge forward and reverse (each contains two edge frames / reverses)
    reset();
    HingeF<T> H;
    hinge_forward(H, xm, xi, xp, tb, d1, tb, d1, th, th, mp);
    const long long hinge_f = flops();
    reset();
    V3<T> a, b, c;
    T ta, tb2;
    hinge_reverse<T, false>(H, tb, d1, tb, d1, T{0.1f}, T{0.2f}, T{0.3f}, T{0.f}, a, b, c, ta, tb2, nullptr,
                            nullptr, nullptr, nullptr);
    const long long hinge_r = flops();
    // energy seeds of one hinge: 3 (1/lbar products) + 3 differences
    const long long seeds = 9;
    // rigid contact of one vertex against one plane when it is not in contact: d, f, test
    reset();
    {
        V3<T> n = c3(0, 0, 1);
        T sdf = dot(xi, n) - (-1.f);
        bool act;
        contact_respond(c3(0, 0, -1), sdf, n, c3(0, 0, 0), 0.002f, 0.001f, 0.5f, 0.f, act);
    }
    const long long plane_far = flops();
    // rigid contact of one vertex against a capsule gripper, not in contact
    reset();
    {
        V3<T> n;
        T sdf = sdf_capsule(xi, c3(0.5f, 0, 0), c3(0.5f, 0, 0.04f), 0.01f, n);
        V3<T> vr = c3(0.1f, 0, 0) + cross(c3(0, 0, 1), xi - c3(0.5f, 0, 0.02f));
        bool act;
        contact_respond(c3(0, 0, -1), sdf, n, vr, 0.002f, 0.001f, 0.5f, 0.f, act);
    }
    const long long capsule_far = flops();
    // plasticity of one hinge (yield test and return mapping): e (2), |e|^2 (3), sqrt,
    // threshold product, g (3), update (4)
    const long long plastic = 14;
    // stretching of one edge: e, |e|, t, (|e|/eb - 1), force (3+5+3+2+4)
    const long long stretch = 17;
    // vertex update: gradient gather (3 hinge slots + 2 stretch terms: 12 adds), gravity,
    // damping and symplectic Euler (v1 = v + h(-w g + grav - c v): 12), displacement (3),
    // velocity rebuild (3), position (3), twist-rate and angle update (6)
    const long long vertex = 39;
    // one inextensibility projection of one edge: e (6), |e| (5), lambda (3), t (3), two
    // corrections (12)
    const long long inext = 29;
    // per vertex-substep: one hinge (its core without the two edge frames / reverses) plus one
    // edge frame, one edge reverse and one stretch term, the vertex update, one plane and two
    // capsule tests, plasticity on the plastic third, N_C = 10 projections on the cable third
    const long long core = (hinge_f - 2 * edge_f) + (hinge_r - 2 * edge_r) + seeds + edge_f + edge_r;
    const double per_vs = core + stretch + vertex + plane_far + 2.0 * capsule_far + plastic / 3.0 + 10.0 * inext / 3.0;
    // ---- adjoint: the same hinge on dual numbers (second order), edge base reverse
    auto D3 = [](float x, float y, float z) { return V3<DC>{{{x}, {0.1f}}, {{y}, {0.2f}}, {{z}, {0.3f}}}; };
    V3<DC> dxm = D3(0, 0, 0), dxi = D3(0.01f, 0.001f, 0), dxp = D3(0.02f, 0, 0.001f);
    V3<DC> dtb = D3(1, 0, 0), dd1 = D3(0, 0, 1);
    DC dth{{0.1f}, {1.f}}, dmp{{0.f}, {0.f}};
    reset();
    EdgeF<DC> DE;
    edge_forward(DE, dxm, dxi, dtb, dd1, dth);
    const long long edge_f_d = flops();
    reset();
    { V3<DC> q1, q2; edge_reverse<DC, true>(DE, dtb, dd1, D3(1, 2, 3), D3(1, 1, 1), DC{{0.f}, {0.f}}, &q1, &q2); }
    const long long edge_r_d = flops();
    reset();
    HingeF<DC> DH;
    hinge_forward(DH, dxm, dxi, dxp, dtb, dd1, dtb, dd1, dth, dth, dmp);
    const long long hinge_f_d = flops();
    reset();
    {
        V3<DC> q[7];
        DC ta2, tb3;
        hinge_reverse<DC, true>(DH, dtb, dd1, dtb, dd1, DC{{0.1f}, {1.f}}, DC{{0.2f}, {1.f}}, DC{{0.3f}, {1.f}},
                                DC{{0.f}, {0.f}}, q[0], q[1], q[2], ta2, tb3, &q[3], &q[4], &q[5], &q[6]);
    }
    const long long hinge_r_d = flops();
    reset();
    { V3<T> q1, q2; edge_reverse<T, true>(E, tb, d1, c3(1, 2, 3), c3(1, 1, 1), T{0.f}, &q1, &q2); }
    const long long edge_r_base = flops();
    const long long core_d = (hinge_f_d - 2 * edge_f_d) + (hinge_r_d - 2 * edge_r_d) + edge_f_d + edge_r_d + 2 * seeds;
    // vertex reverse: contact sequence recompute (one plane, two capsules), symplectic-Euler,
    // damping, twist-rate reverse (~30); stretching Hessian-vector product (~25); gradient
    // gather of the reverse (~12); one inextensibility projection reverse (~45)
    const double adj_vs = core_d + edge_r_base + 30 + plane_far + 2.0 * capsule_far + 25 + 12 + 10.0 * (inext + 45) / 3.0;
    std::printf("{\"edge_frame\": %lld, \"edge_reverse\": %lld, \"hinge_forward\": %lld, \"hinge_reverse\": %lld, "
                "\"plane_far\": %lld, \"capsule_far\": %lld, \"core\": %lld, \"forward_per_vertex_substep\": %.1f, "
                "\"dual_core\": %lld, \"adjoint_per_vertex_substep\": %.1f, "
                "\"backward_per_vertex_substep\": %.1f}\n",
                edge_f, edge_r, hinge_f, hinge_r, plane_far, capsule_far, core, per_vs, core_d, adj_vs,
                per_vs + adj_vs);
    return 0;
}
