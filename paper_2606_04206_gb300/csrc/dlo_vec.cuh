// dlo_vec.cuh -- small vector and forward-mode dual-number types for the rod kernels.
//
// Every element function of the stepper is written once as a template on its scalar type.
// With float it is the forward step; with dualf (value + one directional derivative) the
// same code yields Jacobian-vector products, which the adjoint kernels use.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace dlo {

#define DLO_HD __host__ __device__ __forceinline__

// ----------------------------------------------------------------- dual numbers
struct dualf {
    float v, d;
};

DLO_HD dualf mkd(float v, float d = 0.f) { return dualf{v, d}; }
DLO_HD float vof(float a) { return a; }
DLO_HD float vof(dualf a) { return a.v; }
DLO_HD float dof(float) { return 0.f; }
DLO_HD float dof(dualf a) { return a.d; }

DLO_HD dualf operator+(dualf a, dualf b) { return {a.v + b.v, a.d + b.d}; }
DLO_HD dualf operator-(dualf a, dualf b) { return {a.v - b.v, a.d - b.d}; }
DLO_HD dualf operator*(dualf a, dualf b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
// Quotient of a derivative part.  The value parts keep IEEE division, so that a dual
// evaluation's values (and the branches taken on them) are those of the float evaluation;
// a derivative tolerates the fast quotient's 2 ulp and then needs no IEEE slow path.
DLO_HD float ddiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
DLO_HD dualf operator/(dualf a, dualf b) {
    float q = a.v / b.v;
    return {q, ddiv(a.d - q * b.d, b.v)};
}
DLO_HD dualf operator-(dualf a) { return {-a.v, -a.d}; }
DLO_HD dualf operator+(dualf a, float b) { return {a.v + b, a.d}; }
DLO_HD dualf operator+(float a, dualf b) { return {a + b.v, b.d}; }
DLO_HD dualf operator-(dualf a, float b) { return {a.v - b, a.d}; }
DLO_HD dualf operator-(float a, dualf b) { return {a - b.v, -b.d}; }
DLO_HD dualf operator*(dualf a, float b) { return {a.v * b, a.d * b}; }
DLO_HD dualf operator*(float a, dualf b) { return {a * b.v, a * b.d}; }
DLO_HD dualf operator/(dualf a, float b) { return {a.v / b, ddiv(a.d, b)}; }
DLO_HD dualf operator/(float a, dualf b) {
    float q = a / b.v;
    return {q, -ddiv(q * b.d, b.v)};
}
DLO_HD dualf& operator+=(dualf& a, dualf b) { a = a + b; return a; }
DLO_HD dualf& operator-=(dualf& a, dualf b) { a = a - b; return a; }
DLO_HD dualf& operator*=(dualf& a, dualf b) { a = a * b; return a; }

DLO_HD float dsqrt(float a) { return sqrtf(a); }
DLO_HD dualf dsqrt(dualf a) {
    float s = sqrtf(a.v);
    return {s, s > 0.f ? ddiv(0.5f * a.d, s) : 0.f};
}
DLO_HD float dsin(float a) { return sinf(a); }
DLO_HD float dcos(float a) { return cosf(a); }
DLO_HD dualf dsin(dualf a) { return {sinf(a.v), cosf(a.v) * a.d}; }
DLO_HD dualf dcos(dualf a) { return {cosf(a.v), -sinf(a.v) * a.d}; }
DLO_HD float dexp(float a) { return expf(a); }
DLO_HD dualf dexp(dualf a) {
    float e = expf(a.v);
    return {e, e * a.d};
}
DLO_HD float datan2(float y, float x) { return atan2f(y, x); }
DLO_HD dualf datan2(dualf y, dualf x) {
    float r2 = x.v * x.v + y.v * y.v;
    return {atan2f(y.v, x.v), ddiv(x.v * y.d - y.v * x.d, r2)};
}
template <class T> DLO_HD T cst(float a);
template <> DLO_HD float cst<float>(float a) { return a; }
template <> DLO_HD dualf cst<dualf>(float a) { return dualf{a, 0.f}; }
// min / max / clamp select by value; the derivative follows the selected branch
template <class T> DLO_HD T dmin(T a, T b) { return vof(a) <= vof(b) ? a : b; }
template <class T> DLO_HD T dmax(T a, T b) { return vof(a) >= vof(b) ? a : b; }
template <class T> DLO_HD T dclamp(T a, float lo, float hi) {
    return vof(a) < lo ? cst<T>(lo) : (vof(a) > hi ? cst<T>(hi) : a);
}

// ----------------------------------------------------------------- 3-vectors
template <class T>
struct V3 {
    T x, y, z;
};

template <class T> DLO_HD V3<T> mk3(T x, T y, T z) { return V3<T>{x, y, z}; }
DLO_HD V3<float> f3(float4 a) { return V3<float>{a.x, a.y, a.z}; }
DLO_HD V3<float> f3(float x, float y, float z) { return V3<float>{x, y, z}; }
DLO_HD V3<dualf> lift(V3<float> a) { return V3<dualf>{mkd(a.x), mkd(a.y), mkd(a.z)}; }
DLO_HD V3<dualf> lift(V3<float> a, V3<float> d) {
    return V3<dualf>{mkd(a.x, d.x), mkd(a.y, d.y), mkd(a.z, d.z)};
}
DLO_HD V3<float> vals(V3<dualf> a) { return V3<float>{a.x.v, a.y.v, a.z.v}; }
DLO_HD V3<float> vals(V3<float> a) { return a; }
DLO_HD V3<float> ders(V3<dualf> a) { return V3<float>{a.x.d, a.y.d, a.z.d}; }

template <class T> DLO_HD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> DLO_HD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> DLO_HD V3<T> operator-(V3<T> a) { return {-a.x, -a.y, -a.z}; }
template <class T> DLO_HD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> DLO_HD V3<T> operator*(V3<T> a, T s) { return {s * a.x, s * a.y, s * a.z}; }
DLO_HD V3<dualf> operator*(float s, V3<dualf> a) { return {s * a.x, s * a.y, s * a.z}; }
DLO_HD V3<dualf> operator*(dualf s, V3<float> a) { return {s * a.x, s * a.y, s * a.z}; }
// one reciprocal and three products (float and dual alike, so their values agree)
template <class T> DLO_HD V3<T> operator/(V3<T> a, T s) {
    const T r = 1.f / s;
    return {a.x * r, a.y * r, a.z * r};
}
template <class T> DLO_HD V3<T>& operator+=(V3<T>& a, V3<T> b) { a = a + b; return a; }
template <class T> DLO_HD V3<T>& operator-=(V3<T>& a, V3<T> b) { a = a - b; return a; }
template <class T> DLO_HD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> DLO_HD V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> DLO_HD T norm(V3<T> a) { return dsqrt(dot(a, a)); }
template <class T> DLO_HD V3<T> zero3() { return V3<T>{T(), T(), T()}; }
DLO_HD V3<float> zf3() { return V3<float>{0.f, 0.f, 0.f}; }
DLO_HD float4 f4(V3<float> a, float w) { return make_float4(a.x, a.y, a.z, w); }

// 3x3 rotation matrices (row major) for the gripper poses
struct M3 {
    float m[9];
};
DLO_HD V3<float> mul(const M3& R, V3<float> a) {
    return {R.m[0] * a.x + R.m[1] * a.y + R.m[2] * a.z, R.m[3] * a.x + R.m[4] * a.y + R.m[5] * a.z,
            R.m[6] * a.x + R.m[7] * a.y + R.m[8] * a.z};
}
DLO_HD V3<float> mulT(const M3& R, V3<float> a) {
    return {R.m[0] * a.x + R.m[3] * a.y + R.m[6] * a.z, R.m[1] * a.x + R.m[4] * a.y + R.m[7] * a.z,
            R.m[2] * a.x + R.m[5] * a.y + R.m[8] * a.z};
}
DLO_HD M3 matmul(const M3& A, const M3& B) {
    M3 C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C.m[3 * i + j] = A.m[3 * i] * B.m[j] + A.m[3 * i + 1] * B.m[3 + j] + A.m[3 * i + 2] * B.m[6 + j];
    return C;
}
DLO_HD V3<float> col(const M3& R, int j) { return {R.m[j], R.m[3 + j], R.m[6 + j]}; }

// Rotation exp([phi]x) by Rodrigues' formula; (1 - cos t)/t^2 written as 2 sin^2(t/2)/t^2
// to avoid cancellation in float; Taylor series for tiny angles.
DLO_HD M3 expmap(V3<float> p) {
    float t2 = dot(p, p), A, B;
    if (t2 < 1e-8f) {
        A = 1.f - t2 / 6.f;
        B = 0.5f - t2 / 24.f;
    } else {
        float t = sqrtf(t2), sh = sinf(0.5f * t);
        A = sinf(t) / t;
        B = 2.f * sh * sh / t2;
    }
    M3 R;
    R.m[0] = 1.f - B * (p.y * p.y + p.z * p.z);
    R.m[4] = 1.f - B * (p.x * p.x + p.z * p.z);
    R.m[8] = 1.f - B * (p.x * p.x + p.y * p.y);
    R.m[1] = -A * p.z + B * p.x * p.y;
    R.m[3] = A * p.z + B * p.x * p.y;
    R.m[2] = A * p.y + B * p.x * p.z;
    R.m[6] = -A * p.y + B * p.x * p.z;
    R.m[5] = -A * p.x + B * p.y * p.z;
    R.m[7] = A * p.x + B * p.y * p.z;
    return R;
}

}  // namespace dlo
