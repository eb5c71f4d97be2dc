// dlo_loss.cu -- task losses of App. B ("Reward design") on the device, per rod, with their
// gradient with respect to the vertex positions (the dL/dx_T that dlo_backward takes).
// One CTA per rod; sums are reduced in double in a fixed order, and every gradient is
// gathered without atomics, so results are deterministic.
#include <cmath>

#include "dlo_runtime.h"
#include "dlo_vec.cuh"
#include "dlo_physics.cuh"

namespace dlo {
namespace {

constexpr int kLT = 128;          // threads per rod
constexpr int kMaxPoints = 1024;  // Chamfer point set size per rod
constexpr int kMaxV = 256;        // vertices per rod

__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kLT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float gscale(const float* g, int rod) { return g ? g[rod] : 1.f; }

// (1/N) sum_i |x_i - t_i|^2
__global__ void loss_target(const RodInfo* rods, const float4* X, const float4* Tg, const float* g, float* q,
                            float4* gx) {
    __shared__ double sh[kLT];
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const float c = 2.f * gscale(g, rod) / (float)R.nv;
    double s = 0.0;
    for (int i = threadIdx.x; i < R.nv; i += kLT) {
        const V3<float> d = f3(X[R.v0 + i]) - f3(Tg[R.v0 + i]);
        s += (double)dot(d, d);
        if (gx) gx[R.v0 + i] = f4(c * d, 0.f);
    }
    s = block_sum(s, sh);
    if (q && threadIdx.x == 0) q[rod] = (float)(s / R.nv);
}

// (1/N) sum_i min_j |x_i - y_j|^2 + (1/M) sum_j min_i |x_i - y_j|^2
__global__ void loss_chamfer(const RodInfo* rods, const float4* X, const float4* Y, int m, const float* g,
                             float* q, float4* gx) {
    __shared__ double sh[kLT];
    __shared__ float4 xs[kMaxV];
    __shared__ float4 ys[kMaxPoints];
    __shared__ short nn[kMaxPoints];   // nearest vertex of each point
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const int n = R.nv;
    for (int i = threadIdx.x; i < n; i += kLT) xs[i] = X[R.v0 + i];
    for (int j = threadIdx.x; j < m; j += kLT) ys[j] = Y[(size_t)rod * m + j];
    __syncthreads();
    const float gs = gscale(g, rod);
    double s = 0.0;
    // points to their nearest vertex
    for (int j = threadIdx.x; j < m; j += kLT) {
        const V3<float> y = f3(ys[j]);
        float best = INFINITY;
        int bi = 0;
        for (int i = 0; i < n; ++i) {
            const V3<float> d = f3(xs[i]) - y;
            const float d2 = dot(d, d);
            if (d2 < best) {
                best = d2;
                bi = i;
            }
        }
        nn[j] = (short)bi;
        s += (double)best / m;
    }
    __syncthreads();
    // vertices to their nearest point, and the gradient of both terms at each vertex
    for (int i = threadIdx.x; i < n; i += kLT) {
        const V3<float> x = f3(xs[i]);
        float best = INFINITY;
        int bj = 0;
        V3<float> acc = zf3();
        for (int j = 0; j < m; ++j) {
            const V3<float> d = x - f3(ys[j]);
            const float d2 = dot(d, d);
            if (d2 < best) {
                best = d2;
                bj = j;
            }
            if (nn[j] == i) acc += (2.f / m) * d;
        }
        s += (double)best / n;
        if (gx) gx[R.v0 + i] = f4(gs * ((2.f / n) * (x - f3(ys[bj])) + acc), 0.f);
    }
    s = block_sum(s, sh);
    if (q && threadIdx.x == 0) q[rod] = (float)s;
}

// (1/2pi) sum over segments of the signed angle they subtend at the post (xy-plane); the sum
// telescopes, so only the two ends of an open rod carry gradient: d(phi_j) = (-a_y, a_x) / |a|^2
__global__ void loss_winding(const RodInfo* rods, const float4* X, const float4* posts, const float* g, float* q,
                             float4* gx) {
    __shared__ double sh[kLT];
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const bool closed = R.flags & ROD_CLOSED;
    const int n = R.nv, ne = closed ? n : n - 1;
    const float px = posts[rod].x, py = posts[rod].y;
    double s = 0.0;
    for (int j = threadIdx.x; j < ne; j += kLT) {
        const int j1 = (j + 1 == n) ? 0 : j + 1;
        const float ax = X[R.v0 + j].x - px, ay = X[R.v0 + j].y - py;
        const float bx = X[R.v0 + j1].x - px, by = X[R.v0 + j1].y - py;
        s += (double)atan2f(ax * by - ay * bx, ax * bx + ay * by);
    }
    s = block_sum(s, sh);
    if (q && threadIdx.x == 0) q[rod] = (float)(s / (2.0 * M_PI));
    if (!gx) return;
    const float c = gscale(g, rod) / (2.f * (float)M_PI);
    for (int i = threadIdx.x; i < n; i += kLT) {
        const float coef = closed ? 0.f : (i == n - 1 ? 1.f : (i == 0 ? -1.f : 0.f));
        const float ax = X[R.v0 + i].x - px, ay = X[R.v0 + i].y - py;
        const float r2 = ax * ax + ay * ay;
        gx[R.v0 + i] = coef != 0.f && r2 > 0.f ? make_float4(c * coef * -ay / r2, c * coef * ax / r2, 0.f, 0.f)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ---- the Gauss double integral of two straight segments (exact closed form) on dual numbers.
// The directions r_2 - r_1 of the pair sweep the parallelogram r13, r14, r24, r23; the integral
// is minus its signed solid angle seen from the origin, taken as two triangles with the
// atan2 form of Van Oosterom and Strackee (IEEE TBME 1983), which stays well conditioned in
// float where the arcsine form of the same angle loses its derivative.
__device__ dualf gauss_pair_d(V3<dualf> p1, V3<dualf> p2, V3<dualf> p3, V3<dualf> p4) {
    const V3<dualf> r13 = p3 - p1, r14 = p4 - p1, r23 = p3 - p2, r24 = p4 - p2;
    const dualf l13 = norm(r13), l14 = norm(r14), l23 = norm(r23), l24 = norm(r24);
    const dualf d13_24 = dot(r13, r24);
    const dualf n1 = dot(r13, cross(r14, r24));
    const dualf m1 = l13 * l14 * l24 + dot(r13, r14) * l24 + d13_24 * l14 + dot(r14, r24) * l13;
    const dualf n2 = dot(r13, cross(r24, r23));
    const dualf m2 = l13 * l24 * l23 + d13_24 * l23 + dot(r13, r23) * l24 + dot(r24, r23) * l13;
    return -2.f * (datan2(n1, m1) + datan2(n2, m2));
}

// sum over ordered pairs of non-adjacent edges of Omega / (4 pi); thread of edge a evaluates
// Omega(a, b) for every b with the six coordinates of a's endpoints seeded in turn
__global__ void loss_crossing(const RodInfo* rods, const float4* X, const float* g, float* q, float4* gx) {
    __shared__ double sh[kLT];
    __shared__ float4 xs[kMaxV];
    __shared__ float4 ge0[kMaxV], ge1[kMaxV];   // d/d(first, second endpoint) of each edge's sum
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const bool closed = R.flags & ROD_CLOSED;
    const int n = R.nv, ne = closed ? n : n - 1;
    for (int i = threadIdx.x; i < n; i += kLT) xs[i] = X[R.v0 + i];
    __syncthreads();
    double s = 0.0;
    for (int a = threadIdx.x; a < ne; a += kLT) {
        const int a1 = (a + 1 == n) ? 0 : a + 1;
        const V3<float> pa = f3(xs[a]), pb = f3(xs[a1]);
        float gq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < ne; ++b) {
            int sep = abs(a - b);
            if (closed) sep = min(sep, ne - sep);
            if (sep <= 1) continue;
            const int b1 = (b + 1 == n) ? 0 : b + 1;
            const V3<dualf> p3 = lift(f3(xs[b])), p4 = lift(f3(xs[b1]));
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                V3<float> e1 = zf3(), e2 = zf3();
                if (k < 3) (k == 0 ? e1.x : k == 1 ? e1.y : e1.z) = 1.f;
                else (k == 3 ? e2.x : k == 4 ? e2.y : e2.z) = 1.f;
                const dualf om = gauss_pair_d(lift(pa, e1), lift(pb, e2), p3, p4);
                if (k == 0) s += (double)om.v;
                gq[k] += om.d;
            }
        }
        ge0[a] = make_float4(gq[0], gq[1], gq[2], 0.f);
        ge1[a] = make_float4(gq[3], gq[4], gq[5], 0.f);
    }
    __syncthreads();
    s = block_sum(s, sh);
    if (q && threadIdx.x == 0) q[rod] = (float)(s / (4.0 * M_PI));
    if (!gx) return;
    // each unordered pair appears twice in the sum: d/dx = 2 sum_b dOmega_ab / (4 pi)
    const float c = gscale(g, rod) / (2.f * (float)M_PI);
    for (int i = threadIdx.x; i < n; i += kLT) {
        V3<float> d = zf3();
        if (closed || i < ne) d += f3(ge0[i]);                         // i starts edge i
        if (closed || i > 0) d += f3(ge1[i == 0 ? ne - 1 : i - 1]);     // and ends edge i-1
        gx[R.v0 + i] = f4(c * d, 0.f);
    }
}

// min_i |x_i - o|; the subgradient at the nearest vertex (lowest index on a tie)
__global__ void loss_mindist(const RodInfo* rods, const float4* X, const float4* obj, const float* g, float* q,
                             float4* gx) {
    __shared__ float bd[kLT];
    __shared__ int bi[kLT];
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const V3<float> o = f3(obj[rod]);
    float best = INFINITY;
    int arg = 0;
    for (int i = threadIdx.x; i < R.nv; i += kLT) {
        const V3<float> d = f3(X[R.v0 + i]) - o;
        const float d2 = dot(d, d);
        if (d2 < best) {   // strict: a thread's own vertices come in increasing order
            best = d2;
            arg = i;
        }
    }
    bd[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int s = kLT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const float d2 = bd[threadIdx.x + s];
            const int i2 = bi[threadIdx.x + s];
            if (d2 < bd[threadIdx.x] || (d2 == bd[threadIdx.x] && i2 < bi[threadIdx.x])) {
                bd[threadIdx.x] = d2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const float dmin = sqrtf(bd[0]);
    const int imin = bi[0];
    if (q && threadIdx.x == 0) q[rod] = dmin;
    if (!gx) return;
    const float c = dmin > 0.f ? gscale(g, rod) / dmin : 0.f;
    for (int i = threadIdx.x; i < R.nv; i += kLT)
        gx[R.v0 + i] = i == imin ? f4(c * (f3(X[R.v0 + i]) - o), 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// sum over unordered pairs of edges more than k apart of max(0, delta - d)^2, d the distance of
// the segments' closest points.  The closest-point parameters are each optimal for the other
// (or fixed), so the gradient holds them fixed: dd/dx_a0 = (1 - s) n, dd/dx_a1 = s n.
__global__ void loss_repulsion(const RodInfo* rods, const float4* X, const float4* prm, const float* g, float* q,
                               float4* gx) {
    __shared__ double sh[kLT];
    __shared__ float4 xs[kMaxV];
    __shared__ float4 ge0[kMaxV], ge1[kMaxV];
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const bool closed = R.flags & ROD_CLOSED;
    const int n = R.nv, ne = closed ? n : n - 1;
    const float delta = prm[rod].x;
    const int k = max(1, (int)prm[rod].y);
    for (int i = threadIdx.x; i < n; i += kLT) xs[i] = X[R.v0 + i];
    __syncthreads();
    double s = 0.0;
    for (int a = threadIdx.x; a < ne; a += kLT) {
        const int a1 = (a + 1 == n) ? 0 : a + 1;
        const V3<float> pa = f3(xs[a]), pb = f3(xs[a1]);
        V3<float> g0 = zf3(), g1 = zf3();
        for (int b = 0; b < ne; ++b) {
            int sep = abs(a - b);
            if (closed) sep = min(sep, ne - sep);
            if (sep <= k) continue;
            const int b1 = (b + 1 == n) ? 0 : b + 1;
            // every pair is solved with its lower edge first, as both of its threads must see
            // the same closest points (the near-parallel rule is not symmetric)
            const bool first = a < b;
            const V3<float> qa = f3(xs[b]), qb = f3(xs[b1]);
            const V3<float> p1 = first ? pa : qa, q1 = first ? pb : qb, p2 = first ? qa : pa, q2 = first ? qb : pb;
            float ps, pu;
            closest_params(p1, q1, p2, q2, ps, pu);
            const V3<float> dv = (p1 + ps * (q1 - p1)) - (p2 + pu * (q2 - p2));
            const float d = sqrtf(dot(dv, dv));
            if (d >= delta) continue;
            if (first) s += (double)((delta - d) * (delta - d));
            if (d > 0.f) {
                const V3<float> gd = (-2.f * (delta - d) / d) * dv;   // d(pen)/d(first closest point)
                const float t = first ? ps : pu, sg = first ? 1.f : -1.f;
                g0 += (sg * (1.f - t)) * gd;
                g1 += (sg * t) * gd;
            }
        }
        ge0[a] = f4(g0, 0.f);
        ge1[a] = f4(g1, 0.f);
    }
    __syncthreads();
    s = block_sum(s, sh);
    if (q && threadIdx.x == 0) q[rod] = (float)s;
    if (!gx) return;
    const float c = gscale(g, rod);
    for (int i = threadIdx.x; i < n; i += kLT) {
        V3<float> d = zf3();
        if (closed || i < ne) d += f3(ge0[i]);
        if (closed || i > 0) d += f3(ge1[i == 0 ? ne - 1 : i - 1]);
        gx[R.v0 + i] = f4(c * d, 0.f);
    }
}

}  // namespace
}  // namespace dlo

using namespace dlo;

extern "C" dlo_status dlo_loss(dlo_ctx* c, int kind, const float* x, const float* aux, int m, const float* g,
                               float* q, float* dL_dx) {
    if (!c) return DLO_ERR_INVALID_ARG;
    const float4* X = reinterpret_cast<const float4*>(x);
    float4* GX = reinterpret_cast<float4*>(dL_dx);
    if (!x || ((uintptr_t)x & 15u) || (dL_dx && ((uintptr_t)dL_dx & 15u)) || (aux && ((uintptr_t)aux & 15u)))
        return set_err(c, DLO_ERR_INVALID_ARG, "x, aux and dL_dx must be non-null device float4 arrays (16-byte aligned)");
    for (const auto& R : c->rods_h) {
        if (R.nv > kMaxV) return set_err(c, DLO_ERR_INVALID_ARG, "rod too long for the loss kernels");
        // the losses over a rod's edges take single DLOs: nothing joins the strands of a record
        if ((R.flags & ROD_STRANDS) &&
            (kind == DLO_LOSS_WINDING || kind == DLO_LOSS_CROSSING || kind == DLO_LOSS_REPULSION))
            return set_err(c, DLO_ERR_INVALID_ARG, "edge-based losses need rods without strands");
    }
    switch (kind) {
        case DLO_LOSS_TARGET:
            if (!aux) return set_err(c, DLO_ERR_INVALID_ARG, "the target loss needs target positions");
            loss_target<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, reinterpret_cast<const float4*>(aux), g, q, GX);
            break;
        case DLO_LOSS_CHAMFER:
            if (!aux || m < 1 || m > kMaxPoints)
                return set_err(c, DLO_ERR_INVALID_ARG, "the Chamfer loss needs 1..1024 points per rod");
            loss_chamfer<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, reinterpret_cast<const float4*>(aux), m, g, q, GX);
            break;
        case DLO_LOSS_WINDING:
            if (!aux) return set_err(c, DLO_ERR_INVALID_ARG, "the winding number needs a post per rod");
            loss_winding<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, reinterpret_cast<const float4*>(aux), g, q, GX);
            break;
        case DLO_LOSS_CROSSING:
            loss_crossing<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, g, q, GX);
            break;
        case DLO_LOSS_MINDIST:
            if (!aux) return set_err(c, DLO_ERR_INVALID_ARG, "the minimum distance needs an object centre per rod");
            loss_mindist<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, reinterpret_cast<const float4*>(aux), g, q, GX);
            break;
        case DLO_LOSS_REPULSION:
            if (!aux) return set_err(c, DLO_ERR_INVALID_ARG, "the repulsion penalty needs (delta, k) per rod");
            loss_repulsion<<<c->B, kLT, 0, c->stream>>>(c->d_rods, X, reinterpret_cast<const float4*>(aux), g, q,
                                                        GX);
            break;
        default:
            return set_err(c, DLO_ERR_INVALID_ARG, "unknown loss kind");
    }
    c->launches++;
    return cuda_err(c, cudaGetLastError(), "loss launch");
}
