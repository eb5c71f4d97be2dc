// dlo_silhouette.cu -- the system-identification loss: the projection error between the
// simulated rope's silhouette and a camera's binary mask (Sec. 5, "System Identification"),
// made differentiable.  Each edge is drawn as a capsule of the rod's projected radius, its
// soft occupancy of a pixel is sigma((rho_e - dist) / tau), and a pixel's occupancy is
// 1 - prod_e (1 - sigma_e), composited in log space.  The loss is the mean over cameras and
// pixels of (occupancy - mask)^2.
//
// One CTA per rod walks the cameras.  Pass 1 (a thread per pixel) composites the pixel and
// stores dL/d(occupancy) * prod_e (1 - sigma_e), the factor every edge's gradient at that
// pixel shares.  Pass 2 (a thread per edge) walks the pixels of the edge's bounding box
// and sums its endpoints' gradient, so nothing is accumulated with atomics and the result
// is deterministic.
#include <cmath>

#include "dlo_runtime.h"
#include "dlo_vec.cuh"

namespace dlo {
namespace {

constexpr int kSilT = 256;      // threads per rod
constexpr int kSilMaxV = 256;   // vertices per rod
// an edge is skipped at pixels farther than rho_e + kReach tau from it: sigma < 1.4e-11 there
constexpr float kReach = 25.f;
constexpr float kNear = 1e-3f;  // edges with an endpoint this close to the camera plane or behind it are not drawn

struct Cam {
    float fx, fy, cx, cy;
    float R[9];   // world to camera, row major
    float t[3];
};

__device__ __forceinline__ float softplus(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }
__device__ __forceinline__ float logistic(float z) {
    if (z >= 0.f) return 1.f / (1.f + expf(-z));
    const float e = expf(z);
    return e / (1.f + e);
}

// (u, v, rho, Z): pixel coordinates, projected radius (fx r / Z), depth
__device__ __forceinline__ float4 project(const Cam& c, V3<float> x, float r) {
    const float X = c.R[0] * x.x + c.R[1] * x.y + c.R[2] * x.z + c.t[0];
    const float Y = c.R[3] * x.x + c.R[4] * x.y + c.R[5] * x.z + c.t[1];
    const float Z = c.R[6] * x.x + c.R[7] * x.y + c.R[8] * x.z + c.t[2];
    const float iz = 1.f / Z;
    return make_float4(c.fx * X * iz + c.cx, c.fy * Y * iz + c.cy, c.fx * r * iz, Z);
}

// signed distance of pixel centre (pu, pv) to the capsule of edge (a, b): distance to the
// segment minus the edge radius; t is the closest point's parameter, (nu, nv) the unit
// direction from the closest point to the pixel (zero when they coincide)
__device__ __forceinline__ float capsule_sd(float pu, float pv, float4 a, float4 b, float rho, float& t, float& nu,
                                            float& nv) {
    const float du = b.x - a.x, dv = b.y - a.y;
    const float l2 = du * du + dv * dv;
    t = l2 > 0.f ? fminf(fmaxf(((pu - a.x) * du + (pv - a.y) * dv) / l2, 0.f), 1.f) : 0.f;
    const float eu = pu - (a.x + t * du), ev = pv - (a.y + t * dv);
    const float d = sqrtf(eu * eu + ev * ev);
    nu = d > 0.f ? eu / d : 0.f;
    nv = d > 0.f ? ev / d : 0.f;
    return d - rho;
}

__global__ void __launch_bounds__(kSilT) sil_kernel(const RodInfo* rods, const float4* X, const float* cams, int C,
                                                    int H, int W, const unsigned char* masks, float tau,
                                                    const float* g, float* q, float4* gx, float* render,
                                                    float* wbuf) {
    __shared__ float4 pu[kSilMaxV];     // projected vertices
    __shared__ float4 box[kSilMaxV];    // per edge: reach box (umin, umax, vmin, vmax); empty if not drawn
    __shared__ float4 ga[kSilMaxV], gb[kSilMaxV];   // per edge: world gradient at its two endpoints
    __shared__ float4 gv[kSilMaxV];     // per vertex: world gradient summed over cameras
    __shared__ double red[kSilT];
    __shared__ Cam cm;
    const int rod = blockIdx.x;
    const RodInfo R = rods[rod];
    const bool closed = R.flags & ROD_CLOSED;
    const int n = R.nv, ne = closed ? n : n - 1;
    const int HW = H * W;
    const float inv_tau = 1.f / tau;
    const float coef = 2.f * (g ? g[rod] : 1.f) / ((float)C * (float)HW);
    float* wr = wbuf + (size_t)rod * HW;
    for (int i = threadIdx.x; i < n; i += kSilT) gv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    double lsum = 0.0;
    for (int c = 0; c < C; ++c) {
        if (threadIdx.x < 16) reinterpret_cast<float*>(&cm)[threadIdx.x] = cams[16 * c + threadIdx.x];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kSilT) pu[i] = project(cm, f3(X[R.v0 + i]), R.radius);
        __syncthreads();
        for (int e = threadIdx.x; e < ne; e += kSilT) {
            const float4 a = pu[e], b = pu[e + 1 == n ? 0 : e + 1];
            if (a.w > kNear && b.w > kNear) {
                const float m = 0.5f * (a.z + b.z) + kReach * tau;
                box[e] = make_float4(fminf(a.x, b.x) - m, fmaxf(a.x, b.x) + m, fminf(a.y, b.y) - m, fmaxf(a.y, b.y) + m);
            } else {
                box[e] = make_float4(1.f, -1.f, 1.f, -1.f);
            }
        }
        __syncthreads();
        // ---- pass 1: composite every pixel
        const unsigned char* mk = masks + ((size_t)rod * C + c) * HW;
        for (int p = threadIdx.x; p < HW; p += kSilT) {
            const float px = (float)(p % W) + 0.5f, py = (float)(p / W) + 0.5f;
            float S = 0.f;   // log prod_e (1 - sigma_e)
            for (int e = 0; e < ne; ++e) {
                const float4 bx = box[e];
                if (px < bx.x || px > bx.y || py < bx.z || py > bx.w) continue;
                const float4 a = pu[e], b = pu[e + 1 == n ? 0 : e + 1];
                float t, nu, nv;
                const float sd = capsule_sd(px, py, a, b, 0.5f * (a.z + b.z), t, nu, nv);
                S -= softplus(-sd * inv_tau);
            }
            const float o = -expm1f(S);
            const float d = o - (mk[p] ? 1.f : 0.f);
            lsum += (double)d * d;
            wr[p] = coef * d * expf(S);
            if (render) render[((size_t)rod * C + c) * HW + p] = o;
        }
        __syncthreads();
        // ---- pass 2: each edge's endpoint gradient over its reach box
        for (int e = threadIdx.x; e < ne; e += kSilT) {
            const float4 bx = box[e];
            const float4 a = pu[e], b = pu[e + 1 == n ? 0 : e + 1];
            const float rho = 0.5f * (a.z + b.z);
            float gau = 0.f, gav = 0.f, gbu = 0.f, gbv = 0.f, gr = 0.f;   // d L / d(u_a, v_a, u_b, v_b, rho_e)
            if (bx.x <= bx.y) {
                const int i0 = max(0, (int)floorf(bx.x - 0.5f)), i1 = min(W - 1, (int)ceilf(bx.y - 0.5f));
                const int j0 = max(0, (int)floorf(bx.z - 0.5f)), j1 = min(H - 1, (int)ceilf(bx.w - 0.5f));
                for (int j = j0; j <= j1; ++j) {
                    const float py = (float)j + 0.5f;
                    for (int i = i0; i <= i1; ++i) {
                        const float px = (float)i + 0.5f;
                        if (px < bx.x || px > bx.y || py < bx.z || py > bx.w) continue;
                        float t, nu, nv;
                        const float sd = capsule_sd(px, py, a, b, rho, t, nu, nv);
                        // dL/d(sd) = w(p) sigma(z) dz/d(sd), z = -sd / tau
                        const float gs = -wr[j * W + i] * logistic(-sd * inv_tau) * inv_tau;
                        gau -= gs * (1.f - t) * nu;
                        gav -= gs * (1.f - t) * nv;
                        gbu -= gs * t * nu;
                        gbv -= gs * t * nv;
                        gr -= gs;
                    }
                }
            }
            // (u, v, rho) = (fx X / Z + cx, fy Y / Z + cy, fx r / Z); then world = R^T camera
            auto to_world = [&](float4 pv, float g_u, float g_v, float g_r) {
                const float iz = 1.f / pv.w;
                const float Xc = (pv.x - cm.cx) * pv.w / cm.fx, Yc = (pv.y - cm.cy) * pv.w / cm.fy;
                const float gX = g_u * cm.fx * iz, gY = g_v * cm.fy * iz;
                const float gZ = -(g_u * cm.fx * Xc + g_v * cm.fy * Yc + g_r * cm.fx * R.radius) * iz * iz;
                return make_float4(cm.R[0] * gX + cm.R[3] * gY + cm.R[6] * gZ, cm.R[1] * gX + cm.R[4] * gY + cm.R[7] * gZ,
                                   cm.R[2] * gX + cm.R[5] * gY + cm.R[8] * gZ, 0.f);
            };
            ga[e] = to_world(a, gau, gav, 0.5f * gr);
            gb[e] = to_world(b, gbu, gbv, 0.5f * gr);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kSilT) {
            float4 acc = gv[i];
            if (closed || i < ne) acc = make_float4(acc.x + ga[i].x, acc.y + ga[i].y, acc.z + ga[i].z, 0.f);
            if (closed || i > 0) {
                const float4 o = gb[i == 0 ? ne - 1 : i - 1];
                acc = make_float4(acc.x + o.x, acc.y + o.y, acc.z + o.z, 0.f);
            }
            gv[i] = acc;
        }
        __syncthreads();
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int s = kSilT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (q && threadIdx.x == 0) q[rod] = (float)(red[0] / ((double)C * HW));
    if (gx)
        for (int i = threadIdx.x; i < n; i += kSilT) gx[R.v0 + i] = gv[i];
}

}  // namespace
}  // namespace dlo

using namespace dlo;

extern "C" dlo_status dlo_loss_silhouette(dlo_ctx* c, const float* x, const float* cams, int n_cams, int height,
                                          int width, const unsigned char* masks, float tau, const float* g, float* q,
                                          float* dL_dx, float* render) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!x || ((uintptr_t)x & 15u) || (dL_dx && ((uintptr_t)dL_dx & 15u)) || !cams || !masks)
        return set_err(c, DLO_ERR_INVALID_ARG, "x, cams and masks are required; x and dL_dx must be 16-byte aligned");
    if (n_cams < 1 || height < 1 || width < 1 || (long long)height * width > (1LL << 24))
        return set_err(c, DLO_ERR_INVALID_ARG, "need 1 or more cameras and 1..2^24 pixels per image");
    if (!(tau > 0.f)) return set_err(c, DLO_ERR_INVALID_ARG, "tau must be positive");
    for (const auto& R : c->rods_h) {
        if (R.nv > kSilMaxV) return set_err(c, DLO_ERR_INVALID_ARG, "rod too long for the silhouette kernel");
        if (R.flags & ROD_STRANDS)   // its edges are drawn as capsules; nothing joins two strands
            return set_err(c, DLO_ERR_INVALID_ARG, "the silhouette loss needs rods without strands");
    }
    const size_t need = (size_t)c->B * height * width * sizeof(float);
    if (need > c->sil_bytes) {
        dev_free(c, c->sil_mem);
        c->sil_mem = dev_alloc(c, need);
        c->sil_bytes = c->sil_mem ? need : 0;
        if (!c->sil_mem) return set_err(c, DLO_ERR_OOM, "silhouette scratch allocation failed");
    }
    sil_kernel<<<c->B, kSilT, 0, c->stream>>>(c->d_rods, reinterpret_cast<const float4*>(x), cams, n_cams, height,
                                              width, masks, tau, g, q, reinterpret_cast<float4*>(dL_dx), render,
                                              reinterpret_cast<float*>(c->sil_mem));
    c->launches++;
    return cuda_err(c, cudaGetLastError(), "silhouette launch");
}
