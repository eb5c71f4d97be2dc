// dlo_init.cu -- initial adapted reference frames of every rod, in FP64 (App. A.1).
//
// Edge 0 takes the projection of a fixed axis (z, or x when the first edge lies within about
// 25 degrees of z); later edges get their frame by space-parallel transport.  For closed
// loops the holonomy psi_H (mismatch after transporting the last frame across the closing
// hinge, measured about t^0) is spread as phi^j = -psi_H j / N_e and each (d1, d2) rotated by
// phi^j ("Loop Topology").  The reference twist of each hinge is the signed angle from the
// transported d1 of the previous edge to d1 of the next; in rest mode it becomes the rest
// twist, so the rest state stores no twist energy.  A record of several strands (ROD_STRANDS)
// starts each strand like edge 0; a break edge between two strands gets tangent z and d1 = x,
// and the hinges at its two ends a reference (and rest) twist of 0.
#include "dlo_kernels.h"
#include "dlo_physics.cuh"

namespace dlo {

__device__ __forceinline__ V3<double> unit_d(V3<double> a) { return a / sqrt(dot(a, a)); }
__device__ __forceinline__ V3<double> adapt_d(V3<double> d, V3<double> t) { return unit_d(d - dot(d, t) * t); }
__device__ __forceinline__ V3<double> ld(float4 a) { return V3<double>{(double)a.x, (double)a.y, (double)a.z}; }

__global__ void init_kernel(InitParams P) {
    const int rod = blockIdx.x * blockDim.x + threadIdx.x;
    if (rod >= P.B) return;
    const RodInfo R = P.rods[rod];
    const int nv = R.nv, ne = R.ne, v0 = R.v0, e0 = R.e0;
    const bool closed = R.flags & ROD_CLOSED;
    auto X = [&](int i) { return ld(P.xin[v0 + i]); };
    auto T = [&](int j) { return unit_d(X(j + 1 == nv ? 0 : j + 1) - X(j)); };
    // the first frame of an open rod or strand: the projection of a fixed axis
    auto first_d1 = [](V3<double> t) {
        V3<double> ax = fabs(t.z) < 0.9 ? V3<double>{0.0, 0.0, 1.0} : V3<double>{1.0, 0.0, 0.0};
        return adapt_d(ax, t);
    };
    const bool strands = R.flags & ROD_STRANDS;
    auto brk = [&](int j) { return strands && !(P.ES[e0 + j].x > 0.f); };
    // edge 0
    V3<double> t0 = T(0);
    V3<double> d = first_d1(t0);
    double psi = 0.0;
    if (closed) {   // first pass: holonomy of the space-parallel transport around the loop
        V3<double> tp = t0, dd = d;
        for (int j = 1; j < ne; ++j) {
            V3<double> tj = T(j);
            dd = adapt_d(transport_d(tp, tj, dd), tj);
            tp = tj;
        }
        V3<double> u = adapt_d(transport_d(tp, t0, dd), t0);
        psi = atan2(dot(cross(d, u), t0), dot(d, u));
    }
    // second pass: frames (with the holonomy correction) and reference twists
    V3<double> tp = t0, dp = d, d1p = d, tfirst = t0, d1first = d;
    for (int j = 0; j < ne; ++j) {
        const bool bj = brk(j), start = j > 0 && brk(j - 1);
        V3<double> tj = bj ? V3<double>{0.0, 0.0, 1.0} : T(j);
        V3<double> dj = bj ? V3<double>{1.0, 0.0, 0.0}
                           : (j == 0 ? d : (start ? first_d1(tj) : adapt_d(transport_d(tp, tj, dp), tj)));
        dp = dj;
        V3<double> d1 = dj;
        if (closed) {
            double phi = -psi * (double)j / (double)ne;
            d1 = cos(phi) * dj + sin(phi) * cross(tj, dj);
        }
        if (j > 0) {   // hinge at vertex j between edges j-1 and j
            V3<double> u = transport_d(tp, tj, d1p);
            double ang = (bj || start) ? 0.0 : atan2(dot(cross(u, d1), tj), dot(u, d1));
            if (P.rest_mode) P.rest[v0 + j].z = (float)ang;
            else {
                float4 rs = P.rest[v0 + j];
                P.S.HG[v0 + j] = make_float4(rs.x, rs.y, rs.z, (float)ang);
            }
        }
        if (j == 0) d1first = d1;
        if (!P.rest_mode) {
            float th = P.thin ? P.thin[e0 + j] : 0.f;
            P.S.ED[e0 + j] = make_float4((float)d1.x, (float)d1.y, (float)d1.z, th);
            P.S.ET[e0 + j] = make_float4((float)tj.x, (float)tj.y, (float)tj.z, P.ES[e0 + j].x);
        }
        tp = tj;
        d1p = d1;
    }
    if (closed) {  // closing hinge at vertex 0 between edges ne-1 and 0
        V3<double> u = transport_d(tp, tfirst, d1p);
        double ang = atan2(dot(cross(u, d1first), tfirst), dot(u, d1first));
        if (P.rest_mode) P.rest[v0].z = (float)ang;
        else {
            float4 rs = P.rest[v0];
            P.S.HG[v0] = make_float4(rs.x, rs.y, rs.z, (float)ang);
        }
    }
    if (P.rest_mode) return;
    if (!closed) {
        P.S.HG[v0] = make_float4(0.f, 0.f, 0.f, 0.f);
        P.S.HG[v0 + nv - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = 0; i < nv; ++i) {
        float4 x = P.xin[v0 + i];
        P.S.X[v0 + i] = make_float4(x.x, x.y, x.z, P.mass[v0 + i].y);
        float4 v = P.vin ? P.vin[v0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (!closed && i == nv - 1) v.w = 0.f;
        P.S.Vl[v0 + i] = v;
    }
    for (int k = 0; k < 24; ++k) P.S.GP[24 * rod + k] = P.GP0[24 * rod + k];
}

cudaError_t launch_init(const InitParams& P, cudaStream_t st) {
    if (P.B <= 0) return cudaSuccess;
    init_kernel<<<(P.B + 127) / 128, 128, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace dlo
