// dlo_api.cu -- the C ABI (include/dlo.h): context, host-side rod setup, launches, queries.
//
// Host setup follows DLO-Lab App. A.1 / App. B.1 in FP64: rest lengths from the rest shape,
// lumped Voronoi masses, solid-cylinder axial inertias, per-rod substep counts (App. B.1's 5
// substeps per frame kept as the minimum, raised to ceil(dt * omega_max) where explicit
// stability needs it), grasped (kinematic) vertices of each gripper (Sec. 3.2) and rest
// curvatures (straight for open rods, a planar circle for loops).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dlo.h"
#include "dlo_kernels.h"
#include "dlo_runtime.h"

using namespace dlo;

// ------------------------------------------------------------------ helpers
static const char* kStatusNames[] = {"ok", "invalid argument", "CUDA error", "out of memory",
                                     "non-finite state", "capacity exceeded", "timeout", "call out of order",
                                     "index out of bounds (debug build)"};

dlo_status set_err(dlo_ctx* c, dlo_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

dlo_status cuda_err(dlo_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return DLO_OK;
    return set_err(c, DLO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(dlo_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (c->alloc.alloc) {
        p = c->alloc.alloc(bytes, c->alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocs.push_back(p);
        c->bytes += bytes;
    }
    return p;
}

void dev_free(dlo_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    if (c->alloc.free)
        c->alloc.free(p, c->alloc.user);
    else
        cudaFree(p);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }


// Per-rod substep count: n = max(n_min, ceil(dt * omega_max)), omega_max the largest of the
// stretching 2 sqrt(K/rho)/l, bending 2 r sqrt(E/rho)/l^2 and twisting 2 sqrt(G/rho)/l
// frequencies of the shortest rest edge l: a factor 2 under the symplectic-Euler limit.
static int substeps_for(double dt, int nmin, double rho, double r, double K, double E, double G, bool inext,
                        double l) {
    double wb = 2.0 * r * std::sqrt(E / rho) / (l * l);
    double ws = inext ? 0.0 : 2.0 * std::sqrt(K / rho) / l;
    double wt = 2.0 * std::sqrt(G / rho) / l;
    double w = std::max(wb, std::max(ws, wt));
    return std::max(nmin, (int)std::ceil(dt * w));
}

// The material-dependent constants of a rod (App. A.1: k_s = K A, B = E A r^2 / 4,
// beta = G A r^2 / 2; yield curvature, creep rate, damping) and its substep.
static void set_moduli(RodInfo& R, const dlo_material& m, int ns, double dt) {
    const double r = m.radius, A = M_PI * r * r;
    R.nsub = ns;
    R.h = (float)(dt / ns);
    R.kA = m.inextensible ? 0.f : (float)(m.K_stretch * A);
    R.Bm = (float)(m.E_bend * A * r * r / 4.0);
    R.beta = (float)(m.G_twist * A * r * r / 2.0);
    R.sy = m.yield_curv;
    R.rc = m.creep_rate;
    R.cd = m.damping;
}

static bool material_ok(const dlo_material& m) {
    return m.density > 0.f && m.radius > 0.f && m.K_stretch >= 0.f && m.E_bend >= 0.f && m.G_twist >= 0.f &&
           m.strain_limit >= 0.f && m.strain_limit < 1.f && m.yield_curv >= 0.f && m.creep_rate >= 0.f &&
           m.creep_rate <= 1.f && m.damping >= 0.f;
}

// ------------------------------------------------------------------ create / destroy
extern "C" dlo_status dlo_create(dlo_ctx** out, int batch, const int* n_verts, const dlo_material* mat,
                                 const float* x_rest, const dlo_scene* scene, const dlo_options* opt,
                                 const dlo_allocator* alloc, void* cuda_stream) {
    if (!out) return DLO_ERR_INVALID_ARG;
    *out = nullptr;
    if (batch <= 0 || batch > (1 << 24) || !n_verts || !mat || !x_rest || !opt) return DLO_ERR_INVALID_ARG;
    if (!(opt->dt > 0.f) || opt->n_iter_pbd < 0 || opt->n_iter_pbd > 1000 || opt->substeps_min < 1 ||
        opt->checkpoint_every < 0 || opt->warps_per_cta < 0 || opt->warps_per_cta > 8 || !(opt->eps_soft > 0.f) ||
        opt->contact_margin < 0.f || opt->mu_self < 0.f || opt->mu_rigid < 0.f || opt->restitution < 0.f ||
        opt->broad_phase < 0 || opt->broad_phase > 1)
        return DLO_ERR_INVALID_ARG;
    // self-contact friction acts on the contact set of the first projection iteration
    if (opt->self_contact && opt->n_iter_pbd < 1) return DLO_ERR_INVALID_ARG;
    if (scene && (scene->n_planes < 0 || scene->n_planes > kMaxPlanes || scene->n_boxes < 0 ||
                  scene->n_boxes > kMaxBoxes || (scene->n_planes && !scene->planes) ||
                  (scene->n_boxes && !scene->boxes)))
        return DLO_ERR_INVALID_ARG;
    dlo_ctx* c = new (std::nothrow) dlo_ctx();
    if (!c) return DLO_ERR_OOM;
    c->B = batch;
    c->stream = (cudaStream_t)cuda_stream;
    if (alloc) c->alloc = *alloc;
    c->opt = *opt;
    // ---- host-side rod setup (FP64)
    long long V = 0, Et = 0;
    std::vector<int> vo(batch + 1), eo(batch + 1);
    for (int b = 0; b < batch; ++b) {
        const int nv = n_verts[b];
        const bool closed = mat[b].closed != 0;
        if (nv < 2 || nv > kMaxVerts || (closed && nv < 3)) {
            delete c;
            return DLO_ERR_INVALID_ARG;
        }
        const dlo_material& m = mat[b];
        if (!material_ok(m)) {
            delete c;
            return DLO_ERR_INVALID_ARG;
        }
        vo[b] = (int)V;
        eo[b] = (int)Et;
        V += nv;
        Et += nv - 1 + (closed ? 1 : 0);
    }
    vo[batch] = (int)V;
    eo[batch] = (int)Et;
    c->V = V;
    c->Et = Et;
    int ngrip_any = 0;
    if (scene && scene->n_grippers) {
        for (int b = 0; b < batch; ++b) {
            if (scene->n_grippers[b] < 0 || scene->n_grippers[b] > 2) {
                delete c;
                return DLO_ERR_INVALID_ARG;
            }
            ngrip_any |= scene->n_grippers[b];
        }
        if (ngrip_any && (!scene->grip_pose || !(scene->grip_radius > 0.f) || !(scene->grip_half_len >= 0.f))) {
            delete c;
            return DLO_ERR_INVALID_ARG;
        }
    }
    std::vector<RodInfo> rods(batch);
    std::vector<float4> kin(V), rest(V, make_float4(0.f, 0.f, 0.f, 0.f)), xr4(V);
    std::vector<float2> massv(V), es(Et);
    std::vector<float> gp0((size_t)batch * 24, 0.f);
    c->nsub.resize(batch);
    c->lmin_h.resize(batch);
    c->mat_h.assign(mat, mat + batch);
    for (int b = 0; b < batch; ++b) {
        const dlo_material& m = mat[b];
        const int nv = n_verts[b], v0 = vo[b], e0 = eo[b];
        const bool closed = m.closed != 0;
        const int ne = nv - 1 + (closed ? 1 : 0);
        const double r = m.radius, rho = m.density, A = M_PI * r * r;
        // strands: edge j is a break edge when vertex j + 1 begins another DLO; every strand
        // has at least two vertices, and only open rods have strands
        std::vector<char> brk(ne, 0);
        bool has_strands = false;
        if (scene && scene->strand_start) {
            int last = 0;
            for (int i = 1; i < nv; ++i)
                if (scene->strand_start[v0 + i]) {
                    if (closed || i - last < 2) {
                        delete c;
                        return DLO_ERR_INVALID_ARG;
                    }
                    brk[i - 1] = 1;
                    last = i;
                    has_strands = true;
                }
            if (has_strands && nv - last < 2) {
                delete c;
                return DLO_ERR_INVALID_ARG;
            }
        }
        std::vector<double> eb(ne);
        double lmin = 1e300;
        for (int j = 0; j < ne; ++j) {
            if (brk[j]) {   // rest length 0, no axial inertia (its twist angle only decays)
                eb[j] = 0.0;
                es[e0 + j] = make_float2(0.f, 0.f);
                continue;
            }
            int j1 = (j + 1 == nv) ? 0 : j + 1;
            double dx = (double)x_rest[3 * (v0 + j1)] - x_rest[3 * (v0 + j)];
            double dy = (double)x_rest[3 * (v0 + j1) + 1] - x_rest[3 * (v0 + j) + 1];
            double dz = (double)x_rest[3 * (v0 + j1) + 2] - x_rest[3 * (v0 + j) + 2];
            eb[j] = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (!(eb[j] > 0.0)) {
                delete c;
                return DLO_ERR_INVALID_ARG;
            }
            lmin = std::min(lmin, eb[j]);
            // with no twist stiffness (G = 0) the twist angle has no dynamics: an edge without a
            // restoring torque and with an axial inertia this small (1/2 rho A r^2 |e|) would
            // spin up under the bending-twist coupling alone (reading O41 of the paper's
            // "Twisting -" rows)
            const double invI = m.G_twist > 0.f ? 1.0 / (0.5 * rho * A * eb[j] * r * r) : 0.0;
            es[e0 + j] = make_float2((float)eb[j], (float)invI);
        }
        const bool inext = m.inextensible != 0;
        const int ns = substeps_for(opt->dt, opt->substeps_min, rho, r, m.K_stretch, m.E_bend, m.G_twist, inext, lmin);
        c->nsub[b] = ns;
        c->lmin_h[b] = lmin;
        // kinematic kinds: pinned, grasped (every vertex touching the capsule, at least the nearest)
        std::vector<int> kind(nv, 0);
        std::vector<double> off(3 * nv, 0.0);
        if (scene && scene->pinned)
            for (int i = 0; i < nv; ++i) kind[i] = scene->pinned[v0 + i] ? 1 : 0;
        const int ng = (scene && scene->n_grippers) ? scene->n_grippers[b] : 0;
        for (int g = 0; g < ng; ++g) {
            const float* P = scene->grip_pose + (size_t)b * 24 + 12 * g;
            double p[3] = {P[0], P[1], P[2]}, Rm[9];
            for (int k = 0; k < 9; ++k) Rm[k] = P[3 + k];
            double ax[3] = {Rm[2], Rm[5], Rm[8]}, hl = scene->grip_half_len;
            double a0[3], a1[3], ab[3];
            for (int k = 0; k < 3; ++k) {
                a0[k] = p[k] - ax[k] * hl;
                a1[k] = p[k] + ax[k] * hl;
                ab[k] = a1[k] - a0[k];
            }
            double abab = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
            std::vector<double> sd(nv);
            int best = 0;
            for (int i = 0; i < nv; ++i) {
                const float* x = x_rest + 3 * (v0 + i);
                double s = abab > 0 ? ((x[0] - a0[0]) * ab[0] + (x[1] - a0[1]) * ab[1] + (x[2] - a0[2]) * ab[2]) / abab : 0.0;
                s = std::min(std::max(s, 0.0), 1.0);
                double d0 = x[0] - (a0[0] + s * ab[0]), d1 = x[1] - (a0[1] + s * ab[1]), d2 = x[2] - (a0[2] + s * ab[2]);
                sd[i] = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) - scene->grip_radius;
                if (sd[i] < sd[best]) best = i;
            }
            for (int i = 0; i < nv; ++i) {
                bool grab = sd[i] < r || i == best;
                if (grab && kind[i] == 0) {
                    kind[i] = 2 + g;
                    const float* x = x_rest + 3 * (v0 + i);
                    double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
                    for (int k = 0; k < 3; ++k) off[3 * i + k] = d[0] * Rm[k] + d[1] * Rm[3 + k] + d[2] * Rm[6 + k];
                }
            }
            for (int k = 0; k < 12; ++k) gp0[(size_t)b * 24 + 12 * g + k] = P[k];
        }
        for (int g = ng; g < 2; ++g) {   // unused gripper slots: identity pose
            gp0[(size_t)b * 24 + 12 * g + 3] = gp0[(size_t)b * 24 + 12 * g + 7] = gp0[(size_t)b * 24 + 12 * g + 11] = 1.f;
        }
        for (int i = 0; i < nv; ++i) {
            double lv;
            if (closed)
                lv = 0.5 * (eb[i] + eb[(i + ne - 1) % ne]);
            else
                lv = 0.5 * ((i > 0 ? eb[i - 1] : 0.0) + (i < ne ? eb[i] : 0.0));
            double mass = rho * A * lv;
            massv[v0 + i] = make_float2((float)mass, kind[i] == 0 ? (float)(1.0 / mass) : 0.f);
            kin[v0 + i] = make_float4((float)off[3 * i], (float)off[3 * i + 1], (float)off[3 * i + 2], (float)kind[i]);
            xr4[v0 + i] = make_float4(x_rest[3 * (v0 + i)], x_rest[3 * (v0 + i) + 1], x_rest[3 * (v0 + i) + 2], 0.f);
        }
        if (closed) {
            float k1 = (float)(2.0 * std::tan(M_PI / ne));
            for (int i = 0; i < nv; ++i) rest[v0 + i] = make_float4(0.f, k1, 0.f, 0.f);
        }
        RodInfo& R = rods[b];
        R.v0 = v0;
        R.nv = nv;
        R.e0 = e0;
        R.ne = ne;
        R.nsub = ns;
        R.flags = (inext ? ROD_INEXT : 0) | (m.plastic ? ROD_PLASTIC : 0) |
                  (!inext && m.strain_limit > 0.f ? ROD_SLIMIT : 0) | (opt->self_contact ? ROD_SELF : 0) |
                  (closed ? ROD_CLOSED : 0) | (opt->broad_phase == 1 ? ROD_HASH : 0) |
                  (has_strands ? ROD_STRANDS : 0);
        R.ngrip = ng;
        R.excl = std::max(1, (int)std::ceil(2.0 * r / lmin));
        set_moduli(R, m, ns, opt->dt);
        R.radius = m.radius;
        R.slim = (!inext && m.strain_limit > 0.f) ? m.strain_limit : 0.f;
        R.contact_d = (float)(2.0 * r + opt->contact_margin * r);
        R.eps = (float)(opt->eps_soft * r);
        R.pair_cap = kPairsPerVertex * size_class(nv);
        R.pair_off = 0;
    }
    c->rods_h = rods;
    // scene
    SceneDev& sc = c->scene;
    memset(&sc, 0, sizeof(sc));
    sc.n_planes = scene ? scene->n_planes : 0;
    sc.n_boxes = scene ? scene->n_boxes : 0;
    for (int k = 0; k < sc.n_planes; ++k)
        sc.planes[k] = make_float4(scene->planes[4 * k], scene->planes[4 * k + 1], scene->planes[4 * k + 2],
                                   scene->planes[4 * k + 3]);
    for (int k = 0; k < sc.n_boxes; ++k) {
        const float* bx = scene->boxes + 6 * k;
        sc.box_c[k] = make_float4(bx[0], bx[1], bx[2], 0.f);
        sc.box_h[k] = make_float4(bx[3], bx[4], bx[5], 0.f);
    }
    sc.n_iter = opt->n_iter_pbd;
    sc.self_contact = opt->self_contact;
    sc.grip_r = scene ? scene->grip_radius : 0.f;
    sc.grip_hl = scene ? scene->grip_half_len : 0.f;
    sc.gravity = opt->gravity;
    sc.dt = opt->dt;
    sc.mu_self = opt->mu_self;
    sc.mu_rigid = opt->mu_rigid;
    sc.restitution = opt->restitution;
    // ---- device
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) {
        dlo_status st = cuda_err(c, ce, "device query");
        delete c;
        return st;
    }
    dlo_status st = runtime_allocate(c, rods, kin, massv, es, rest, gp0, xr4);
    if (st != DLO_OK) {
        dlo_destroy(c);
        return st;
    }
    *out = c;
    return DLO_OK;
}

extern "C" void dlo_destroy(dlo_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    runtime_release(c);
    std::vector<void*> all = c->allocs;
    for (void* p : all) dev_free(c, p);
    delete c;
}

extern "C" int dlo_build_flags(void) {
#ifdef DLO_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

extern "C" const char* dlo_status_string(dlo_status s) {
    int i = (int)s;
    if (i < 0 || i > 8) return "unknown status";
    return kStatusNames[i];
}

extern "C" const char* dlo_last_error(const dlo_ctx* c) { return c ? c->err.c_str() : "null context"; }

// ------------------------------------------------------------------ state
extern "C" dlo_status dlo_set_state(dlo_ctx* c, const float* x, const float* v, const float* theta) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!x || !aligned16(x) || (v && !aligned16(v))) return set_err(c, DLO_ERR_INVALID_ARG, "x/v must be 16-byte aligned");
    InitParams P{};
    P.rods = c->d_rods;
    P.B = c->B;
    P.xin = reinterpret_cast<const float4*>(x);
    P.vin = reinterpret_cast<const float4*>(v);
    P.thin = theta;
    P.mass = c->d_mass;
    P.ES = c->d_es;
    P.rest = c->d_rest;
    P.S = c->S;
    P.GP0 = c->d_gp0;
    P.rest_mode = 0;
    dlo_status st = cuda_err(c, launch_init(P, c->stream), "init kernel");
    c->launches++;
    if (st != DLO_OK) return st;
    st = cuda_err(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned) * c->B, c->stream), "status reset");
    c->from_set_state = true;
    c->rec_active = false;
    return st;
}

// ------------------------------------------------------------------ material
extern "C" dlo_status dlo_set_material(dlo_ctx* c, const dlo_material* mat) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (!mat) return set_err(c, DLO_ERR_INVALID_ARG, "mat is NULL");
    std::vector<RodInfo> rods = c->rods_h;
    std::vector<int> nsub = c->nsub;
    for (int b = 0; b < c->B; ++b) {
        const dlo_material& m = mat[b], &m0 = c->mat_h[b];
        if (!material_ok(m))
            return set_err(c, DLO_ERR_INVALID_ARG, "rod " + std::to_string(b) + ": material value out of range");
        if (m.density != m0.density || m.radius != m0.radius || m.inextensible != m0.inextensible ||
            m.strain_limit != m0.strain_limit || m.plastic != m0.plastic || m.closed != m0.closed ||
            (m.G_twist > 0.f) != (m0.G_twist > 0.f))
            return set_err(c, DLO_ERR_INVALID_ARG,
                           "rod " + std::to_string(b) +
                               ": density, radius, inextensibility, strain limit, plasticity, topology and whether "
                               "the twist modulus is zero are fixed at dlo_create");
        nsub[b] = substeps_for(c->opt.dt, c->opt.substeps_min, m.density, m.radius, m.K_stretch, m.E_bend,
                               m.G_twist, m.inextensible != 0, c->lmin_h[b]);
        set_moduli(rods[b], m, nsub[b], c->opt.dt);
    }
    cudaError_t e = cudaMemcpyAsync(c->d_rods, rods.data(), sizeof(RodInfo) * c->B, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // the host vector is released on return
    if (e != cudaSuccess) return cuda_err(c, e, "material upload");
    c->rods_h = rods;
    c->nsub = nsub;
    c->mat_h.assign(mat, mat + c->B);
    c->rec_active = false;   // a recorded rollout ran with the previous material
    return DLO_OK;
}

dlo_status check_status(dlo_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "stream");
    std::vector<unsigned> s(c->B);
    e = cudaMemcpy(s.data(), c->d_status, sizeof(unsigned) * c->B, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(c, e, "status copy");
    for (int b = 0; b < c->B; ++b) {
        if (s[b] & 1u) return set_err(c, DLO_ERR_NONFINITE, "rod " + std::to_string(b) + " has a non-finite state");
        if (s[b] & 2u)
            return set_err(c, DLO_ERR_CAPACITY, "rod " + std::to_string(b) + " overflowed its self-contact pair list");
        if (s[b] & 8u)
            return set_err(c, DLO_ERR_BOUNDS, "rod " + std::to_string(b) + ": an index failed a bounds check (debug build)");
    }
    return DLO_OK;
}

extern "C" dlo_status dlo_get_state(dlo_ctx* c, float* x, float* v, float* theta) {
    if (!c) return DLO_ERR_INVALID_ARG;
    if (x && cudaMemcpyAsync(x, c->S.X, 16 * c->V, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return cuda_err(c, cudaGetLastError(), "get x");
    if (v && cudaMemcpyAsync(v, c->S.Vl, 16 * c->V, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return cuda_err(c, cudaGetLastError(), "get v");
    if (theta && cudaMemcpy2DAsync(theta, 4, reinterpret_cast<char*>(c->S.ED) + 12, 16, 4, c->Et,
                                   cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return cuda_err(c, cudaGetLastError(), "get theta");
    return check_status(c);
}

extern "C" dlo_status dlo_get_internal(dlo_ctx* c, float* ref, float* tan, float* hinge, float* grip) {
    if (!c) return DLO_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (ref) e = cudaMemcpyAsync(ref, c->S.ED, 16 * c->Et, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && tan) e = cudaMemcpyAsync(tan, c->S.ET, 16 * c->Et, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && hinge) e = cudaMemcpyAsync(hinge, c->S.HG, 16 * c->V, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && grip)
        e = cudaMemcpyAsync(grip, c->S.GP, sizeof(float) * 24 * c->B, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "get internal");
    return check_status(c);
}

// ------------------------------------------------------------------ query
extern "C" dlo_status dlo_query(dlo_ctx* c, int what, void* out) {
    if (!c || !out) return DLO_ERR_INVALID_ARG;
    switch (what) {
        case DLO_Q_SUBSTEPS:
            memcpy(out, c->nsub.data(), sizeof(int) * c->B);
            return DLO_OK;
        case DLO_Q_STATUS: {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) e = cudaMemcpy(out, c->d_status, sizeof(unsigned) * c->B, cudaMemcpyDeviceToHost);
            return cuda_err(c, e, "query status");
        }
        case DLO_Q_BYTES:
            *reinterpret_cast<size_t*>(out) = c->bytes;
            return DLO_OK;
        case DLO_Q_CONFIG: {
            int* o = reinterpret_cast<int*>(out);
            o[0] = c->buckets.empty() ? 0 : c->buckets[0].warps;
            o[1] = c->ck_every;
            o[2] = c->buckets.empty() ? 0 : c->buckets[0].grid;
            o[3] = c->buckets.empty() ? 0 : (int)(warp_smem_bytes(c->buckets[0].nv_max, c->buckets[0].contact) *
                                                 c->buckets[0].warps);
            return DLO_OK;
        }
        case DLO_Q_RESIDUAL: {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) e = cudaMemcpy(out, c->d_residual, sizeof(double) * c->B, cudaMemcpyDeviceToHost);
            return cuda_err(c, e, "query residual");
        }
        case DLO_Q_PAIRS: {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) e = cudaMemcpy(out, c->d_npairs, sizeof(int) * c->B, cudaMemcpyDeviceToHost);
            return cuda_err(c, e, "query pairs");
        }
        case DLO_Q_PAIR_LIST: {
            const size_t stride = 1 + (size_t)kPairListStride;
            uint32_t* o = reinterpret_cast<uint32_t*>(out);
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess && c->d_pair_list)
                e = cudaMemcpy(o, c->d_pair_list, sizeof(uint32_t) * stride * c->B, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_err(c, e, "query pair list");
            for (int b = 0; b < c->B; ++b) {
                uint32_t* r = o + stride * b;
                if (!c->d_pair_list) r[0] = 0;
                const uint32_t n = std::min<uint32_t>(r[0], (uint32_t)kPairListStride);
                for (size_t k = 1 + n; k < stride; ++k) r[k] = 0xffffffffu;
            }
            return DLO_OK;
        }
        case DLO_Q_LAUNCHES:
            *reinterpret_cast<long long*>(out) = c->launches;
            return DLO_OK;
        case DLO_Q_MASS: {
            std::vector<float2> m(c->V);
            std::vector<float4> k(c->V);
            cudaError_t e = cudaMemcpy(m.data(), c->d_mass, 8 * c->V, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(k.data(), c->d_kin, 16 * c->V, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_err(c, e, "query mass");
            float* o = reinterpret_cast<float*>(out);
            for (long long i = 0; i < c->V; ++i) {
                o[4 * i] = m[i].x;
                o[4 * i + 1] = m[i].y;
                o[4 * i + 2] = k[i].w;
                o[4 * i + 3] = 0.f;
            }
            return DLO_OK;
        }
    }
    return set_err(c, DLO_ERR_INVALID_ARG, "unknown query");
}
