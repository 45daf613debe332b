// Ground-state solver (Sec. 5, Algorithm 1 on one mesh) driving the device
// kernels: RGBB (Riemannian gradient, BB step, Zhang-Hager nonmonotone search)
// and ARNT (regularised Newton model m_k, modified CG, curvilinear Armijo
// search, ratio test and sigma update).  Every vector operation runs on the
// device.  The modified CG runs in chunks of cg_chunk iterations whose
// coefficients and stopping tests are computed on the device (k_cg_update), each
// chunk the replay of a CUDA graph (one per state array, slot parity and set of
// launched instances); the host reads the scalar block once per
// chunk, line-search trial or outer iteration and keeps the rest of the control
// flow.
//
// Readings where the paper defers to the cited ARNT paper or is silent:
//  * RGBB: first step gamma_0 = 1e-3; BB step |<s,v>|/<v,v> clamped to
//    [1e-10, 1e10]; rho = 1e-4, varrho = 0.85, delta = 0.2; at most 10
//    reductions, after which the last trial is taken; a trial whose energy is
//    within the rounding floor (below) of the current one passes the test.
//  * ARNT: eta1 = 0.01, eta2 = 0.9, gamma0 = 0.2, gamma1 = 1, gamma2 = 10,
//    sigma_k = sigma_hat_k ||grad||, sigma_hat_0 = 1 (Sec. 7.1); after negative
//    curvature sigma_{k+1} = max(sigma_{k+1}, sigma_est) (gamma_tilde = 0).
//  * modified CG: Steihaug-type CG from 0 on Hess m_k[xi] = -grad; stop at
//    ||r|| <= min(0.1, ||grad||) ||grad||; <p,Hp> <= 1e-12 ||p||^2 ends it: at
//    the first iteration with s = -grad, later with s = the iterate and d = p
//    when the curvature is negative; cap 100 inner iterations while
//    ||grad|| > 1e-3, else 300.
//  * curvilinear search: alpha0 = 1, delta = 0.2, rho = 1e-4, at most 10
//    reductions; m_k(z) is evaluated exactly with one Euclidean
//    Hessian-vector product.  Below the rounding floor 100 eps max(1, |E|)
//    of E (eps of the handle's precision) the Armijo test and the ratio are
//    taken as satisfied.
#include <math.h>
#include <string.h>

#include <vector>

#include <cuda_runtime.h>

#include "sbec_handle.h"

namespace {

using sbec::Lin;
using sbec::Ops;

// solver slots of the scalar block (pairs: a dot writes slot and slot + 1)
enum {
    SL_D0 = sbec::S_SOLVER,       // generic dot pair
    SL_KAP = SL_D0 + 2,           // <p, Hp>, <p, p>
    SL_ALPHA = SL_D0 + 4,         // CG alpha and its guard flag
    SL_RRA = SL_D0 + 6,           // <r, r> of even iterations (pair)
    SL_RRB = SL_D0 + 8,           // <r, r> of odd iterations (pair)
    SL_MA = SL_D0 + 10,           // <dz, g>, <dz, dz>
    SL_MB = SL_D0 + 12,           // <dz, H dz>
    SL_T = SL_D0 + 14,            // step length per instance
    SL_SIG = SL_D0 + 15,          // sigma per instance
    SL_ACT = SL_D0 + 16,          // instance still iterating
    SL_CG = SL_D0 + 17,           // instance still in the modified CG
    SL_BETA = SL_D0 + 18,         // CG beta
    SL_TAU = SL_D0 + 19,          // tau of Eq. (xi)
    SL_NEG = SL_D0 + 20,          // xi = -grad
    SL_HD = SL_D0 + 21,           // xi = s + tau d
    SL_ACC = SL_D0 + 22,          // trial accepted
    SL_J = SL_D0 + 23,            // CG iterations run
    SL_STOP = SL_D0 + 24,         // CG residual threshold min(0.1, ||grad||) ||grad||
    SL_MAXIN = SL_D0 + 25,        // CG iteration cap
    SL_SEST = SL_D0 + 26,         // |<p,Hp>| / <p,p> at a non-positive-curvature exit, else -1
    SL_CGNEG = SL_D0 + 27,        // CG ended at its first iteration on curvature: xi = -grad
    SL_CGHD = SL_D0 + 28,         // CG ended later on negative curvature: xi = s + tau d
};
static_assert(int(SL_CGHD) < int(sbec::S_COUNT), "solver slots exceed the scalar block");

// S_SKIP value of an instance whose modified CG has ended inside a chunk
constexpr double kSkipCg = 2.0;

// elementwise precision change of n reals
template <typename TS, typename TD>
__global__ void k_cast(const TS* __restrict__ src, TD* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = TD(src[i]);
}

template <typename TS, typename TD>
int cast_field(const void* src, void* dst, long long nreal, int num_sms, cudaStream_t s) {
    k_cast<TS, TD><<<4 * num_sms, 256, 0, s>>>(static_cast<const TS*>(src), static_cast<TD*>(dst), nreal);
    return cudaGetLastError() == cudaSuccess ? SBEC_OK : SBEC_ERR_CUDA;
}

// S_SKIP of every instance back to 0
__global__ void k_unskip(double* scal0, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) scal0[(size_t)b * sbec::S_COUNT + sbec::S_SKIP] = 0.0;
}

// after a solve: every instance on again, launches over the whole batch
int clear_skip(sbec_handle* h) {
    h->geom.nl = h->B;
    h->geom.imap = nullptr;
    k_unskip<<<(h->B + 127) / 128, 128, 0, h->stream>>>(h->work.scal, h->B);
    return cudaGetLastError() == cudaSuccess ? SBEC_OK : SBEC_ERR_CUDA;
}

// Chunks of the modified CG (Sec. 5, Eq. prob-lsub) on Hess m_k p = Hess f p +
// sigma p with sigma from each instance's SL_SIG: per iteration the projected
// Hessian-vector product, <p,Hp> and <p,p>, alpha = <r,r>/<p,Hp> (guarded),
// x += alpha p, r -= alpha Hp with <r,r> and the CG control, p = r + beta p.  With
// graphs, the chunk for a given state array and slot parity is captured once
// on a private stream and replayed on the handle's stream.
template <typename T>
struct CgChunks {
    sbec_handle* h;
    const sbec::Geom& g;
    const sbec::Work& w;
    int K;
    bool graphs;
    cudaStream_t cap = nullptr;
    struct Entry { const void* u; int par; int nl; const int* imap; cudaGraphExec_t exec; long long nodes; };
    std::vector<Entry> cache;

    CgChunks(sbec_handle* hh, int k, bool gr)
        : h(hh), g(hh->geom), w(hh->work), K(k), graphs(gr && !(hh->work.prof && hh->work.prof->enabled)) {}
    ~CgChunks() {
        for (auto& e : cache) cudaGraphExecDestroy(e.exec);
        if (cap) cudaStreamDestroy(cap);
    }

    int lin(cudaStream_t cs, void* out, const void* A, double cb, const void* Bv, int ib, int guard,
            const void* D1, int slot) {
        Lin L;
        L.out = out; L.A = A; L.B = Bv; L.ca = 1.0; L.cb = cb; L.ia = -1; L.ib = ib; L.ineg = -1;
        L.D1 = D1; L.D2 = nullptr; L.guard = guard;
        return Ops<T>::lincomb(g, w, L, slot, cs);
    }

    // one iteration: Hp = Hess p; <p,Hp>, <p,p> and alpha (k_cg_curv); x, r, <r,r> and
    // the CG control (k_cg_update, in its last block per instance); p = r + beta p
    int launch(cudaStream_t cs, const void* u, void* p, void* Hp, void* x, void* r, int par0) {
        for (int i = 0; i < K; ++i) {
            const int par = (par0 + i) & 1;
            const int rr_now = par ? SL_RRB : SL_RRA, rr_next = par ? SL_RRA : SL_RRB;
            const sbec::CgSlots sl{SL_KAP, SL_ALPHA, rr_now, rr_next, SL_BETA, SL_J, SL_STOP, SL_MAXIN,
                                   SL_CG, SL_SEST, SL_CGNEG, SL_CGHD, kSkipCg};
            int e = Ops<T>::hessvec(g, w, u, p, 1.0, 1, Hp, cs, SL_SIG, true);
            if (!e) e = Ops<T>::cg_curv(g, w, p, Hp, sl, cs);
            if (!e) e = Ops<T>::cg_update(g, w, x, r, p, Hp, sl, cs);
            if (!e) e = lin(cs, p, r, 1.0, p, SL_BETA, -1, nullptr, SL_D0);
            if (e) return e;
        }
        return SBEC_OK;
    }

    // one chunk on the handle's stream, starting at slot parity par0
    int run(const void* u, void* p, void* Hp, void* x, void* r, int par0) {
        if (!graphs) return launch(h->stream, u, p, Hp, x, r, par0);
        const Entry* hit = nullptr;
        for (const auto& e : cache)
            if (e.u == u && e.par == par0 && e.nl == g.nl && e.imap == g.imap) hit = &e;
        if (!hit) {
            if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return SBEC_ERR_CUDA;
            sbec::Prof* pr = w.prof;
            const long long before = pr ? pr->launches : 0;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                cudaGetLastError();
                return SBEC_ERR_CUDA;
            }
            const int e = launch(cap, u, p, Hp, x, r, par0);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
            Entry ent{u, par0, g.nl, g.imap, nullptr, pr ? pr->launches - before : 0};
            if (pr) pr->launches = before;       // captured, not launched
            if (e || ce != cudaSuccess || !graph) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return e ? e : SBEC_ERR_CUDA;
            }
            const cudaError_t ie = cudaGraphInstantiate(&ent.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) { cudaGetLastError(); return SBEC_ERR_CUDA; }
            cache.push_back(ent);
            hit = &cache.back();
        }
        if (cudaGraphLaunch(hit->exec, h->stream) != cudaSuccess) { cudaGetLastError(); return SBEC_ERR_CUDA; }
        if (w.prof) w.prof->launches += hit->nodes;
        return SBEC_OK;
    }
};

// FP32 context of the modified CG inside an FP64 solve (the refinement phase of
// sbec_solve_mixed): the Newton systems of ARNT are solved with Hessian-vector
// products of the mixed handle of the same problem at u rounded to float, while
// the gradient, the energy, the model value m_k, the search and the retraction
// stay in FP64.  The CG only has to produce a descent direction of the model;
// the stopping test on ||grad E|| is always taken in FP64.
struct InnerCg {
    sbec_handle* h = nullptr;      // SBEC_MIXED handle (same problem and stream)
    void* f[6] = {};               // float fields: u, rg, x, r, p, Hp
};

constexpr double kEps = 2.220446049250313e-16;

template <typename T>
struct Solver {
    sbec_handle* h;
    const sbec::Geom& g;
    const sbec::Work& w;
    cudaStream_t s;
    sbec_solve_opts o;
    sbec_stats* st;
    void* f[10];
    int status = SBEC_OK;
    CgChunks<T> cgc;
    const InnerCg* in;
    CgChunks<float>* cg32 = nullptr;

    Solver(sbec_handle* hh, const sbec_solve_opts& oo, void* ws, sbec_stats* stt, const InnerCg* inner = nullptr)
        : h(hh), g(hh->geom), w(hh->work), s(hh->stream), o(oo), st(stt), cgc(hh, oo.cg_chunk, oo.cuda_graphs != 0),
          in(inner && inner->h && sizeof(T) == 8 ? inner : nullptr) {
        char* b = static_cast<char*>(ws);
        for (int i = 0; i < 10; ++i) f[i] = b + (size_t)i * hh->field_bytes;
        if (in) cg32 = new CgChunks<float>(in->h, oo.cg_chunk, oo.cuda_graphs != 0);
    }
    ~Solver() { delete cg32; }
    Solver(const Solver&) = delete;
    Solver& operator=(const Solver&) = delete;

    // scalars of the block after the launched work; returns the device status
    int pull() { return sbec_read_scalars(h); }
    double sc(int i) const { return h->h_scal[i]; }
    // host-written slots back to the device (the block is in sync after pull)
    int push() {
        return cudaMemcpyAsync(w.scal, h->h_scal, sbec::S_COUNT * sizeof(double), cudaMemcpyHostToDevice, s) ==
                       cudaSuccess
                   ? SBEC_OK
                   : SBEC_ERR_CUDA;
    }

    int lin(void* out, double ca, const void* A, double cb, const void* B, int ib = -1, int guard = -1,
            const void* D1 = nullptr, const void* D2 = nullptr, int slot = SL_D0) {
        Lin L;
        L.out = out; L.A = A; L.B = B; L.ca = ca; L.cb = cb; L.ia = -1; L.ib = ib; L.ineg = -1;
        L.D1 = D1; L.D2 = D2; L.guard = guard;
        return Ops<T>::lincomb(g, w, L, slot, s);
    }

    int grad(const void* u, void* gE, void* rg) {
        ++st->n_grad;
        return Ops<T>::grad(g, w, u, gE, rg, true, s);
    }
    int energy(const void* x) {
        ++st->n_energy;
        return Ops<T>::energy(g, w, x, s);
    }
    int hess(const void* u, const void* z, double sigma, int riem, void* out) {
        ++st->n_hvp;
        return Ops<T>::hessvec(g, w, u, z, sigma, riem, out, s, -1, true);
    }
    int retract(const void* u, const void* xi, double t, void* out) {
        return Ops<T>::retract(g, w, u, xi, t, o.retraction, out, s);
    }

#define TRY(x) do { int e_ = (x); if (e_) return e_; } while (0)
// a device status other than a domain error aborts the solve
#define PULL(var) do { var = pull(); if (var != SBEC_OK && var != SBEC_ERR_DOMAIN) return var; } while (0)

    // RGBB from u (Sec. 5, Eq. NMN and the C_k, Q_k recursion)
    int rgbb(void*& u, void*& up, void*& z, void*& rg, void*& rgp, double tol, long long maxit, double& E,
             double& gn) {
        int ds;
        TRY(energy(u));
        PULL(ds);
        E = sc(SBEC_S_ENERGY);
        double Ck = E, Qk = 1.0;
        bool have_prev = false;
        for (long long k = 0; k <= maxit; ++k) {
            TRY(grad(u, nullptr, rg));
            if (have_prev) TRY(Ops<T>::bbdots(g, w, u, up, rg, rgp, SL_D0, s));
            PULL(ds);
            if (ds == SBEC_ERR_DOMAIN) return SBEC_ERR_DOMAIN;
            gn = sqrt(sc(SBEC_S_RGRAD_NORM2));
            if (gn <= tol || k == maxit) return SBEC_OK;
            double gam = 1e-3;
            if (have_prev) {
                const double sv = sc(SL_D0), vv = sc(SL_D0 + 1);
                gam = vv > 0.0 ? fabs(sv) / vv : 1e-3;
                gam = fmin(fmax(gam, 1e-10), 1e10);
            }
            const double slope = -gn * gn;
            const double noise = 100.0 * (sizeof(T) == 8 ? kEps : 1.1920928955078125e-07) * fmax(1.0, fabs(E));
            double t = gam, Ez = INFINITY;
            for (int bt = 0; bt <= 10; ++bt) {
                TRY(retract(u, rg, -t, z));
                TRY(energy(z));
                PULL(ds);
                Ez = (ds == SBEC_ERR_DOMAIN) ? INFINITY : sc(SBEC_S_ENERGY);
                if (Ez <= Ck + 1e-4 * t * slope || fabs(Ez - E) <= noise) break;
                t *= 0.2;
            }
            if (!isfinite(Ez)) return SBEC_ERR_DOMAIN;
            void* tmp = up; up = u; u = z; z = tmp;
            tmp = rgp; rgp = rg; rg = tmp;
            have_prev = true;
            E = Ez;
            const double Qn = 0.85 * Qk + 1.0;
            Ck = (0.85 * Qk * Ck + E) / Qn;
            Qk = Qn;
            ++st->rgbb_iters;
        }
        return SBEC_OK;
    }

    // Modified CG of one ARNT iteration on the FP32 handle of the inner context:
    // u and grad are rounded to float, the Lemma 4.2 coefficients of the FP64
    // gradient at u are copied into the float handle's scalar block, and the same
    // device-driven chunks as the FP64 path run there.  On return x (FP64) holds
    // the direction s + tau d of Eq. (xi), unless the CG ended at its first
    // iteration on curvature (s_is_neg_rg: the caller takes -grad).
    int cg_fp32(const void* u, const void* rg, void* x, double sigma, double stop, int max_inner, bool& s_is_neg_rg,
                double& sig_est) {
        if constexpr (sizeof(T) != 8) {
            return SBEC_ERR_ARG;
        } else {
            sbec_handle* h32 = in->h;
            const sbec::Geom& g32 = h32->geom;
            const sbec::Work& w32 = h32->work;
            void *u32 = in->f[0], *rg32 = in->f[1], *x32 = in->f[2], *r32 = in->f[3], *p32 = in->f[4],
                 *Hp32 = in->f[5];
            const long long nreal = 2LL * g.C * g.G;
            TRY((cast_field<double, float>(u, u32, nreal, w.num_sms, s)));
            TRY((cast_field<double, float>(rg, rg32, nreal, w.num_sms, s)));
            if (cudaMemcpyAsync(w32.scal + SBEC_S_ALPHA_G, w.scal + SBEC_S_ALPHA_G, 2 * sizeof(double),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return SBEC_ERR_CUDA;
            auto lin32 = [&](void* out, double ca, const void* A, double cb, const void* B, int ib, int guard,
                             const void* D1, int slot) {
                Lin L;
                L.out = out; L.A = A; L.B = B; L.ca = ca; L.cb = cb; L.ia = -1; L.ib = ib; L.ineg = -1;
                L.D1 = D1; L.D2 = nullptr; L.guard = guard;
                return Ops<float>::lincomb(g32, w32, L, slot, s);
            };
            TRY(lin32(x32, 0.0, rg32, 0.0, nullptr, -1, -1, nullptr, SL_D0));
            TRY(lin32(r32, -1.0, rg32, 0.0, nullptr, -1, -1, r32, SL_RRA));
            TRY(lin32(p32, 1.0, r32, 0.0, nullptr, -1, -1, nullptr, SL_D0));
            int ds = sbec_read_scalars(h32);
            if (ds) return ds;
            double* q = h32->h_scal;
            if (!(q[SL_RRA] > 0.0)) return SBEC_OK;          // grad rounds to 0 in float: x = 0
            q[SL_SIG] = sigma; q[SL_STOP] = stop; q[SL_MAXIN] = (double)max_inner;
            q[SL_J] = 0.0; q[SL_CG] = 1.0; q[SL_SEST] = -1.0; q[SL_CGNEG] = 0.0; q[SL_CGHD] = 0.0;
            q[sbec::S_SKIP] = 0.0;
            auto push32 = [&]() {
                return cudaMemcpyAsync(w32.scal, h32->h_scal, sbec::S_COUNT * sizeof(double), cudaMemcpyHostToDevice,
                                       s) == cudaSuccess
                           ? SBEC_OK
                           : SBEC_ERR_CUDA;
            };
            TRY(push32());
            long long done_its = 0;
            while (true) {
                TRY(cg32->run(u32, p32, Hp32, x32, r32, (int)(done_its & 1)));
                done_its += cg32->K;
                ds = sbec_read_scalars(h32);
                if (ds) return ds;
                if (q[SL_CG] == 0.0) break;
                if (done_its >= max_inner) return SBEC_ERR_CUDA;   // k_cg_update ends every CG by the cap
            }
            const long long its = (long long)q[SL_J];
            st->inner_iters += its;
            st->n_hvp += its;
            sig_est = q[SL_SEST];
            const bool neg = q[SL_CGNEG] != 0.0, hd = q[SL_CGHD] != 0.0;
            q[sbec::S_SKIP] = 0.0;
            TRY(push32());
            if (neg) {
                s_is_neg_rg = true;
                return SBEC_OK;
            }
            double tau = 0.0;
            if (hd) {
                TRY(Ops<float>::dot2(g32, w32, p32, rg32, p32, Hp32, SL_D0, s));
                ds = sbec_read_scalars(h32);
                if (ds) return ds;
                tau = q[SL_D0] / q[SL_D0 + 1];
                TRY(lin32(x32, 1.0, x32, tau, p32, -1, -1, nullptr, SL_D0));
            }
            return cast_field<float, double>(x32, x, nreal, w.num_sms, s);
        }
    }

    // ARNT from u (Algorithm 1, second loop)
    int arnt(void*& u, void*& z, void* gE, void* rg, void* x, void* r, void* p, void* Hp, double tol,
             long long maxit, double& E, double& gn) {
        int ds;
        TRY(energy(u));
        PULL(ds);
        E = sc(SBEC_S_ENERGY);
        double sig_hat = 1.0, sig_floor = 0.0;
        TRY(grad(u, gE, rg));
        PULL(ds);
        gn = sqrt(sc(SBEC_S_RGRAD_NORM2));
        for (long long k = 0; k <= maxit; ++k) {
            if (gn <= tol || k == maxit) break;
            const double sigma = fmax(sig_hat * gn, sig_floor);
            const int max_inner = gn > 1e-3 ? 100 : 300;
            // ---- modified CG on Hess m_k [xi] = -grad m_k (Eq. prob-lsub) ----
            const double stop = fmin(0.1, gn) * gn;
            bool s_is_neg_rg = false, have_d = false;
            double sig_est = -1.0;
            double rr = 0.0;
            if (in) {
                // the Newton system in FP32 on the mixed handle; x receives s + tau d
                TRY(cg_fp32(u, rg, x, sigma, stop, max_inner, s_is_neg_rg, sig_est));
            } else {
                TRY(lin(x, 0.0, rg, 0.0, nullptr));
                TRY(lin(r, -1.0, rg, 0.0, nullptr, -1, -1, r, nullptr, SL_RRA));
                TRY(lin(p, 1.0, r, 0.0, nullptr));
                PULL(ds);
                rr = sc(SL_RRA);
            }
            if (!in && rr > 0.0) {
                // device-driven chunks (k_cg_update); the host reads the block once per chunk
                double* hsc = h->h_scal;
                hsc[SL_SIG] = sigma; hsc[SL_STOP] = stop; hsc[SL_MAXIN] = (double)max_inner;
                hsc[SL_J] = 0.0; hsc[SL_CG] = 1.0; hsc[SL_SEST] = -1.0; hsc[SL_CGNEG] = 0.0; hsc[SL_CGHD] = 0.0;
                hsc[sbec::S_SKIP] = 0.0;
                TRY(push());
                long long done_its = 0;
                while (true) {
                    TRY(cgc.run(u, p, Hp, x, r, (int)(done_its & 1)));
                    done_its += cgc.K;
                    PULL(ds);
                    if (sc(SL_CG) == 0.0) break;
                            if (done_its >= max_inner) return SBEC_ERR_CUDA;   // k_cg_update ends every CG by the cap
                }
                const long long its = (long long)sc(SL_J);
                st->inner_iters += its;
                st->n_hvp += its;
                if (sc(SL_CGNEG) != 0.0) s_is_neg_rg = true;
                if (sc(SL_CGHD) != 0.0) have_d = true;
                sig_est = sc(SL_SEST);
                h->h_scal[sbec::S_SKIP] = 0.0;
                TRY(push());
            }
            // ---- direction xi = s + tau d (Eq. xi), kept in x ----
            if (s_is_neg_rg) {
                TRY(lin(x, -1.0, rg, 0.0, nullptr));
            } else if (have_d && !in) {
                TRY(Ops<T>::dot2(g, w, p, rg, p, Hp, SL_D0, s));
                PULL(ds);
                const double tau = sc(SL_D0) / sc(SL_D0 + 1);
                TRY(lin(x, 1.0, x, tau, p));
            }
            TRY(Ops<T>::dot2(g, w, rg, x, nullptr, nullptr, SL_D0, s));
            PULL(ds);
            double slope = sc(SL_D0);
            if (!(slope < 0.0) || !isfinite(slope)) {
                TRY(lin(x, -1.0, rg, 0.0, nullptr));
                slope = -gn * gn;
            }
            // ---- curvilinear search z = R_u(alpha0 delta^k xi) (Eq. tp1, tp2) ----
            // rounding floor of E: the energy's pointwise terms are summed from values
            // of the handle's precision T
            const double noise = 100.0 * (sizeof(T) == 8 ? kEps : 1.1920928955078125e-07) * fmax(1.0, fabs(E));
            double t = 1.0, mz = INFINITY;
            for (int bt = 0; bt <= 10; ++bt) {
                TRY(retract(u, x, t, z));
                TRY(lin(r, 1.0, z, -1.0, u, -1, -1, gE, r, SL_MA));     // dz = z - u
                TRY(hess(u, r, 0.0, 0, Hp));                          // H dz (Euclidean)
                TRY(Ops<T>::dot2(g, w, r, Hp, nullptr, nullptr, SL_MB, s));
                PULL(ds);
                mz = (ds == SBEC_ERR_DOMAIN) ? INFINITY
                                             : sc(SL_MA) + 0.5 * sc(SL_MB) + 0.5 * sigma * sc(SL_MA + 1);
                if (mz <= 1e-4 * t * slope || fabs(mz) <= noise) break;
                t *= 0.2;
            }
            TRY(energy(z));
            PULL(ds);
            const double Ez = (ds == SBEC_ERR_DOMAIN) ? INFINITY : sc(SBEC_S_ENERGY);
            double ratio;
            if (fabs(mz) <= noise && fabs(Ez - E) <= noise) ratio = 1.0;
            else ratio = (mz < 0.0 && isfinite(Ez)) ? (Ez - E) / mz : -1.0;
            if (ratio >= 0.01) {
                void* tmp = u; u = z; z = tmp;
                E = Ez;
                TRY(grad(u, gE, rg));
                PULL(ds);
                gn = sqrt(sc(SBEC_S_RGRAD_NORM2));
                sig_hat *= (ratio >= 0.9) ? 0.2 : 1.0;
            } else {
                sig_hat *= 10.0;
            }
            sig_floor = sig_est >= 0.0 ? sig_est : 0.0;
            ++st->outer_iters;
            if (sig_hat > 1e20) break;
        }
        return SBEC_OK;
    }

    int run(void* Xdev) {
        // fields: 0 u, 1 up, 2 z, 3 gE, 4 rg, 5 rgp, 6 x, 7 r, 8 p, 9 Hp
        void *u = f[0], *up = f[1], *z = f[2], *rg = f[4], *rgp = f[5];
        if (cudaMemcpyAsync(u, Xdev, h->field_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SBEC_ERR_CUDA;
        int ds;
        if (o.project_initial) {
            // P_M(X) (Lemma 5.1) whatever retraction the iteration uses
            TRY(Ops<T>::retract(g, w, u, u, 0.0, 1, u, s));
            PULL(ds);
            if (ds) return ds;
        }
        double E = 0.0, gn = INFINITY;
        if (o.method == SBEC_RGBB) {
            TRY(rgbb(u, up, z, rg, rgp, o.tol, o.maxit, E, gn));
        } else {
            TRY(rgbb(u, up, z, rg, rgp, fmax(o.tol, o.rgbb_tol), o.rgbb_maxit, E, gn));
            if (gn > o.tol) {
                // u and z are two distinct ones of fields 0..2 after RGBB's rotation
                TRY(arnt(u, z, f[3], rg, f[6], f[7], f[8], f[9], o.tol, o.maxit, E, gn));
            }
        }
        // final energy and gradient norm at the returned state
        TRY(grad(u, nullptr, rg));
        PULL(ds);
        st->energy = sc(SBEC_S_ENERGY);
        st->grad_norm = sqrt(sc(SBEC_S_RGRAD_NORM2));
        st->converged = st->grad_norm <= o.tol;
        if (cudaMemcpyAsync(Xdev, u, h->field_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SBEC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SBEC_ERR_CUDA;
        return st->converged ? SBEC_OK : SBEC_ERR_NOCONV;
    }
#undef TRY
#undef PULL
};

// ---------------------------------------------------------------------------
// Lock-step solver for a batch handle: every instance runs the same kernel
// sequence; per-instance steps, sigma, CG coefficients and active / accept flags
// live in each instance's scalar block and guard the updates, so finished
// instances are left unchanged (or recomputed identically).  The decisions are
// those of Solver<T> applied to each instance.
// ---------------------------------------------------------------------------

template <typename T>
struct BatchSolver {
    sbec_handle* h;
    const sbec::Geom& g;
    const sbec::Work& w;
    cudaStream_t s;
    sbec_solve_opts o;
    sbec_stats* st;
    int B;
    void* f[10];
    std::vector<int> dstat;
    CgChunks<T> cgc;

    BatchSolver(sbec_handle* hh, const sbec_solve_opts& oo, void* ws, sbec_stats* stt)
        : h(hh), g(hh->geom), w(hh->work), s(hh->stream), o(oo), st(stt), B(hh->B), dstat(hh->B, 0),
          cgc(hh, oo.cg_chunk, oo.cuda_graphs != 0) {
        char* b = static_cast<char*>(ws);
        for (int i = 0; i < 10; ++i) f[i] = b + (size_t)i * hh->field_bytes;
    }

    double* hs(int b) { return h->h_scal + (size_t)b * sbec::S_COUNT; }

    // scalars of every instance; per-instance device statuses go to dstat and are cleared
    int pull() {
        const size_t n = (size_t)B * sbec::S_COUNT;
        if (cudaMemcpyAsync(h->h_scal, w.scal, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SBEC_ERR_CUDA;
        bool any = false;
        for (int b = 0; b < B; ++b) {
            dstat[b] = (int)hs(b)[SBEC_S_STATUS];
            if (dstat[b]) { any = true; hs(b)[SBEC_S_STATUS] = 0.0; }
            if (dstat[b] && dstat[b] != SBEC_ERR_DOMAIN) return dstat[b];
        }
        return any ? push() : SBEC_OK;
    }
    // host-written parameter slots back to the device (the block is in sync after
    // pull), and the launches narrowed to the instances runset() left running: the
    // next kernels cover only those (slot -> instance map), so instances outside the
    // phase cost no blocks at all
    int push() {
        const size_t n = (size_t)B * sbec::S_COUNT;
        if (cudaMemcpyAsync(w.scal, h->h_scal, n * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SBEC_ERR_CUDA;
        int nl = 0;
        for (int b = 0; b < B; ++b)
            if (hs(b)[sbec::S_SKIP] == 0.0) h->h_imap[nl++] = b;
        if (nl == 0 || nl == B) {
            h->geom.nl = B;
            h->geom.imap = nullptr;
            return SBEC_OK;
        }
        if (cudaMemcpyAsync(h->d_imap, h->h_imap, (size_t)nl * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SBEC_ERR_CUDA;
        h->geom.nl = nl;
        h->geom.imap = h->d_imap;
        return SBEC_OK;
    }

    int lin(void* out, double ca, const void* A, double cb, const void* Bv, int ib = -1, int guard = -1,
            const void* D1 = nullptr, const void* D2 = nullptr, int slot = SL_D0) {
        Lin L;
        L.out = out; L.A = A; L.B = Bv; L.ca = ca; L.cb = cb; L.ia = -1; L.ib = ib; L.ineg = -1;
        L.D1 = D1; L.D2 = D2; L.guard = guard;
        return Ops<T>::lincomb(g, w, L, slot, s);
    }
    // only the instances with run[b] set take part in the next launches (the others'
    // arrays and scalars stay as they are); takes effect with the next push()
    void runset(const std::vector<char>& run) {
        for (int b = 0; b < B; ++b) hs(b)[sbec::S_SKIP] = run[b] ? 0.0 : 1.0;
    }
    void runall() {
        for (int b = 0; b < B; ++b) hs(b)[sbec::S_SKIP] = 0.0;
    }
    int grad(const void* u, void* gE, void* rg) {
        for (int b = 0; b < B; ++b) ++st[b].n_grad;
        return Ops<T>::grad(g, w, u, gE, rg, true, s);
    }
    int energy(const void* x) {
        for (int b = 0; b < B; ++b) ++st[b].n_energy;
        return Ops<T>::energy(g, w, x, s);
    }

#define TRY(x) do { int e_ = (x); if (e_) return e_; } while (0)

    int rgbb(void* u, void* up, void* z, void* rg, void* rgp, double tol, long long maxit, std::vector<double>& E,
             std::vector<double>& gn, std::vector<char>& act) {
        runset(act);
        TRY(push());
        TRY(energy(u));
        TRY(pull());
        std::vector<double> Ck(B), Qk(B, 1.0), t(B), slope(B), Ez(B);
        std::vector<char> tr(B);
        for (int b = 0; b < B; ++b) { E[b] = hs(b)[SBEC_S_ENERGY]; Ck[b] = E[b]; }
        bool have_prev = false;
        for (long long k = 0; k <= maxit; ++k) {
            TRY(grad(u, nullptr, rg));
            if (have_prev) TRY(Ops<T>::bbdots(g, w, u, up, rg, rgp, SL_D0, s));
            TRY(pull());
            bool any = false;
            for (int b = 0; b < B; ++b) {
                gn[b] = sqrt(hs(b)[SBEC_S_RGRAD_NORM2]);
                if (act[b] && (gn[b] <= tol || k == maxit)) act[b] = 0;
                any = any || act[b];
            }
            if (!any) return SBEC_OK;
            runset(act);
            for (int b = 0; b < B; ++b) {
                double gam = 1e-3;
                if (have_prev) {
                    const double sv = hs(b)[SL_D0], vv = hs(b)[SL_D0 + 1];
                    gam = vv > 0.0 ? fabs(sv) / vv : 1e-3;
                    gam = fmin(fmax(gam, 1e-10), 1e10);
                }
                t[b] = gam;
                slope[b] = -gn[b] * gn[b];
                tr[b] = act[b];
                Ez[b] = INFINITY;
            }
            for (int bt = 0; bt <= 10; ++bt) {
                for (int b = 0; b < B; ++b) hs(b)[SL_T] = act[b] ? -t[b] : 0.0;
                runset(tr);                              // accepted trials are kept as they are
                TRY(push());
                TRY(Ops<T>::retract(g, w, u, rg, 1.0, o.retraction, z, s, SL_T));
                TRY(energy(z));
                TRY(pull());
                bool more = false;
                for (int b = 0; b < B; ++b) {
                    if (!tr[b]) continue;
                    Ez[b] = dstat[b] == SBEC_ERR_DOMAIN ? INFINITY : hs(b)[SBEC_S_ENERGY];
                    const double noise = 100.0 * (sizeof(T) == 8 ? kEps : 1.1920928955078125e-07) *
                                         fmax(1.0, fabs(E[b]));
                    if (Ez[b] <= Ck[b] + 1e-4 * t[b] * slope[b] || fabs(Ez[b] - E[b]) <= noise) tr[b] = 0;
                    else if (bt < 10) t[b] *= 0.2;
                    more = more || tr[b];
                }
                if (!more) break;
            }
            for (int b = 0; b < B; ++b) {
                if (act[b] && !isfinite(Ez[b])) act[b] = 0;       // no admissible trial: stop this instance
                hs(b)[SL_ACT] = act[b] ? 1.0 : 0.0;
            }
            runset(act);
            TRY(push());
            TRY(lin(up, 1.0, u, 0.0, nullptr, -1, SL_ACT));
            TRY(lin(rgp, 1.0, rg, 0.0, nullptr, -1, SL_ACT));
            TRY(lin(u, 1.0, z, 0.0, nullptr, -1, SL_ACT));
            for (int b = 0; b < B; ++b) {
                if (!act[b]) continue;
                E[b] = Ez[b];
                const double Qn = 0.85 * Qk[b] + 1.0;
                Ck[b] = (0.85 * Qk[b] * Ck[b] + E[b]) / Qn;
                Qk[b] = Qn;
                ++st[b].rgbb_iters;
            }
            have_prev = true;
        }
        return SBEC_OK;
    }

    int arnt(void* u, void* z, void* gE, void* rg, void* x, void* r, void* p, void* Hp, double tol, long long maxit,
             std::vector<double>& E, std::vector<double>& gn) {
        runall();
        TRY(push());
        TRY(energy(u));
        TRY(pull());
        for (int b = 0; b < B; ++b) E[b] = hs(b)[SBEC_S_ENERGY];
        std::vector<double> sig_hat(B, 1.0), sig_floor(B, 0.0), sigma(B), rr(B), stop(B), sest(B), t(B), slope(B),
            mz(B), Ez(B);
        std::vector<int> maxin(B);
        std::vector<char> act(B), cg(B), neg(B), hd(B), ls(B);
        TRY(grad(u, gE, rg));
        TRY(pull());
        for (int b = 0; b < B; ++b) { gn[b] = sqrt(hs(b)[SBEC_S_RGRAD_NORM2]); act[b] = 1; }
        for (long long k = 0; k <= maxit; ++k) {
            bool any = false;
            for (int b = 0; b < B; ++b) {
                if (act[b] && (gn[b] <= tol || k == maxit)) act[b] = 0;
                any = any || act[b];
            }
            if (!any) break;
            for (int b = 0; b < B; ++b) {
                sigma[b] = fmax(sig_hat[b] * gn[b], sig_floor[b]);
                maxin[b] = gn[b] > 1e-3 ? 100 : 300;
                stop[b] = fmin(0.1, gn[b]) * gn[b];
                hs(b)[SL_SIG] = sigma[b];
            }
            runset(act);
            TRY(push());
            // ---- modified CG, lock-step over the instances still in it ----
            TRY(lin(x, 0.0, rg, 0.0, nullptr));
            TRY(lin(r, -1.0, rg, 0.0, nullptr, -1, -1, r, nullptr, SL_RRA));
            TRY(lin(p, 1.0, r, 0.0, nullptr));
            TRY(pull());
            bool incg = false;
            int cap_in = 0;
            for (int b = 0; b < B; ++b) {
                rr[b] = hs(b)[SL_RRA];
                cg[b] = act[b] && rr[b] > 0.0;
                neg[b] = 0; hd[b] = 0; sest[b] = -1.0;
                incg = incg || cg[b];
                double* q = hs(b);
                q[SL_CG] = cg[b] ? 1.0 : 0.0; q[SL_SIG] = sigma[b]; q[SL_STOP] = stop[b];
                q[SL_MAXIN] = (double)maxin[b]; q[SL_J] = 0.0; q[SL_SEST] = -1.0; q[SL_CGNEG] = 0.0;
                q[SL_CGHD] = 0.0;
                if (cg[b] && maxin[b] > cap_in) cap_in = maxin[b];
            }
            if (incg) {
                runset(cg);                              // instances outside the CG keep p, Hp, x, r
                TRY(push());
                // device-driven chunks (k_cg_update); the host reads the blocks once per chunk
                long long done_its = 0;
                while (true) {
                    TRY(cgc.run(u, p, Hp, x, r, (int)(done_its & 1)));
                    done_its += cgc.K;
                    TRY(pull());
                    int still = 0;
                    for (int b = 0; b < B; ++b) still += (cg[b] && hs(b)[SL_CG] != 0.0) ? 1 : 0;
                    if (!still) break;
                    if (done_its >= cap_in) return SBEC_ERR_CUDA;   // k_cg_update ends every CG by the cap
                    // once half of the launched instances have ended their CG, narrow the
                    // launches to the others (a new chunk graph per launched set)
                    if (2 * still <= h->geom.nl) TRY(push());
                }
                for (int b = 0; b < B; ++b) {
                    if (!cg[b]) continue;
                    const long long its = (long long)hs(b)[SL_J];
                    st[b].inner_iters += its;
                    st[b].n_hvp += its;
                    neg[b] = hs(b)[SL_CGNEG] != 0.0;
                    hd[b] = hs(b)[SL_CGHD] != 0.0;
                    sest[b] = hs(b)[SL_SEST];
                }
            }
            // ---- xi (Eq. xi) into x ----
            runset(act);
            bool anyneg = false, anyhd = false;
            for (int b = 0; b < B; ++b) {
                hs(b)[SL_NEG] = (act[b] && neg[b]) ? 1.0 : 0.0;
                anyneg = anyneg || (act[b] && neg[b]);
                anyhd = anyhd || (act[b] && hd[b]);
            }
            TRY(push());
            if (anyneg) TRY(lin(x, -1.0, rg, 0.0, nullptr, -1, SL_NEG));
            if (anyhd) {
                TRY(Ops<T>::dot2(g, w, p, rg, p, Hp, SL_D0, s));
                TRY(pull());
                for (int b = 0; b < B; ++b) {
                    const bool on = act[b] && hd[b];
                    hs(b)[SL_HD] = on ? 1.0 : 0.0;
                    hs(b)[SL_TAU] = on ? hs(b)[SL_D0] / hs(b)[SL_D0 + 1] : 0.0;
                }
                TRY(push());
                TRY(lin(x, 1.0, x, 1.0, p, SL_TAU, SL_HD));
            }
            TRY(Ops<T>::dot2(g, w, rg, x, nullptr, nullptr, SL_D0, s));
            TRY(pull());
            bool anyfix = false;
            for (int b = 0; b < B; ++b) {
                slope[b] = hs(b)[SL_D0];
                const bool fix = act[b] && (!(slope[b] < 0.0) || !isfinite(slope[b]));
                hs(b)[SL_NEG] = fix ? 1.0 : 0.0;
                if (fix) slope[b] = -gn[b] * gn[b];
                anyfix = anyfix || fix;
            }
            if (anyfix) {
                TRY(push());
                TRY(lin(x, -1.0, rg, 0.0, nullptr, -1, SL_NEG));
            }
            // ---- curvilinear search, lock-step ----
            const double eps = sizeof(T) == 8 ? kEps : 1.1920928955078125e-07;
            for (int b = 0; b < B; ++b) { t[b] = 1.0; ls[b] = act[b]; mz[b] = INFINITY; }
            for (int bt = 0; bt <= 10; ++bt) {
                for (int b = 0; b < B; ++b) hs(b)[SL_T] = act[b] ? t[b] : 0.0;
                runset(ls);                              // accepted trials are kept as they are
                TRY(push());
                TRY(Ops<T>::retract(g, w, u, x, 1.0, o.retraction, z, s, SL_T));
                TRY(lin(r, 1.0, z, -1.0, u, -1, -1, gE, r, SL_MA));
                for (int b = 0; b < B; ++b) ++st[b].n_hvp;
                TRY(Ops<T>::hessvec(g, w, u, r, 0.0, 0, Hp, s, -1, true));
                TRY(Ops<T>::dot2(g, w, r, Hp, nullptr, nullptr, SL_MB, s));
                TRY(pull());
                bool more = false;
                for (int b = 0; b < B; ++b) {
                    if (!ls[b]) continue;
                    const double noise = 100.0 * eps * fmax(1.0, fabs(E[b]));
                    mz[b] = dstat[b] == SBEC_ERR_DOMAIN
                                ? INFINITY
                                : hs(b)[SL_MA] + 0.5 * hs(b)[SL_MB] + 0.5 * sigma[b] * hs(b)[SL_MA + 1];
                    if (mz[b] <= 1e-4 * t[b] * slope[b] || fabs(mz[b]) <= noise) ls[b] = 0;
                    else if (bt < 10) t[b] *= 0.2;
                    more = more || ls[b];
                }
                if (!more) break;
            }
            runset(act);
            TRY(push());
            TRY(energy(z));
            TRY(pull());
            bool anyacc = false;
            for (int b = 0; b < B; ++b) {
                bool acc = false;
                if (act[b]) {
                    Ez[b] = dstat[b] == SBEC_ERR_DOMAIN ? INFINITY : hs(b)[SBEC_S_ENERGY];
                    const double noise = 100.0 * eps * fmax(1.0, fabs(E[b]));
                    double ratio;
                    if (fabs(mz[b]) <= noise && fabs(Ez[b] - E[b]) <= noise) ratio = 1.0;
                    else ratio = (mz[b] < 0.0 && isfinite(Ez[b])) ? (Ez[b] - E[b]) / mz[b] : -1.0;
                    acc = ratio >= 0.01;
                    if (acc) { E[b] = Ez[b]; sig_hat[b] *= (ratio >= 0.9) ? 0.2 : 1.0; }
                    else sig_hat[b] *= 10.0;
                    sig_floor[b] = sest[b] >= 0.0 ? sest[b] : 0.0;
                    ++st[b].outer_iters;
                }
                hs(b)[SL_ACC] = acc ? 1.0 : 0.0;
                anyacc = anyacc || acc;
            }
            std::vector<char> accv(B);
            for (int b = 0; b < B; ++b) accv[b] = hs(b)[SL_ACC] != 0.0;
            runset(accv);                                // rejected instances keep u, g, grad
            TRY(push());
            if (anyacc) {
                TRY(lin(u, 1.0, z, 0.0, nullptr, -1, SL_ACC));
                TRY(grad(u, gE, rg));
                TRY(pull());
                for (int b = 0; b < B; ++b)
                    if (accv[b]) gn[b] = sqrt(hs(b)[SBEC_S_RGRAD_NORM2]);
            }
            for (int b = 0; b < B; ++b)
                if (act[b] && sig_hat[b] > 1e20) act[b] = 0;
        }
        return SBEC_OK;
    }

    int run(void* Xdev) {
        void *u = f[0], *up = f[1], *z = f[2], *gE = f[3], *rg = f[4], *rgp = f[5];
        if (cudaMemcpyAsync(u, Xdev, h->field_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SBEC_ERR_CUDA;
        TRY(pull());
        runall();
        TRY(push());
        if (o.project_initial) {
            TRY(Ops<T>::retract(g, w, u, u, 0.0, 1, u, s));
            TRY(pull());
            for (int b = 0; b < B; ++b)
                if (dstat[b]) return SBEC_ERR_DOMAIN;
        }
        std::vector<double> E(B, 0.0), gn(B, INFINITY);
        std::vector<char> act(B, 1);
        if (o.method == SBEC_RGBB) {
            TRY(rgbb(u, up, z, rg, rgp, o.tol, o.maxit, E, gn, act));
        } else {
            TRY(rgbb(u, up, z, rg, rgp, fmax(o.tol, o.rgbb_tol), o.rgbb_maxit, E, gn, act));
            bool any = false;
            for (int b = 0; b < B; ++b) any = any || gn[b] > o.tol;
            if (any) TRY(arnt(u, z, gE, rg, f[6], f[7], f[8], f[9], o.tol, o.maxit, E, gn));
        }
        runall();
        TRY(push());
        TRY(grad(u, nullptr, rg));
        TRY(pull());
        bool all = true;
        for (int b = 0; b < B; ++b) {
            st[b].energy = hs(b)[SBEC_S_ENERGY];
            st[b].grad_norm = sqrt(hs(b)[SBEC_S_RGRAD_NORM2]);
            st[b].converged = st[b].grad_norm <= o.tol;
            all = all && st[b].converged;
        }
        if (cudaMemcpyAsync(Xdev, u, h->field_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SBEC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SBEC_ERR_CUDA;
        return all ? SBEC_OK : SBEC_ERR_NOCONV;
    }
#undef TRY
};

int solve_one(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
              sbec_stats* stats, const InnerCg* inner);

bool opts_valid(const sbec_solve_opts& o) {
    return o.retraction >= 1 && o.retraction <= 3 && o.tol > 0.0 && o.maxit >= 0 && o.rgbb_maxit >= 0 &&
           o.cg_chunk >= 1 && o.cg_chunk <= 64 && (o.cuda_graphs == 0 || o.cuda_graphs == 1) &&
           (o.refine_cg_fp32 == 0 || o.refine_cg_fp32 == 1);
}

}  // namespace

extern "C" {

void sbec_solve_defaults(sbec_solve_opts* o) {
    if (!o) return;
    o->method = SBEC_ARNT;
    o->retraction = 1;
    o->tol = 1e-6;
    o->maxit = 10000;
    o->rgbb_tol = 1e-2;
    o->rgbb_maxit = 2000;
    o->project_initial = 1;
    o->cg_chunk = 4;
    o->cuda_graphs = 1;
    o->refine_cg_fp32 = 1;
}

int sbec_solve_batch(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
                     sbec_stats* stats) {
    if (!h || !X || !workspace || !stats) return SBEC_ERR_ARG;
    if (workspace_bytes < 10 * h->field_bytes || !sbec_is_device_ptr(workspace) || !sbec_is_device_ptr(X))
        return SBEC_ERR_ARG;
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    if (!opts_valid(o)) return SBEC_ERR_ARG;
    memset(stats, 0, sizeof(sbec_stats) * (size_t)h->B);
    int rc;
    if (h->prob.precision == SBEC_FP64) {
        BatchSolver<double> S(h, o, workspace, stats);
        rc = S.run(X);
    } else {
        BatchSolver<float> S(h, o, workspace, stats);
        rc = S.run(X);
    }
    if (clear_skip(h) && rc == SBEC_OK) rc = SBEC_ERR_CUDA;
    h->last_grad_X = nullptr;
    return rc;
}

int sbec_solve_workspace_bytes(const sbec_handle* h, size_t* bytes) {
    if (!h || !bytes) return SBEC_ERR_ARG;
    *bytes = 10 * h->field_bytes;
    return SBEC_OK;
}

int sbec_solve(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
               sbec_stats* stats) {
    return solve_one(h, X, opts, workspace, workspace_bytes, stats, nullptr);
}

}  // extern "C"

namespace {

// sbec_solve, optionally with the modified CG of an FP64 solve on an FP32 context
int solve_one(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
              sbec_stats* stats, const InnerCg* inner) {
    if (!h || !X || !workspace) return SBEC_ERR_ARG;
    if (workspace_bytes < 10 * h->field_bytes || !sbec_is_device_ptr(workspace)) return SBEC_ERR_ARG;
    if (h->B != 1) return SBEC_ERR_ARG;       // batches: sbec_solve_batch
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    if (!opts_valid(o)) return SBEC_ERR_ARG;
    sbec_stats local;
    sbec_stats* st = stats ? stats : &local;
    memset(st, 0, sizeof(*st));
    // host arrays are staged through the handle's first staging field
    const bool host = !sbec_is_device_ptr(X);
    void* Xd = X;
    if (host) {
        Xd = h->stage[0];
        h->stage0_src = nullptr;     // the solve changes the staged copy
        if (cudaMemcpyAsync(Xd, X, h->field_bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
            return SBEC_ERR_CUDA;
    }
    int rc;
    if (h->prob.precision == SBEC_FP64) {
        Solver<double> S(h, o, workspace, st, inner);
        rc = S.run(Xd);
    } else {
        Solver<float> S(h, o, workspace, st);
        rc = S.run(Xd);
    }
    if (clear_skip(h) && rc == SBEC_OK) rc = SBEC_ERR_CUDA;
    if (inner && clear_skip(inner->h) && rc == SBEC_OK) rc = SBEC_ERR_CUDA;
    h->last_grad_X = nullptr;
    if (host && (rc == SBEC_OK || rc == SBEC_ERR_NOCONV)) {
        if (cudaMemcpyAsync(X, Xd, h->field_bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return SBEC_ERR_CUDA;
    }
    return rc;
}

}  // namespace


extern "C" {

// Mixed form (FP32 FFT and pointwise arithmetic, FP64 reductions and scalars)
// followed by an FP64 refinement from its result.
int sbec_solve_mixed_workspace_bytes(const sbec_handle* h64, const sbec_handle* h32, size_t* bytes) {
    if (!h64 || !h32 || !bytes) return SBEC_ERR_ARG;
    *bytes = 10 * h64->field_bytes + 11 * h32->field_bytes;
    return SBEC_OK;
}

int sbec_solve_mixed(sbec_handle* h64, sbec_handle* h32, void* X, const sbec_solve_opts* opts, double tol_mixed,
                     void* workspace, size_t workspace_bytes, sbec_stats* st_mixed, sbec_stats* st_fp64) {
    if (!h64 || !h32 || !X || !workspace) return SBEC_ERR_ARG;
    if (h64->prob.precision != SBEC_FP64 || h32->prob.precision != SBEC_MIXED) return SBEC_ERR_ARG;
    if (h64->geom.G != h32->geom.G || h64->geom.C != h32->geom.C || h64->stream != h32->stream) return SBEC_ERR_ARG;
    if (h64->B != h32->B) return SBEC_ERR_ARG;
    size_t need = 0;
    sbec_solve_mixed_workspace_bytes(h64, h32, &need);
    if (workspace_bytes < need || !sbec_is_device_ptr(X) || !sbec_is_device_ptr(workspace)) return SBEC_ERR_ARG;
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    char* base = static_cast<char*>(workspace);
    void* ws64 = base;
    void* X32 = base + 10 * h64->field_bytes;
    void* ws32 = base + 10 * h64->field_bytes + h32->field_bytes;
    const long long nreal = 2LL * h64->B * h64->geom.C * h64->geom.G;
    // one solve per phase: the lock-step batch solver for batch handles
    auto phase = [&](sbec_handle* h, void* Xp, const sbec_solve_opts* po, void* ws, sbec_stats* st) {
        return h->B > 1 ? sbec_solve_batch(h, Xp, po, ws, 10 * h->field_bytes, st)
                        : sbec_solve(h, Xp, po, ws, 10 * h->field_bytes, st);
    };
    const int blocks = 4 * h64->work.num_sms;
    k_cast<double, float><<<blocks, 256, 0, h64->stream>>>(static_cast<const double*>(X), static_cast<float*>(X32), nreal);
    if (cudaGetLastError() != cudaSuccess) return SBEC_ERR_CUDA;
    sbec_solve_opts om = o;
    om.tol = tol_mixed > o.tol ? tol_mixed : o.tol;
    // the FP32 phase only has to get close: below its rounding floor ARNT can stall
    // short of tol_mixed, so it stops after at most 300 iterations and the FP64
    // phase completes the solve from wherever it got
    if (om.maxit > 300) om.maxit = 300;
    int rc = phase(h32, X32, &om, ws32, st_mixed);
    if (rc != SBEC_OK && rc != SBEC_ERR_NOCONV) return rc;
    k_cast<float, double><<<blocks, 256, 0, h64->stream>>>(static_cast<const float*>(X32), static_cast<double*>(X), nreal);
    if (cudaGetLastError() != cudaSuccess) return SBEC_ERR_CUDA;
    sbec_solve_opts of = o;
    of.project_initial = 1;            // the float state is back on M to double precision
    if (h64->B == 1 && o.refine_cg_fp32) {
        // the FP32 phase is over: its fields hold the inner CG's float vectors
        InnerCg in;
        in.h = h32;
        for (int i = 0; i < 6; ++i) in.f[i] = static_cast<char*>(ws32) + (size_t)i * h32->field_bytes;
        return solve_one(h64, X, &of, ws64, 10 * h64->field_bytes, st_fp64, &in);
    }
    return phase(h64, X, &of, ws64, st_fp64);
}

// Cascadic multigrid (Algorithm 1, outer loop over meshes).
int sbec_prolongate(sbec_handle* hc, const void* Xc, sbec_handle* hf, void* Xf) {
    if (!hc || !hf || !Xc || !Xf) return SBEC_ERR_ARG;
    const sbec_problem &a = hc->prob, &b = hf->prob;
    if (a.F != b.F || a.dim != b.dim || a.precision != b.precision || hc->stream != hf->stream) return SBEC_ERR_ARG;
    for (int ax = 0; ax < a.dim; ++ax)
        if (b.n[ax] < a.n[ax] || a.lo[ax] != b.lo[ax] || a.hi[ax] != b.hi[ax]) return SBEC_ERR_ARG;
    bool host = false;
    const void* Xcd = Xc;
    if (!sbec_is_device_ptr(Xc)) {
        host = true;
        hc->stage0_src = nullptr;
        if (cudaMemcpyAsync(hc->stage[0], Xc, hc->field_bytes, cudaMemcpyHostToDevice, hc->stream) != cudaSuccess)
            return SBEC_ERR_CUDA;
        Xcd = hc->stage[0];
    }
    void* Xfd = Xf;
    if (!sbec_is_device_ptr(Xf)) { host = true; Xfd = hf->stage[2]; }
    const int st = a.precision == SBEC_FP64
                       ? sbec::Ops<double>::prolongate(hc->geom, hc->work, Xcd, hf->geom, hf->work, Xfd, hf->stream)
                       : sbec::Ops<float>::prolongate(hc->geom, hc->work, Xcd, hf->geom, hf->work, Xfd, hf->stream);
    if (st) return st;
    if (Xfd != Xf && cudaMemcpyAsync(Xf, Xfd, hf->field_bytes, cudaMemcpyDeviceToHost, hf->stream) != cudaSuccess)
        return SBEC_ERR_CUDA;
    hf->last_grad_X = nullptr;
    return host ? sbec_read_scalars(hf) : SBEC_OK;
}

int sbec_solve_cascadic(sbec_handle* const* levels, int nlevels, void* const* X, const sbec_solve_opts* opts,
                        double tol_coarse, void* workspace, size_t workspace_bytes, sbec_stats* stats) {
    if (!levels || !X || nlevels < 1) return SBEC_ERR_ARG;
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    int rc = SBEC_OK;
    for (int j = 0; j < nlevels; ++j) {
        if (!levels[j] || !X[j]) return SBEC_ERR_ARG;
        if (j > 0) {
            rc = sbec_prolongate(levels[j - 1], X[j - 1], levels[j], X[j]);
            if (rc) return rc;
        }
        sbec_solve_opts oj = o;
        const bool finest = (j == nlevels - 1);
        oj.tol = finest ? o.tol : (tol_coarse > o.tol ? tol_coarse : o.tol);
        oj.project_initial = (j == 0) ? o.project_initial : 0;     // the prolongation ends with R1
        sbec_stats local;
        rc = sbec_solve(levels[j], X[j], &oj, workspace, workspace_bytes, finest && stats ? stats : &local);
        if (rc != SBEC_OK && !(rc == SBEC_ERR_NOCONV && !finest)) return rc;
    }
    return rc;
}

// Cascadic multigrid with the mixed form on every level: sbec_solve_mixed per
// level (FP32 phase, FP64 refinement), prolongation of the refined FP64 state.
int sbec_solve_cascadic_mixed(sbec_handle* const* levels64, sbec_handle* const* levels32, int nlevels,
                              void* const* X, const sbec_solve_opts* opts, double tol_coarse, double tol_mixed,
                              void* workspace, size_t workspace_bytes, sbec_stats* st_mixed, sbec_stats* st_fp64) {
    if (!levels64 || !levels32 || !X || nlevels < 1) return SBEC_ERR_ARG;
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    int rc = SBEC_OK;
    for (int j = 0; j < nlevels; ++j) {
        if (!levels64[j] || !levels32[j] || !X[j]) return SBEC_ERR_ARG;
        if (levels64[j]->B != 1) return SBEC_ERR_ARG;
        if (j > 0) {
            rc = sbec_prolongate(levels64[j - 1], X[j - 1], levels64[j], X[j]);
            if (rc) return rc;
        }
        sbec_solve_opts oj = o;
        const bool finest = (j == nlevels - 1);
        oj.tol = finest ? o.tol : (tol_coarse > o.tol ? tol_coarse : o.tol);
        oj.project_initial = (j == 0) ? o.project_initial : 0;
        sbec_stats lm, lf;
        rc = sbec_solve_mixed(levels64[j], levels32[j], X[j], &oj, tol_mixed, workspace, workspace_bytes,
                              finest && st_mixed ? st_mixed : &lm, finest && st_fp64 ? st_fp64 : &lf);
        if (rc != SBEC_OK && !(rc == SBEC_ERR_NOCONV && !finest)) return rc;
    }
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Device-driven solve (Algorithm 1 as one CUDA graph).  Every decision the
// lock-step batch solver takes on the host -- the RGBB step and its nonmonotone
// search, the modified CG's end, the direction of Eq. (xi), the curvilinear
// search, the ratio test and the sigma update -- is taken per instance by
// one-block control kernels on the device, in the same formulas and order.  The
// loops are conditional WHILE nodes of the graph whose condition the control
// kernels set (cudaGraphSetConditional); kernels of instances outside the
// current sub-phase return at once through the instances' S_SKIP flags.  Several
// batch handles (e.g. the grid-size classes of an uneven sweep) are parallel
// branches of the same graph, so one launch solves all of them; the host reads
// the scalar blocks once, after the graph.  Every loop counts its body
// executions and stops at a cap, recording SBEC_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
namespace {

// per-instance state of the device-driven solve (scalar-block slots after the
// solver slots of the host-driven solvers)
enum {
    DS_E = 64, DS_GN, DS_CK, DS_QK, DS_T, DS_SLOPE, DS_EZ, DS_BT, DS_ACT, DS_TR, DS_K, DS_PREV,
    DS_SIGHAT, DS_SIGFLOOR, DS_MZ, DS_CGON, DS_NEG, DS_HD, DS_SEST, DS_OUTER, DS_INNER, DS_RGBBIT,
    DS_NGRAD, DS_NENERGY, DS_NHVP, DS_ERR, DS_DOM, DS_LOOP0 /* 5 loop counters, instance 0 */
};
static_assert(int(DS_LOOP0) + 5 <= int(sbec::S_COUNT), "device solver slots exceed the scalar block");

enum GPhase {
    G_INIT, G_RGBB_GRAD, G_RGBB_LS, G_RGBB_ACC, G_RGBB_END, G_ARNT_E, G_ARNT_INIT, G_ARNT_TOP, G_ARNT_CG0,
    G_CG_ANY, G_ARNT_DIR, G_ARNT_TAU, G_ARNT_SLOPE, G_ARNT_LS0, G_ARNT_LS, G_ARNT_E2, G_ARNT_ACC, G_ARNT_END,
    G_FINAL
};

struct GCtl {
    int B;
    double tol_r, tol;          // RGBB tolerance (warm start or final), ARNT tolerance
    long long maxit_r, maxit;
    double eps;                 // unit roundoff of the handle's precision (rounding floor)
    long long cap;              // loop-body executions per loop before SBEC_ERR_TIMEOUT
};

// status of instance b after the latest kernels: 0, DOMAIN (cleared, reported
// back) or a fatal code (recorded in DS_ERR)
__device__ __forceinline__ int take_status(double* sc) {
    const int st = (int)sc[SBEC_S_STATUS];
    sc[SBEC_S_STATUS] = 0.0;
    if (st != 0 && st != SBEC_ERR_DOMAIN && sc[DS_ERR] == 0.0) sc[DS_ERR] = double(st);
    return st;
}

// One block over all instances of a branch; thread 0 sets the loop conditions.
__global__ void __launch_bounds__(1024) k_gctl(double* scal0, const GCtl c, int phase, cudaGraphConditionalHandle h1,
                                               cudaGraphConditionalHandle h2, int loop) {
    __shared__ int any1, any2, over;
    if (threadIdx.x == 0) { any1 = 0; any2 = 0; over = 0; }
    __syncthreads();
    for (int b = threadIdx.x; b < c.B; b += blockDim.x) {
        double* sc = scal0 + (size_t)b * sbec::S_COUNT;
        const double noise = 100.0 * c.eps * fmax(1.0, fabs(sc[DS_E]));
        switch (phase) {
            case G_INIT: {
                const int st = take_status(sc);
                if (st == SBEC_ERR_DOMAIN && sc[DS_ERR] == 0.0) sc[DS_ERR] = double(SBEC_ERR_DOMAIN);
                sc[DS_E] = sc[SBEC_S_ENERGY];
                sc[DS_CK] = sc[DS_E]; sc[DS_QK] = 1.0;
                sc[DS_ACT] = sc[DS_ERR] == 0.0 ? 1.0 : 0.0;
                sc[DS_K] = 0.0; sc[DS_PREV] = 0.0;
                sc[DS_NENERGY] += 1.0;
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                if (sc[DS_ACT] != 0.0) atomicOr(&any1, 1);
                break;
            }
            case G_RGBB_GRAD: {
                sc[DS_NGRAD] += 1.0;
                take_status(sc);
                if (sc[DS_ERR] != 0.0) sc[DS_ACT] = 0.0;
                const double gn = sqrt(sc[SBEC_S_RGRAD_NORM2]);
                if (sc[DS_ACT] != 0.0) sc[DS_GN] = gn;
                if (sc[DS_ACT] != 0.0 && (gn <= c.tol_r || sc[DS_K] == (double)c.maxit_r)) sc[DS_ACT] = 0.0;
                const bool act = sc[DS_ACT] != 0.0;
                if (act) {
                    double gam = 1e-3;
                    if (sc[DS_PREV] != 0.0) {
                        const double sv = sc[SL_D0], vv = sc[SL_D0 + 1];
                        gam = vv > 0.0 ? fabs(sv) / vv : 1e-3;
                        gam = fmin(fmax(gam, 1e-10), 1e10);
                    }
                    sc[DS_T] = gam;
                    sc[DS_SLOPE] = -gn * gn;
                    sc[DS_EZ] = INFINITY;
                    sc[DS_BT] = 0.0;
                    atomicOr(&any1, 1);
                }
                sc[DS_TR] = act ? 1.0 : 0.0;
                sc[SL_T] = act ? -sc[DS_T] : 0.0;
                sc[sbec::S_SKIP] = act ? 0.0 : 1.0;
                break;
            }
            case G_RGBB_LS: {
                sc[DS_NENERGY] += 1.0;
                const int st = take_status(sc);
                if (sc[DS_TR] != 0.0) {
                    const double Ez = (st == SBEC_ERR_DOMAIN) ? INFINITY : sc[SBEC_S_ENERGY];
                    sc[DS_EZ] = Ez;
                    const double t = sc[DS_T];
                    if (sc[DS_ERR] != 0.0) {
                        sc[DS_TR] = 0.0;
                    } else if (Ez <= sc[DS_CK] + 1e-4 * t * sc[DS_SLOPE] || fabs(Ez - sc[DS_E]) <= noise) {
                        sc[DS_TR] = 0.0;
                    } else if (sc[DS_BT] < 10.0) {
                        sc[DS_T] = 0.2 * t;
                    } else {
                        sc[DS_TR] = 0.0;
                    }
                    sc[DS_BT] += 1.0;
                }
                const bool tr = sc[DS_TR] != 0.0;
                sc[SL_T] = (sc[DS_ACT] != 0.0) ? -sc[DS_T] : 0.0;
                sc[sbec::S_SKIP] = tr ? 0.0 : 1.0;
                if (tr) atomicOr(&any1, 1);
                break;
            }
            case G_RGBB_ACC: {
                if (sc[DS_ACT] != 0.0 && (!isfinite(sc[DS_EZ]) || sc[DS_ERR] != 0.0)) sc[DS_ACT] = 0.0;
                sc[SL_ACT] = sc[DS_ACT];
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                break;
            }
            case G_RGBB_END: {
                if (sc[DS_ACT] != 0.0) {
                    sc[DS_E] = sc[DS_EZ];
                    const double Qn = 0.85 * sc[DS_QK] + 1.0;
                    sc[DS_CK] = (0.85 * sc[DS_QK] * sc[DS_CK] + sc[DS_E]) / Qn;
                    sc[DS_QK] = Qn;
                    sc[DS_RGBBIT] += 1.0;
                    sc[DS_K] += 1.0;
                    sc[DS_PREV] = 1.0;
                    atomicOr(&any1, 1);
                }
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_E: {
                // RGBB over: every instance without a fatal error takes part in ARNT
                sc[DS_NENERGY] += 1.0;
                take_status(sc);
                sc[DS_E] = sc[SBEC_S_ENERGY];
                sc[DS_ACT] = sc[DS_ERR] == 0.0 ? 1.0 : 0.0;
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_INIT: {
                sc[DS_NGRAD] += 1.0;
                take_status(sc);
                if (sc[DS_ERR] != 0.0) sc[DS_ACT] = 0.0;
                sc[DS_GN] = sqrt(sc[SBEC_S_RGRAD_NORM2]);
                sc[DS_SIGHAT] = 1.0; sc[DS_SIGFLOOR] = 0.0; sc[DS_K] = 0.0;
                if (sc[DS_ACT] != 0.0 && (sc[DS_GN] <= c.tol || c.maxit == 0)) sc[DS_ACT] = 0.0;
                if (sc[DS_ACT] != 0.0) atomicOr(&any1, 1);
                break;
            }
            case G_ARNT_TOP: {
                if (sc[DS_ACT] != 0.0 && (sc[DS_GN] <= c.tol || sc[DS_K] == (double)c.maxit)) sc[DS_ACT] = 0.0;
                const bool act = sc[DS_ACT] != 0.0;
                const double gn = sc[DS_GN];
                if (act) {
                    sc[SL_SIG] = fmax(sc[DS_SIGHAT] * gn, sc[DS_SIGFLOOR]);
                    sc[SL_MAXIN] = gn > 1e-3 ? 100.0 : 300.0;
                    sc[SL_STOP] = fmin(0.1, gn) * gn;
                }
                sc[sbec::S_SKIP] = act ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_CG0: {
                const bool act = sc[DS_ACT] != 0.0;
                const bool cg = act && sc[SL_RRA] > 0.0;
                sc[DS_CGON] = cg ? 1.0 : 0.0;
                sc[DS_NEG] = 0.0; sc[DS_HD] = 0.0; sc[DS_SEST] = -1.0;
                sc[SL_CG] = cg ? 1.0 : 0.0;
                sc[SL_J] = 0.0; sc[SL_SEST] = -1.0; sc[SL_CGNEG] = 0.0; sc[SL_CGHD] = 0.0;
                sc[sbec::S_SKIP] = cg ? 0.0 : 1.0;
                if (cg) atomicOr(&any1, 1);
                break;
            }
            case G_CG_ANY: {
                take_status(sc);
                if (sc[DS_CGON] != 0.0 && sc[SL_CG] != 0.0) atomicOr(&any1, 1);
                break;
            }
            case G_ARNT_DIR: {
                const bool act = sc[DS_ACT] != 0.0;
                if (sc[DS_CGON] != 0.0) {
                    sc[DS_INNER] += sc[SL_J];
                    sc[DS_NHVP] += sc[SL_J];
                    sc[DS_NEG] = sc[SL_CGNEG] != 0.0 ? 1.0 : 0.0;
                    sc[DS_HD] = sc[SL_CGHD] != 0.0 ? 1.0 : 0.0;
                    sc[DS_SEST] = sc[SL_SEST];
                }
                sc[SL_NEG] = (act && sc[DS_NEG] != 0.0) ? 1.0 : 0.0;
                sc[SL_HD] = (act && sc[DS_HD] != 0.0) ? 1.0 : 0.0;
                sc[sbec::S_SKIP] = act ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_TAU: {
                sc[SL_TAU] = sc[SL_HD] != 0.0 ? sc[SL_D0] / sc[SL_D0 + 1] : 0.0;
                break;
            }
            case G_ARNT_SLOPE: {
                const bool act = sc[DS_ACT] != 0.0;
                double slope = sc[SL_D0];
                const bool fix = act && (!(slope < 0.0) || !isfinite(slope));
                if (fix) slope = -sc[DS_GN] * sc[DS_GN];
                sc[DS_SLOPE] = slope;
                sc[SL_NEG] = fix ? 1.0 : 0.0;
                break;
            }
            case G_ARNT_LS0: {
                const bool act = sc[DS_ACT] != 0.0;
                sc[DS_T] = 1.0; sc[DS_MZ] = INFINITY; sc[DS_BT] = 0.0;
                sc[DS_TR] = act ? 1.0 : 0.0;
                sc[SL_T] = act ? 1.0 : 0.0;
                sc[sbec::S_SKIP] = act ? 0.0 : 1.0;
                if (act) atomicOr(&any1, 1);
                break;
            }
            case G_ARNT_LS: {
                sc[DS_NHVP] += 1.0;
                const int st = take_status(sc);
                if (sc[DS_TR] != 0.0) {
                    const double mz = (st == SBEC_ERR_DOMAIN)
                                          ? INFINITY
                                          : sc[SL_MA] + 0.5 * sc[SL_MB] + 0.5 * sc[SL_SIG] * sc[SL_MA + 1];
                    sc[DS_MZ] = mz;
                    const double t = sc[DS_T];
                    if (sc[DS_ERR] != 0.0 || mz <= 1e-4 * t * sc[DS_SLOPE] || fabs(mz) <= noise) {
                        sc[DS_TR] = 0.0;
                    } else if (sc[DS_BT] < 10.0) {
                        sc[DS_T] = 0.2 * t;
                    } else {
                        sc[DS_TR] = 0.0;
                    }
                    sc[DS_BT] += 1.0;
                }
                const bool tr = sc[DS_TR] != 0.0;
                sc[SL_T] = sc[DS_ACT] != 0.0 ? sc[DS_T] : 0.0;
                sc[sbec::S_SKIP] = tr ? 0.0 : 1.0;
                if (tr) atomicOr(&any1, 1);
                break;
            }
            case G_ARNT_E2: {
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_ACC: {
                sc[DS_NENERGY] += 1.0;
                const int st = take_status(sc);
                bool acc = false;
                if (sc[DS_ACT] != 0.0) {
                    const double Ez = (st == SBEC_ERR_DOMAIN) ? INFINITY : sc[SBEC_S_ENERGY];
                    const double mz = sc[DS_MZ], E = sc[DS_E];
                    double ratio;
                    if (fabs(mz) <= noise && fabs(Ez - E) <= noise) ratio = 1.0;
                    else ratio = (mz < 0.0 && isfinite(Ez)) ? (Ez - E) / mz : -1.0;
                    acc = ratio >= 0.01 && sc[DS_ERR] == 0.0;
                    if (acc) {
                        sc[DS_E] = Ez;
                        sc[DS_SIGHAT] *= (ratio >= 0.9) ? 0.2 : 1.0;
                    } else {
                        sc[DS_SIGHAT] *= 10.0;
                    }
                    sc[DS_SIGFLOOR] = sc[DS_SEST] >= 0.0 ? sc[DS_SEST] : 0.0;
                    sc[DS_OUTER] += 1.0;
                }
                sc[SL_ACC] = acc ? 1.0 : 0.0;
                sc[sbec::S_SKIP] = acc ? 0.0 : 1.0;
                break;
            }
            case G_ARNT_END: {
                if (sc[SL_ACC] != 0.0) {
                    sc[DS_NGRAD] += 1.0;
                    take_status(sc);
                    sc[DS_GN] = sqrt(sc[SBEC_S_RGRAD_NORM2]);
                }
                if (sc[DS_ERR] != 0.0) sc[DS_ACT] = 0.0;
                if (sc[DS_ACT] != 0.0) {
                    sc[DS_K] += 1.0;
                    if (sc[DS_SIGHAT] > 1e20) sc[DS_ACT] = 0.0;
                }
                // the next iteration's top test, so that the loop ends without an empty pass
                if (sc[DS_ACT] != 0.0 && !(sc[DS_GN] <= c.tol || sc[DS_K] == (double)c.maxit)) atomicOr(&any1, 1);
                sc[sbec::S_SKIP] = sc[DS_ACT] != 0.0 ? 0.0 : 1.0;
                break;
            }
            case G_FINAL: {
                sc[DS_NGRAD] += 1.0;
                sc[sbec::S_SKIP] = 0.0;
                break;
            }
            default:
                break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // loop bookkeeping: body executions of loop `loop` (instance 0's block)
        if (loop >= 0) {
            double* cnt = scal0 + DS_LOOP0 + loop;
            cnt[0] += 1.0;
            if (cnt[0] >= (double)c.cap) {
                over = 1;
                if (scal0[DS_ERR] == 0.0) scal0[DS_ERR] = double(SBEC_ERR_TIMEOUT);
            }
        }
        if (h1) cudaGraphSetConditional(h1, (any1 && !over) ? 1u : 0u);
        if (h2) cudaGraphSetConditional(h2, (any2 && !over) ? 1u : 0u);
    }
}

// every instance's device-solver state back to zero (the launch of a solve)
__global__ void k_gclear(double* scal0, int B) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * (sbec::S_COUNT - DS_E); i += gridDim.x * blockDim.x) {
        const int b = i / (sbec::S_COUNT - DS_E), k = i % (sbec::S_COUNT - DS_E);
        scal0[(size_t)b * sbec::S_COUNT + DS_E + k] = 0.0;
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        scal0[(size_t)b * sbec::S_COUNT + sbec::S_SKIP] = 0.0;
        scal0[(size_t)b * sbec::S_COUNT + SBEC_S_STATUS] = 0.0;
    }
}

// Builds one branch (one handle) of the device-driven graph by stream capture.
template <typename T>
struct GraphBranch {
    sbec_handle* h;
    sbec::Geom g;
    sbec::Work w;          // the handle's work area without the event profiler
    sbec_solve_opts o;
    GCtl ctl;
    void* f[10];
    void* Xdev;
    cudaStream_t st[4] = {};   // capture streams by nesting depth
    CgChunks<T>* cg = nullptr;
    int err = SBEC_OK;

    GraphBranch(sbec_handle* hh, const sbec_solve_opts& oo, void* ws, void* X, long long cap) : h(hh), g(hh->geom), w(hh->work), o(oo) {
        w.prof = nullptr;
        g.nl = hh->B;
        g.imap = nullptr;
        char* b = static_cast<char*>(ws);
        for (int i = 0; i < 10; ++i) f[i] = b + (size_t)i * hh->field_bytes;
        Xdev = X;
        ctl.B = hh->B;
        ctl.tol = o.tol;
        ctl.tol_r = o.method == SBEC_RGBB ? o.tol : fmax(o.tol, o.rgbb_tol);
        ctl.maxit_r = o.method == SBEC_RGBB ? o.maxit : o.rgbb_maxit;
        ctl.maxit = o.maxit;
        ctl.eps = sizeof(T) == 8 ? kEps : 1.1920928955078125e-07;
        ctl.cap = cap;
        for (auto& s : st)
            if (!err && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) err = SBEC_ERR_CUDA;
        cg = new CgChunks<T>(hh, 2, false);
    }
    ~GraphBranch() {
        delete cg;
        for (auto& s : st)
            if (s) cudaStreamDestroy(s);
    }

#define GTRY(x) do { int e_ = (x); if (e_) return e_; } while (0)
    int ctlk(cudaStream_t s, int phase, cudaGraphConditionalHandle h1 = 0, cudaGraphConditionalHandle h2 = 0,
             int loop = -1) {
        k_gctl<<<1, 1024, 0, s>>>(w.scal, ctl, phase, h1, h2, loop);
        return cudaGetLastError() == cudaSuccess ? SBEC_OK : SBEC_ERR_CUDA;
    }
    int lin(cudaStream_t s, void* out, double ca, const void* A, double cb, const void* B, int ib = -1,
            int guard = -1, const void* D1 = nullptr, const void* D2 = nullptr, int slot = SL_D0) {
        Lin L;
        L.out = out; L.A = A; L.B = B; L.ca = ca; L.cb = cb; L.ia = -1; L.ib = ib; L.ineg = -1;
        L.D1 = D1; L.D2 = D2; L.guard = guard;
        return Ops<T>::lincomb(g, w, L, slot, s);
    }

    // WHILE node on the stream capturing at `depth`: the body is captured on the
    // stream of depth + 1 by body(stream); the handle is created before the node so
    // that the kernel ahead of it (set_cond) can set its first value.
    template <typename Body>
    int while_node(int depth, cudaGraphConditionalHandle hnd, Body body) {
        cudaStream_t s = st[depth], sb = st[depth + 1];
        cudaStreamCaptureStatus cs;
        cudaGraph_t graph;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess ||
            cs != cudaStreamCaptureStatusActive)
            return SBEC_ERR_CUDA;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp) != cudaSuccess) return SBEC_ERR_CUDA;
        cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(sb, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess)
            return SBEC_ERR_CUDA;
        const int e = body(sb);
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(sb, &out);
        if (e) return e;
        if (ee != cudaSuccess) return SBEC_ERR_CUDA;
        if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
            return SBEC_ERR_CUDA;
        return SBEC_OK;
    }
    int handle_in(int depth, cudaGraphConditionalHandle* hnd) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t graph;
        if (cudaStreamGetCaptureInfo(st[depth], &cs, nullptr, &graph, nullptr, nullptr, nullptr) != cudaSuccess ||
            cs != cudaStreamCaptureStatusActive)
            return SBEC_ERR_CUDA;
        return cudaGraphConditionalHandleCreate(hnd, graph, 0, 0) == cudaSuccess ? SBEC_OK : SBEC_ERR_CUDA;
    }

    // Captures the whole solve of this handle on st[0] (already capturing).
    int build() {
        if (err) return err;
        cudaStream_t s0 = st[0];
        void *u = f[0], *up = f[1], *z = f[2], *gE = f[3], *rg = f[4], *rgp = f[5];
        void *x = f[6], *r = f[7], *p = f[8], *Hp = f[9];
        k_gclear<<<8, 256, 0, s0>>>(w.scal, h->B);
        if (cudaGetLastError() != cudaSuccess) return SBEC_ERR_CUDA;
        // every work field starts at zero: the kernels that run for all instances (the
        // BB dots before the first step, the direction dots) then only see finite values
        if (cudaMemsetAsync(f[0], 0, 10 * h->field_bytes, s0) != cudaSuccess) return SBEC_ERR_CUDA;
        if (cudaMemcpyAsync(u, Xdev, h->field_bytes, cudaMemcpyDeviceToDevice, s0) != cudaSuccess) return SBEC_ERR_CUDA;
        if (o.project_initial) GTRY(Ops<T>::retract(g, w, u, u, 0.0, 1, u, s0));
        GTRY(Ops<T>::energy(g, w, u, s0));
        // ---- RGBB (warm start, or the whole solve) ----
        cudaGraphConditionalHandle c_rgbb, c_rls;
        GTRY(handle_in(0, &c_rgbb));
        GTRY(ctlk(s0, G_INIT, c_rgbb));
        GTRY(while_node(0, c_rgbb, [&](cudaStream_t s1) -> int {
            GTRY(Ops<T>::grad(g, w, u, nullptr, rg, true, s1));
            GTRY(Ops<T>::bbdots(g, w, u, up, rg, rgp, SL_D0, s1));
            GTRY(handle_in(1, &c_rls));
            GTRY(ctlk(s1, G_RGBB_GRAD, c_rls, 0, 0));
            GTRY(while_node(1, c_rls, [&](cudaStream_t s2) -> int {
                GTRY(Ops<T>::retract(g, w, u, rg, 1.0, o.retraction, z, s2, SL_T));
                GTRY(Ops<T>::energy(g, w, z, s2));
                return ctlk(s2, G_RGBB_LS, c_rls, 0, 1);
            }));
            GTRY(ctlk(s1, G_RGBB_ACC));
            GTRY(lin(s1, up, 1.0, u, 0.0, nullptr, -1, SL_ACT));
            GTRY(lin(s1, rgp, 1.0, rg, 0.0, nullptr, -1, SL_ACT));
            GTRY(lin(s1, u, 1.0, z, 0.0, nullptr, -1, SL_ACT));
            return ctlk(s1, G_RGBB_END, c_rgbb);
        }));
        if (o.method != SBEC_RGBB) {
            // ---- ARNT (Algorithm 1, second loop) ----
            k_unskip<<<(h->B + 127) / 128, 128, 0, s0>>>(w.scal, h->B);
            if (cudaGetLastError() != cudaSuccess) return SBEC_ERR_CUDA;
            GTRY(Ops<T>::energy(g, w, u, s0));
            GTRY(ctlk(s0, G_ARNT_E));
            GTRY(Ops<T>::grad(g, w, u, gE, rg, true, s0));
            cudaGraphConditionalHandle c_arnt, c_cg, c_ls;
            GTRY(handle_in(0, &c_arnt));
            GTRY(ctlk(s0, G_ARNT_INIT, c_arnt));
            GTRY(while_node(0, c_arnt, [&](cudaStream_t s1) -> int {
                GTRY(ctlk(s1, G_ARNT_TOP));
                GTRY(lin(s1, x, 0.0, rg, 0.0, nullptr));
                GTRY(lin(s1, r, -1.0, rg, 0.0, nullptr, -1, -1, r, nullptr, SL_RRA));
                GTRY(lin(s1, p, 1.0, r, 0.0, nullptr));
                GTRY(handle_in(1, &c_cg));
                GTRY(ctlk(s1, G_ARNT_CG0, c_cg));
                GTRY(while_node(1, c_cg, [&](cudaStream_t s2) -> int {
                    GTRY(cg->launch(s2, u, p, Hp, x, r, 0));
                    return ctlk(s2, G_CG_ANY, c_cg, 0, 2);
                }));
                GTRY(ctlk(s1, G_ARNT_DIR));
                GTRY(lin(s1, x, -1.0, rg, 0.0, nullptr, -1, SL_NEG));
                GTRY(Ops<T>::dot2(g, w, p, rg, p, Hp, SL_D0, s1));
                GTRY(ctlk(s1, G_ARNT_TAU));
                GTRY(lin(s1, x, 1.0, x, 1.0, p, SL_TAU, SL_HD));
                GTRY(Ops<T>::dot2(g, w, rg, x, nullptr, nullptr, SL_D0, s1));
                GTRY(ctlk(s1, G_ARNT_SLOPE));
                GTRY(lin(s1, x, -1.0, rg, 0.0, nullptr, -1, SL_NEG));
                GTRY(handle_in(1, &c_ls));
                GTRY(ctlk(s1, G_ARNT_LS0, c_ls));
                GTRY(while_node(1, c_ls, [&](cudaStream_t s2) -> int {
                    GTRY(Ops<T>::retract(g, w, u, x, 1.0, o.retraction, z, s2, SL_T));
                    GTRY(lin(s2, r, 1.0, z, -1.0, u, -1, -1, gE, r, SL_MA));
                    GTRY(Ops<T>::hessvec(g, w, u, r, 0.0, 0, Hp, s2, -1, true));
                    GTRY(Ops<T>::dot2(g, w, r, Hp, nullptr, nullptr, SL_MB, s2));
                    return ctlk(s2, G_ARNT_LS, c_ls, 0, 3);
                }));
                GTRY(ctlk(s1, G_ARNT_E2));
                GTRY(Ops<T>::energy(g, w, z, s1));
                GTRY(ctlk(s1, G_ARNT_ACC));
                GTRY(lin(s1, u, 1.0, z, 0.0, nullptr, -1, SL_ACC));
                GTRY(Ops<T>::grad(g, w, u, gE, rg, true, s1));
                return ctlk(s1, G_ARNT_END, c_arnt, 0, 4);
            }));
        }
        // ---- the returned state: energy and gradient norm of every instance ----
        GTRY(ctlk(s0, G_FINAL));
        GTRY(Ops<T>::grad(g, w, u, nullptr, rg, true, s0));
        if (cudaMemcpyAsync(Xdev, u, h->field_bytes, cudaMemcpyDeviceToDevice, s0) != cudaSuccess) return SBEC_ERR_CUDA;
        return SBEC_OK;
    }
#undef GTRY
};

}  // namespace

extern "C" int sbec_solve_graph(sbec_handle* const* handles, int nh, void* const* X, const sbec_solve_opts* opts,
                                void* const* workspaces, const size_t* workspace_bytes, long long loop_cap,
                                sbec_stats* const* stats) {
    if (!handles || nh < 1 || nh > 16 || !X || !workspaces || !workspace_bytes || !stats) return SBEC_ERR_ARG;
    sbec_solve_opts o;
    if (opts) o = *opts; else sbec_solve_defaults(&o);
    if (!opts_valid(o)) return SBEC_ERR_ARG;
    if (loop_cap <= 0) loop_cap = 1000000;
    sbec_handle* h0 = handles[0];
    for (int i = 0; i < nh; ++i) {
        sbec_handle* h = handles[i];
        if (!h || !X[i] || !workspaces[i] || !stats[i]) return SBEC_ERR_ARG;
        if (h->prob.precision != h0->prob.precision || h->device != h0->device || h->B > 1024) return SBEC_ERR_ARG;
        if (workspace_bytes[i] < 10 * h->field_bytes || !sbec_is_device_ptr(workspaces[i]) ||
            !sbec_is_device_ptr(X[i]))
            return SBEC_ERR_ARG;
        if (h->prof.enabled) return SBEC_ERR_ARG;     // event timing cannot be captured
    }
    const bool fp64 = h0->prob.precision == SBEC_FP64;
    std::vector<void*> branches(nh, nullptr);
    auto cleanup = [&]() {
        for (int i = 0; i < nh; ++i) {
            if (fp64) delete static_cast<GraphBranch<double>*>(branches[i]);
            else delete static_cast<GraphBranch<float>*>(branches[i]);
        }
    };
    for (int i = 0; i < nh; ++i) {
        if (fp64) branches[i] = new GraphBranch<double>(handles[i], o, workspaces[i], X[i], loop_cap);
        else branches[i] = new GraphBranch<float>(handles[i], o, workspaces[i], X[i], loop_cap);
    }
    // one capture: the origin stream forks into one stream per branch and joins them
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins(nh, nullptr);
    int rc = SBEC_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
        rc = SBEC_ERR_CUDA;
    for (int i = 0; i < nh && !rc; ++i)
        if (cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming) != cudaSuccess) rc = SBEC_ERR_CUDA;
    // the handles' streams finish their pending work before the graph starts
    for (int i = 0; i < nh && !rc; ++i)
        if (cudaStreamSynchronize(handles[i]->stream) != cudaSuccess) rc = SBEC_ERR_CUDA;
    if (!rc && cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = SBEC_ERR_CUDA;
    bool capturing = !rc;
    if (!rc && cudaEventRecord(fork, origin) != cudaSuccess) rc = SBEC_ERR_CUDA;
    for (int i = 0; i < nh && !rc; ++i) {
        cudaStream_t s0 = fp64 ? static_cast<GraphBranch<double>*>(branches[i])->st[0]
                               : static_cast<GraphBranch<float>*>(branches[i])->st[0];
        if (cudaStreamWaitEvent(s0, fork, 0) != cudaSuccess) { rc = SBEC_ERR_CUDA; break; }
        rc = fp64 ? static_cast<GraphBranch<double>*>(branches[i])->build()
                  : static_cast<GraphBranch<float>*>(branches[i])->build();
        if (!rc && (cudaEventRecord(joins[i], s0) != cudaSuccess || cudaStreamWaitEvent(origin, joins[i], 0) != cudaSuccess))
            rc = SBEC_ERR_CUDA;
    }
    if (capturing) {
        const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
        if (!rc && ce != cudaSuccess) rc = SBEC_ERR_CUDA;
    }
    cudaGetLastError();
    if (!rc && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = SBEC_ERR_CUDA;
    if (!rc && (cudaGraphLaunch(exec, origin) != cudaSuccess || cudaStreamSynchronize(origin) != cudaSuccess))
        rc = SBEC_ERR_CUDA;
    // results: one read of every handle's scalar blocks
    int out = rc;
    for (int i = 0; i < nh && !rc; ++i) {
        sbec_handle* h = handles[i];
        if (sbec_read_scalars(h) == SBEC_ERR_CUDA) { out = SBEC_ERR_CUDA; break; }
        const double tol = o.tol;
        bool all = true;
        for (int b = 0; b < h->B; ++b) {
            const double* sc = h->h_scal + (size_t)b * sbec::S_COUNT;
            sbec_stats& s = stats[i][b];
            memset(&s, 0, sizeof(s));
            s.energy = sc[SBEC_S_ENERGY];
            s.grad_norm = sqrt(sc[SBEC_S_RGRAD_NORM2]);
            s.outer_iters = (long long)sc[DS_OUTER];
            s.inner_iters = (long long)sc[DS_INNER];
            s.rgbb_iters = (long long)sc[DS_RGBBIT];
            s.n_grad = (long long)sc[DS_NGRAD];
            s.n_energy = (long long)sc[DS_NENERGY];
            s.n_hvp = (long long)sc[DS_NHVP];
            s.converged = s.grad_norm <= tol;
            all = all && s.converged;
            const int e = (int)sc[DS_ERR];
            if (e && (out == SBEC_OK || out == SBEC_ERR_NOCONV)) out = e;
        }
        if (!all && out == SBEC_OK) out = SBEC_ERR_NOCONV;
        if (clear_skip(h) && out == SBEC_OK) out = SBEC_ERR_CUDA;
        h->last_grad_X = nullptr;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : joins)
        if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
    cleanup();
    cudaGetLastError();
    return out;
}
