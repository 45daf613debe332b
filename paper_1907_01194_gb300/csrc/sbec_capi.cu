// libsbec C ABI: handle management, argument checking, host/device staging and
// dispatch to the per-precision kernel orchestration.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "sbec.h"
#include "sbec_internal.h"

#include "sbec_handle.h"

namespace sbec {

void prof_begin(Prof* p, int kid, cudaStream_t s) {
    if (!p) return;
    ++p->launches;
    if (p->enabled && p->nrec < p->cap) {
        cudaEventRecord(p->ev[2 * p->nrec], s);
        p->kid[p->nrec] = kid;
    }
}

void prof_end(Prof* p, cudaStream_t s) {
    if (!p) return;
    if (p->enabled && p->nrec < p->cap) {
        cudaEventRecord(p->ev[2 * p->nrec + 1], s);
        ++p->nrec;
    }
}

}  // namespace sbec

namespace {

bool is_pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }
int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

#define TRY_CUDA(expr)                                          \
    do {                                                        \
        if ((expr) != cudaSuccess) { cudaGetLastError(); return SBEC_ERR_CUDA; } \
    } while (0)

int read_scalars(sbec_handle* h) {
    const size_t n = (size_t)h->B * sbec::S_COUNT;
    TRY_CUDA(cudaMemcpyAsync(h->h_scal, h->work.scal, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TRY_CUDA(cudaStreamSynchronize(h->stream));
    int st = 0;
    for (int b = 0; b < h->B; ++b) {
        double& v = h->h_scal[(size_t)b * sbec::S_COUNT + SBEC_S_STATUS];
        if (v != 0.0 && st == 0) st = (int)v;
    }
    if (st != 0) {
        // clear every instance's status: write the (now synchronised) block back with zeros there
        for (int b = 0; b < h->B; ++b) h->h_scal[(size_t)b * sbec::S_COUNT + SBEC_S_STATUS] = 0.0;
        TRY_CUDA(cudaMemcpyAsync(h->work.scal, h->h_scal, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        TRY_CUDA(cudaStreamSynchronize(h->stream));
    }
    return st;
}

// Page-locked host arrays up to this size are read in place by the kernels over
// the CPU-GPU link (for a few KB that costs less than a staging copy and its
// wait); larger ones are copied once, since several passes read each input again
// (measured end to end through the C ABI: 12 KB arrays 7% faster in place, 5 MB
// arrays 9% slower).
constexpr size_t kInPlaceHostBytes = size_t(1) << 20;

// Resolve an input array: device pointers pass through; host arrays are read in
// place (page-locked and small) or copied into staging buffer `slot`.
// reuse (slot 0 only): the caller's contract says p's contents are those stage[0]
// received from p last (sbec_hessvec at the X of the latest sbec_grad), so that
// copy is not repeated
int stage_in(sbec_handle* h, const void* p, int slot, const void** out, bool* host, bool reuse = false) {
    if (!p) { *out = nullptr; return SBEC_ERR_ARG; }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
        attr.devicePointer = nullptr;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) { *out = p; return SBEC_OK; }
    *host = true;
    if (attr.type == cudaMemoryTypeHost && attr.devicePointer && h->field_bytes <= kInPlaceHostBytes) {
        *out = attr.devicePointer;
        return SBEC_OK;
    }
    if (slot == 0) {
        if (reuse && p == h->stage0_src) { *out = h->stage[0]; return SBEC_OK; }
        h->stage0_src = nullptr;
    }
    TRY_CUDA(cudaMemcpyAsync(h->stage[slot], p, h->field_bytes, cudaMemcpyHostToDevice, h->stream));
    if (slot == 0) h->stage0_src = p;
    *out = h->stage[slot];
    return SBEC_OK;
}

void* stage_out_ptr(sbec_handle* h, void* p, int slot, bool* host) {
    if (!p) return nullptr;
    if (is_device_ptr(p)) return p;
    *host = true;
    return h->stage[slot];
}

}  // namespace

int sbec_read_scalars(sbec_handle* h) { return read_scalars(h); }
bool sbec_is_device_ptr(const void* p) { return is_device_ptr(p); }

namespace {

int copy_back(sbec_handle* h, void* user, void* dev) {
    if (user && user != dev) TRY_CUDA(cudaMemcpyAsync(user, dev, h->field_bytes, cudaMemcpyDeviceToHost, h->stream));
    return SBEC_OK;
}

void free_handle(sbec_handle* h) {
    if (!h) return;
    cudaFree(h->d_tw);
    cudaFree(h->d_lam2);
    cudaFree(h->d_V);
    cudaFree(h->work.work);
    cudaFree(h->work.work2);
    cudaFree(h->work.partA);
    cudaFree(h->work.partB);
    cudaFree(h->work.scal);
    cudaFree(h->work.dens);
    cudaFree(h->d_ppb);
    cudaFree(h->d_Mb);
    cudaFree(h->d_imap);
    if (h->h_imap) cudaFreeHost(h->h_imap);
    for (int i = 0; i < 3; ++i) cudaFree(h->stage[i]);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->prof.ev) {
        for (int i = 0; i < 2 * h->prof.cap; ++i) cudaEventDestroy(h->prof.ev[i]);
        free(h->prof.ev);
        free(h->prof.kid);
    }
    free(h);
}

}  // namespace

extern "C" {

const char* sbec_status_string(int s) {
    switch (s) {
        case SBEC_OK: return "ok";
        case SBEC_ERR_ARG: return "invalid argument";
        case SBEC_ERR_DOMAIN: return "point outside the domain of the retraction or projection";
        case SBEC_ERR_NONFINITE: return "non-finite value in a reduction";
        case SBEC_ERR_CUDA: return "CUDA runtime error";
        case SBEC_ERR_TIMEOUT: return "bounded device wait expired";
        case SBEC_ERR_NOCONV: return "iteration cap reached before the tolerance";
        default: return "unknown status";
    }
}

}  // extern "C"

namespace {

// one problem (B = 1) or a batch of B problems that share spin, grid, box, Zeeman
// terms and precision and differ in beta and M
int create_impl(const sbec_problem* probs, int B, const double* V, void* cuda_stream, sbec_handle** out) {
    if (!probs || !out || B < 1) return SBEC_ERR_ARG;
    *out = nullptr;
    const sbec_problem& P = probs[0];
    if (P.F < 1 || P.F > sbec::kMaxF || P.dim < 1 || P.dim > 3) return SBEC_ERR_ARG;
    if (P.precision != SBEC_FP64 && P.precision != SBEC_MIXED) return SBEC_ERR_ARG;
    for (int ax = 0; ax < 3; ++ax) {
        if (ax < P.dim) {
            if (!is_pow2(P.n[ax]) || P.n[ax] < 2 || P.n[ax] > 1024) return SBEC_ERR_ARG;
            if (!(P.hi[ax] > P.lo[ax])) return SBEC_ERR_ARG;
        } else if (P.n[ax] != 1) {
            return SBEC_ERR_ARG;
        }
    }
    for (int b = 0; b < B; ++b) {
        const sbec_problem& Q = probs[b];
        if (!(fabs(Q.M) < (double)P.F)) return SBEC_ERR_ARG;
        if (Q.F != P.F || Q.dim != P.dim || Q.precision != P.precision || Q.p != P.p || Q.q != P.q) return SBEC_ERR_ARG;
        for (int ax = 0; ax < 3; ++ax)
            if (Q.n[ax] != P.n[ax] || Q.lo[ax] != P.lo[ax] || Q.hi[ax] != P.hi[ax]) return SBEC_ERR_ARG;
    }
    sbec_handle* h = (sbec_handle*)calloc(1, sizeof(sbec_handle));
    if (!h) return SBEC_ERR_CUDA;
    h->prob = P;
    h->B = B;
    h->stream = (cudaStream_t)cuda_stream;
    h->work.prof = &h->prof;
    if (cudaGetDevice(&h->device) != cudaSuccess) { free(h); return SBEC_ERR_CUDA; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->work.num_sms = sms > 0 ? sms : 1;

    sbec::Geom& g = h->geom;
    g.F = P.F; g.C = 2 * P.F + 1; g.dim = P.dim;
    g.B = B;
    g.nl = B;          // launches cover the whole batch unless a solve narrows them
    g.imap = nullptr;
    double dV = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        g.n[ax] = P.n[ax];
        g.logn[ax] = ilog2(P.n[ax]);
        if (ax < P.dim) dV *= (P.hi[ax] - P.lo[ax]) / P.n[ax];
    }
    g.G = (long long)P.n[0] * P.n[1] * P.n[2];
    g.dV = dV;
    g.invG = 1.0 / (double)g.G;
    g.M = P.M;
    for (int i = 0; i < sbec::kMaxC; ++i) {
        const double l = (double)(P.F - i);
        g.bz[i] = (i < g.C) ? (-P.p * l + P.q * l * l) : 0.0;
    }
    // point parameters: beta_i / (2 dV) (energy) and 2 beta_i / dV (gradient, Hessian)
    auto params = [&](const sbec_problem& Q, sbec::PointParams& pp) {
        const double b0 = Q.beta[0], b1 = Q.beta[1];
        const double b2 = Q.F >= 2 ? Q.beta[2] : 0.0, b3 = Q.F == 3 ? Q.beta[3] : 0.0;
        for (int i = 0; i < sbec::kMaxC; ++i) pp.bz[i] = g.bz[i];
        pp.g0 = 2 * b0 / dV; pp.g1 = 2 * b1 / dV; pp.g2 = 2 * b2 / dV; pp.g3 = 2 * b3 / dV;
        pp.e0 = b0 / (2 * dV); pp.e1 = b1 / (2 * dV); pp.e2 = b2 / (2 * dV); pp.e3 = b3 / (2 * dV);
    };
    sbec::PointParams pp0;
    params(P, pp0);
    g.g0 = pp0.g0; g.g1 = pp0.g1; g.g2 = pp0.g2; g.g3 = pp0.g3;
    g.e0 = pp0.e0; g.e1 = pp0.e1; g.e2 = pp0.e2; g.e3 = pp0.e3;

    const bool dbl = P.precision == SBEC_FP64;
    h->elem = dbl ? 2 * sizeof(double) : 2 * sizeof(float);
    h->field_bytes = (size_t)B * (size_t)g.C * (size_t)g.G * h->elem;
    const size_t real_bytes = dbl ? sizeof(double) : sizeof(float);
    const size_t ntw = (size_t)P.n[0] + P.n[1] + P.n[2];
    const size_t part = dbl ? sbec::Ops<double>::partials_needed(g, h->work.num_sms)
                            : sbec::Ops<float>::partials_needed(g, h->work.num_sms);
    h->work.part_cap = part;
    const size_t nscal = (size_t)B * sbec::S_COUNT;

    bool ok = true;
    ok = ok && cudaMalloc(&h->d_tw, ntw * h->elem) == cudaSuccess;
    // lambda^2 (double) followed by lambda^2 / G in the handle's precision
    ok = ok && cudaMalloc((void**)&h->d_lam2, ntw * (sizeof(double) + real_bytes)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->d_V, (size_t)B * g.G * real_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&h->work.work, h->field_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&h->work.work2, h->field_bytes) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&h->work.partA, part * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&h->work.partB, part * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&h->work.scal, nscal * sizeof(double)) == cudaSuccess;
    if (dbl && g.dim >= 2)
        ok = ok && cudaMalloc((void**)&h->work.dens, (size_t)B * sbec::dens_count(g.F) * g.G * sizeof(double)) ==
                       cudaSuccess;
    for (int i = 0; i < 3; ++i) ok = ok && cudaMalloc(&h->stage[i], h->field_bytes) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&h->h_scal, nscal * sizeof(double)) == cudaSuccess;
    if (ok && B > 1) {
        ok = cudaMalloc(&h->d_ppb, (size_t)B * sizeof(sbec::PointParams)) == cudaSuccess &&
             cudaMalloc((void**)&h->d_Mb, (size_t)B * sizeof(double)) == cudaSuccess &&
             cudaMalloc((void**)&h->d_imap, (size_t)B * sizeof(int)) == cudaSuccess &&
             cudaMallocHost((void**)&h->h_imap, (size_t)B * sizeof(int)) == cudaSuccess;
    }
    if (!ok) { cudaGetLastError(); free_handle(h); return SBEC_ERR_CUDA; }

    // lambda_p^2 = (2 pi p / (b - a))^2 with p the signed DFT frequency (Eq. 3.6);
    // per-instance parameters of a batch
    const size_t tab_bytes = ntw * (sizeof(double) + real_bytes);
    const size_t par_off = (tab_bytes + 15) & ~size_t(15);      // batch parameters, 16-byte aligned
    const size_t host_bytes = par_off + (B > 1 ? (size_t)B * (sizeof(sbec::PointParams) + sizeof(double)) : 0);
    char* hostbuf = (char*)malloc(host_bytes);
    if (!hostbuf) { free_handle(h); return SBEC_ERR_CUDA; }
    double* lam = (double*)hostbuf;
    size_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        const int n = P.n[ax];
        for (int j = 0; j < n; ++j) {
            const int p = (j < n / 2) ? j : j - n;
            const double L = (ax < P.dim) ? (P.hi[ax] - P.lo[ax]) : 1.0;
            const double lamp = (n > 1) ? 2.0 * M_PI * (double)p / L : 0.0;
            lam[off + j] = lamp * lamp;
        }
        g.lam2[ax] = h->d_lam2 + off;
        off += n;
    }
    // |k|^2 / G tables of the pass precision: the FP32 passes scale and sum the
    // kinetic term with FP32 arithmetic only
    char* k2s = hostbuf + ntw * sizeof(double);
    char* d_k2s = reinterpret_cast<char*>(h->d_lam2 + ntw);
    for (int ax = 0, o = 0; ax < 3; ++ax) {
        g.k2s[ax] = d_k2s + (size_t)o * real_bytes;
        for (int j = 0; j < P.n[ax]; ++j, ++o) {
            const double v = lam[o] * g.invG;
            if (dbl) reinterpret_cast<double*>(k2s)[o] = v;
            else reinterpret_cast<float*>(k2s)[o] = (float)v;
        }
    }
    cudaError_t ce = cudaMemcpyAsync(h->d_lam2, lam, tab_bytes, cudaMemcpyHostToDevice, h->stream);
    if (B > 1 && ce == cudaSuccess) {
        sbec::PointParams* ppb = (sbec::PointParams*)(hostbuf + par_off);
        double* Mb = (double*)(ppb + B);
        for (int b = 0; b < B; ++b) { params(probs[b], ppb[b]); Mb[b] = probs[b].M; }
        ce = cudaMemcpyAsync(h->d_ppb, ppb, (size_t)B * sizeof(sbec::PointParams), cudaMemcpyHostToDevice, h->stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(h->d_Mb, Mb, (size_t)B * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        g.ppb = h->d_ppb;
        g.Mb = h->d_Mb;
    }
    g.skip = h->work.scal;
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    free(hostbuf);
    if (ce != cudaSuccess) { cudaGetLastError(); free_handle(h); return SBEC_ERR_CUDA; }
    if (cudaMemsetAsync(h->work.scal, 0, nscal * sizeof(double), h->stream) != cudaSuccess) {
        free_handle(h);
        return SBEC_ERR_CUDA;
    }

    g.V = h->d_V;
    int st = dbl ? sbec::Ops<double>::init_tables(g, h->d_tw, h->stream)
                 : sbec::Ops<float>::init_tables(g, h->d_tw, h->stream);
    const double* Vd = V;
    if (st == SBEC_OK && V != nullptr && !is_device_ptr(V)) {
        // the caller's potential goes through a staging field (B G doubles fit in it)
        if (cudaMemcpyAsync(h->stage[0], V, (size_t)B * g.G * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess) st = SBEC_ERR_CUDA;
        Vd = (const double*)h->stage[0];
    }
    for (int b = 0; b < B && st == SBEC_OK; ++b) {
        void* Vb = (char*)h->d_V + (size_t)b * g.G * real_bytes;
        if (V == nullptr) {
            st = dbl ? sbec::Ops<double>::harmonic_potential(g, Vb, P.lo, P.hi, h->stream)
                     : sbec::Ops<float>::harmonic_potential(g, Vb, P.lo, P.hi, h->stream);
        } else {
            st = dbl ? sbec::Ops<double>::convert_potential(g, Vb, Vd + (size_t)b * g.G, h->stream)
                     : sbec::Ops<float>::convert_potential(g, Vb, Vd + (size_t)b * g.G, h->stream);
        }
    }
    if (st == SBEC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = SBEC_ERR_CUDA;
    if (st != SBEC_OK) { cudaGetLastError(); free_handle(h); return st; }
    *out = h;
    return SBEC_OK;
}

}  // namespace

extern "C" {

int sbec_create(const sbec_problem* prob, const double* V, void* cuda_stream, sbec_handle** out) {
    return create_impl(prob, 1, V, cuda_stream, out);
}

int sbec_create_batch(const sbec_problem* probs, int count, const double* V, void* cuda_stream, sbec_handle** out) {
    return create_impl(probs, count, V, cuda_stream, out);
}

int sbec_batch_size(const sbec_handle* h) { return h ? h->B : 0; }

int sbec_destroy(sbec_handle* h) {
    if (!h) return SBEC_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    free_handle(h);
    return SBEC_OK;
}

int sbec_sync(sbec_handle* h) {
    if (!h) return SBEC_ERR_ARG;
    return read_scalars(h);
}

const double* sbec_scalars(const sbec_handle* h) { return h ? h->work.scal : nullptr; }

long long sbec_launch_count(const sbec_handle* h) { return h ? h->prof.launches : -1; }

static const char* kKernelNames[sbec::K_COUNT] = {
    "x_fwd", "x_fwd_energy", "x_inv_grad", "x_inv_hess", "x_full_grad", "x_full_energy", "x_full_hess",
    "s_fwd", "s_inv", "s_k2", "s_parseval", "dot_reduce", "proj_apply", "retract_w", "scale", "finalize",
    "tables", "lincomb", "prolong", "x_inv"};

int sbec_profile(sbec_handle* h, int enable) {
    if (!h) return SBEC_ERR_ARG;
    sbec::Prof& p = h->prof;
    if (enable && !p.ev) {
        p.cap = 16384;
        p.ev = (cudaEvent_t*)calloc(2 * p.cap, sizeof(cudaEvent_t));
        p.kid = (int*)calloc(p.cap, sizeof(int));
        if (!p.ev || !p.kid) return SBEC_ERR_CUDA;
        for (int i = 0; i < 2 * p.cap; ++i) TRY_CUDA(cudaEventCreate(&p.ev[i]));
    }
    if (enable) {
        p.nrec = 0;
        for (int k = 0; k < sbec::K_COUNT; ++k) { p.ms[k] = 0.0; p.cnt[k] = 0; }
    }
    p.enabled = enable ? 1 : 0;
    return SBEC_OK;
}

int sbec_profile_read(sbec_handle* h, int max, char* names, double* ms, long long* counts, int* rows) {
    if (!h || !rows) return SBEC_ERR_ARG;
    sbec::Prof& p = h->prof;
    TRY_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < p.nrec; ++i) {
        float t = 0.f;
        TRY_CUDA(cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]));
        p.ms[p.kid[i]] += t;
        p.cnt[p.kid[i]] += 1;
    }
    p.nrec = 0;
    int r = 0;
    for (int k = 0; k < sbec::K_COUNT && r < max; ++k) {
        if (p.cnt[k] == 0) continue;
        if (names) { strncpy(names + 32 * r, kKernelNames[k], 31); names[32 * r + 31] = 0; }
        if (ms) ms[r] = p.ms[k];
        if (counts) counts[r] = p.cnt[k];
        ++r;
    }
    for (int k = 0; k < sbec::K_COUNT; ++k) { p.ms[k] = 0.0; p.cnt[k] = 0; }
    *rows = r;
    return SBEC_OK;
}

int sbec_energy(sbec_handle* h, const void* X, double* E) {
    if (!h || !X) return SBEC_ERR_ARG;
    bool host = false;
    const void* Xd;
    int st = stage_in(h, X, 0, &Xd, &host);
    if (st) return st;
    st = h->prob.precision == SBEC_FP64 ? sbec::Ops<double>::energy(h->geom, h->work, Xd, h->stream)
                                        : sbec::Ops<float>::energy(h->geom, h->work, Xd, h->stream);
    if (st) return st;
    if (E || host) {
        st = read_scalars(h);
        if (E)
            for (int b = 0; b < h->B; ++b) E[b] = h->h_scal[(size_t)b * sbec::S_COUNT + SBEC_S_ENERGY];
    }
    return st;
}

int sbec_grad(sbec_handle* h, const void* X, void* G_euc, void* G_riem, double* E, double* rgrad_norm) {
    if (!h || !X) return SBEC_ERR_ARG;
    bool host = false;
    const void* Xd;
    int st = stage_in(h, X, 0, &Xd, &host);
    if (st) return st;
    void* ge = stage_out_ptr(h, G_euc, 1, &host);
    void* gr = stage_out_ptr(h, G_riem, 2, &host);
    st = h->prob.precision == SBEC_FP64
             ? sbec::Ops<double>::grad(h->geom, h->work, Xd, ge, gr, rgrad_norm != nullptr, h->stream)
             : sbec::Ops<float>::grad(h->geom, h->work, Xd, ge, gr, rgrad_norm != nullptr, h->stream);
    if (st) return st;
    h->last_grad_X = X;     // host or device: the caller's pointer identifies the state
    if ((st = copy_back(h, G_euc, ge))) return st;
    if ((st = copy_back(h, G_riem, gr))) return st;
    if (E || rgrad_norm || host) {
        st = read_scalars(h);
        for (int b = 0; b < h->B; ++b) {
            const double* sc = h->h_scal + (size_t)b * sbec::S_COUNT;
            if (E) E[b] = sc[SBEC_S_ENERGY];
            if (rgrad_norm) rgrad_norm[b] = sqrt(sc[SBEC_S_RGRAD_NORM2]);
        }
    }
    return st;
}

int sbec_hessvec(sbec_handle* h, const void* X, const void* Z, double sigma, int riemannian, void* HZ) {
    if (!h || !X || !Z || !HZ) return SBEC_ERR_ARG;
    bool host = false;
    const void *Xd, *Zd;
    // X unchanged since the latest sbec_grad at the same pointer (the call's contract):
    // a host X staged by that call is still in stage[0] unless another call replaced it
    int st = stage_in(h, X, 0, &Xd, &host, h->last_grad_X == X);
    if (st) return st;
    st = stage_in(h, Z, 1, &Zd, &host);
    if (st) return st;
    void* hz = stage_out_ptr(h, HZ, 2, &host);
    const bool dbl = h->prob.precision == SBEC_FP64;
    if (riemannian && h->last_grad_X != X) {
        st = dbl ? sbec::Ops<double>::grad(h->geom, h->work, Xd, nullptr, nullptr, false, h->stream)
                 : sbec::Ops<float>::grad(h->geom, h->work, Xd, nullptr, nullptr, false, h->stream);
        if (st) return st;
        h->last_grad_X = X;
    }
    // the densities stored by the latest gradient are those of X when it was at X
    const bool dens = h->last_grad_X == X;
    st = dbl ? sbec::Ops<double>::hessvec(h->geom, h->work, Xd, Zd, sigma, riemannian, hz, h->stream, -1, dens)
             : sbec::Ops<float>::hessvec(h->geom, h->work, Xd, Zd, sigma, riemannian, hz, h->stream, -1, dens);
    if (st) return st;
    if ((st = copy_back(h, HZ, hz))) return st;
    if (host) st = read_scalars(h);
    return st;
}

int sbec_retract(sbec_handle* h, const void* U, const void* Xi, double t, int kind, void* out) {
    if (!h || !U || !Xi || !out || kind < 1 || kind > 3) return SBEC_ERR_ARG;
    bool host = false;
    const void *Ud, *Xd;
    int st = stage_in(h, U, 0, &Ud, &host);
    if (st) return st;
    st = stage_in(h, Xi, 1, &Xd, &host);
    if (st) return st;
    void* o = stage_out_ptr(h, out, 2, &host);
    st = h->prob.precision == SBEC_FP64
             ? sbec::Ops<double>::retract(h->geom, h->work, Ud, Xd, t, kind, o, h->stream)
             : sbec::Ops<float>::retract(h->geom, h->work, Ud, Xd, t, kind, o, h->stream);
    if (st) return st;
    if ((st = copy_back(h, out, o))) return st;
    if (host) st = read_scalars(h);
    return st;
}

}  // extern "C"
