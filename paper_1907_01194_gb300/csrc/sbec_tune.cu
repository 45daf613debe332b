// Autotuner of the launch shapes: the x-pass rows per block, the strided-pass
// tile width and butterfly split per axis, and the blocks per SM of the
// grid-stride kernels are chosen by timing the hot path itself (one
// energy+gradient evaluation plus one Riemannian Hessian-vector product) on the
// handle's problem, one field at a time.
#include <math.h>
#include <string.h>

#include <vector>

#include <cuda_runtime.h>

#include "sbec_handle.h"

namespace {

using sbec::Ops;
using sbec::Tune;

sbec_tune to_c(const Tune& t, double ms) {
    sbec_tune o;
    memset(&o, 0, sizeof(o));
    o.x_rows = t.x_rows;
    for (int a = 0; a < 3; ++a) { o.s_pencils[a] = t.s_pencils[a]; o.s_split[a] = t.s_split[a]; }
    o.elem_per_sm = t.elem_per_sm;
    o.ms = ms;
    return o;
}

Tune from_c(const sbec_tune& o) {
    Tune t{};
    t.x_rows = o.x_rows;
    for (int a = 0; a < 3; ++a) { t.s_pencils[a] = o.s_pencils[a]; t.s_split[a] = o.s_split[a]; }
    t.elem_per_sm = o.elem_per_sm;
    return t;
}

template <typename T>
struct Tuner {
    sbec_handle* h;
    const void* X;
    int reps;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    ~Tuner() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }

    // one untimed pair, then `r` timed pairs; ms per pair
    int measure(int r, double* ms) {
        const sbec::Geom& g = h->geom;
        const sbec::Work& w = h->work;
        cudaStream_t s = h->stream;
        for (int i = 0; i <= r; ++i) {
            if (i == 1 && cudaEventRecord(e0, s) != cudaSuccess) return SBEC_ERR_CUDA;
            int st = Ops<T>::grad(g, w, X, nullptr, h->stage[1], true, s);
            if (!st) st = Ops<T>::hessvec(g, w, X, h->stage[1], 0.0, 1, h->stage[2], s, -1, true);
            if (st) return st;
        }
        float t = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return SBEC_ERR_CUDA;
        *ms = (double)t / r;
        return SBEC_OK;
    }

    int run(sbec_tune* out) {
        sbec::Geom& g = h->geom;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SBEC_ERR_CUDA;
        Tune best = Ops<T>::resolved(g, h->work.num_sms);
        g.tune = best;
        double best_ms = 0.0;
        if (int st = measure(1, &best_ms)) return st;
        int r = reps;
        if (r <= 0) {
            r = best_ms > 0.0 ? (int)ceil(3.0 / best_ms) : 1;
            if (r < 1) r = 1;
            if (r > 200) r = 200;
        }
        if (int st = measure(r, &best_ms)) return st;

        // candidate values per field, in the struct's order
        const int rows[] = {1, 2, 4, 8, 16, 32, 64};
        const int pencils[] = {1, 2, 4, 8, 16, 32, 64};
        const int splits[] = {1, 2, 4, sbec::kTmaSplit};
        const int per_sm[] = {2, 4, 8, 16, 32};
        // field(t) is the member of t under trial
        auto try_field = [&](auto field, const int* cand, int nc) -> int {
            for (int i = 0; i < nc; ++i) {
                if (cand[i] == field(best)) continue;
                Tune t = best;
                field(t) = cand[i];
                if (!Ops<T>::tune_ok(g, t)) continue;
                g.tune = t;
                double ms = 0.0;
                const int st = measure(r, &ms);
                g.tune = best;
                if (st) return st;
                if (ms < 0.98 * best_ms) { best_ms = ms; best = t; g.tune = best; }
            }
            return SBEC_OK;
        };
        int st = try_field([](Tune& t) -> int& { return t.x_rows; }, rows, 7);
        for (int a = 1; a < g.dim && !st; ++a) {
            st = try_field([a](Tune& t) -> int& { return t.s_pencils[a]; }, pencils, 7);
            if (!st) st = try_field([a](Tune& t) -> int& { return t.s_split[a]; }, splits, 4);
        }
        if (!st) st = try_field([](Tune& t) -> int& { return t.elem_per_sm; }, per_sm, 5);
        if (st) return st;
        g.tune = best;
        if (out) *out = to_c(best, best_ms);
        return SBEC_OK;
    }
};

}  // namespace

extern "C" {

int sbec_autotune(sbec_handle* h, const void* X, int reps, sbec_tune* out) {
    if (!h || !X || reps < 0 || !sbec_is_device_ptr(X)) return SBEC_ERR_ARG;
    // timing runs unprofiled; the launches are still counted
    const int prof = h->prof.enabled;
    h->prof.enabled = 0;
    const Tune before = h->geom.tune;
    int st;
    if (h->prob.precision == SBEC_FP64) {
        Tuner<double> t{h, X, reps};
        st = t.run(out);
    } else {
        Tuner<float> t{h, X, reps};
        st = t.run(out);
    }
    h->prof.enabled = prof;
    h->last_grad_X = nullptr;
    if (st) {
        h->geom.tune = before;
        cudaStreamSynchronize(h->stream);
        cudaGetLastError();
        return st;
    }
    // the state may put the timing runs outside the domain: clear the statuses
    const int ds = sbec_read_scalars(h);
    return (ds == SBEC_ERR_CUDA) ? ds : SBEC_OK;
}

int sbec_set_tune(sbec_handle* h, const sbec_tune* t) {
    if (!h || !t) return SBEC_ERR_ARG;
    const Tune v = from_c(*t);
    const bool ok = h->prob.precision == SBEC_FP64 ? Ops<double>::tune_ok(h->geom, v) : Ops<float>::tune_ok(h->geom, v);
    if (!ok) return SBEC_ERR_ARG;
    h->geom.tune = v;
    return SBEC_OK;
}

int sbec_get_tune(const sbec_handle* h, sbec_tune* out) {
    if (!h || !out) return SBEC_ERR_ARG;
    const Tune t = h->prob.precision == SBEC_FP64 ? Ops<double>::resolved(h->geom, h->work.num_sms)
                                                  : Ops<float>::resolved(h->geom, h->work.num_sms);
    *out = to_c(t, 0.0);
    return SBEC_OK;
}

}  // extern "C"
