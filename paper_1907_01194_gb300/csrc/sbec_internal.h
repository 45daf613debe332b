// Host-side internals shared by the C-ABI translation unit and the
// per-precision kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sbec.h"

namespace sbec {

// Spins the kernels are instantiated for: F = 1..kMaxF (C = 2F + 1 components)
constexpr int kMaxF = 4;
constexpr int kMaxC = 2 * kMaxF + 1;
// Real values per grid point of the densities a Hessian epilogue reads (Sec. 2):
// rho, F_z, F_+ (2), and for F = 2, 4 the singlet amplitude A00 (2), for F = 3
// A00 and the five quintet amplitudes A_{2l} (2 each)
__host__ __device__ constexpr int dens_count(int F) { return F == 1 ? 4 : F == 3 ? 16 : 6; }
// sbec_tune s_split value that selects the TMA strided pass (FP32, one instance),
// its tile width being s_pencils (8, 16 or 32 columns)
constexpr int kTmaSplit = 16;

// device scalar-block slots beyond the public SBEC_S_* ones
enum {
    S_C2 = 7,          // u^T Gamma^2 u
    S_PA = 8,          // projection coefficient alpha_w (Lemma 4.1) of the latest projection
    S_PB = 9,          // projection coefficient beta_w
    S_NORM2 = 10,      // scratch squared norm
    S_XFORM = 11,      // reserved
    S_SKIP = 12,       // nonzero: every kernel leaves this instance of a batch untouched
    S_TICKET = 13,     // blocks of the running launch that have stored their partials
    S_SIG = 16,        // kMaxC retraction scales sigma_l (component index order)
    S_SOLVER = 32,     // solver scalars start here
    S_COUNT = 128
};
static_assert(S_SIG + kMaxC <= S_SOLVER, "retraction scales overlap the solver slots");

// Physical parameters handed to the pointwise code (precomputed on the host).
struct PointParams {
    double bz[kMaxC];       // Zeeman diagonal b_l = -p l + q l^2 per component index
    double g0, g1, g2, g3;  // 2 beta_i / dV (gradient / Hessian prefactors)
    double e0, e1, e2, e3;  // beta_i / (2 dV) (energy prefactors)
};

// Launch shapes of the passes (0 = the built-in choice); set by the autotuner
// (sbec_autotune) or sbec_set_tune, checked by Ops<T>::tune_ok before use.
struct Tune {
    int x_rows;        // grid rows per block of the x pass
    int s_pencils[3];  // pencils per tile of the strided pass along axis 1, 2 ([0] unused)
    int s_split[3];    // butterfly items per thread of the strided pass (1, 2, 4, 8)
    int elem_per_sm;   // blocks per SM (whole GPU, all instances) of the grid-stride kernels
};

// Geometry and parameters of one problem as the kernels see it.
struct Geom {
    int F, C, dim;
    int n[3], logn[3];
    long long G;
    double dV, invG, M;
    // device tables
    const void* tw[3];        // twiddles per axis, T2 (precision of the handle)
    const double* lam2[3];    // lambda_p^2 per axis in DFT index order
    const void* k2s[3];       // lambda_p^2 / G per axis, T (precision of the handle)
    const void* V;            // potential, T
    double bz[kMaxC];
    double g0, g1, g2, g3, e0, e1, e2, e3;
    // batches: B instances of one shape stored [B][C][G] (V: [B][G]); per-instance
    // point parameters (beta) and magnetisations on the device, or null when B = 1
    int B;
    const void* ppb;          // PointParams[B]
    const double* Mb;         // M[B]
    const double* skip;       // the handle's scalar blocks: S_SKIP != 0 switches an instance off
    // instances a launch covers: nl of them, listed in imap (device, launch slot ->
    // instance), or all B when imap is null (nl = B)
    int nl;
    const int* imap;
    Tune tune;
};

// Kernel identities for the per-kernel launch counter and event timer.
enum KernelId {
    K_X_FWD, K_X_FWD_EPW, K_X_INV_GRAD, K_X_INV_HESS, K_X_FULL_GRAD, K_X_FULL_ENERGY, K_X_FULL_HESS,
    K_S_FWD, K_S_INV, K_S_K2, K_S_PARSEVAL, K_DOT, K_PROJ, K_RETW, K_SCALE, K_FIN, K_TABLES,
    K_LIN, K_PROLONG, K_X_INV, K_COUNT
};

// Launch bookkeeping of one handle: every library kernel launch is counted;
// while enabled, CUDA events are recorded around each launch on its stream so
// that per-kernel device time can be read back (sbec_profile_read).
struct Prof {
    int enabled;
    long long launches;
    int nrec, cap;
    cudaEvent_t* ev;     // 2 * cap events
    int* kid;            // cap kernel ids
    double ms[K_COUNT];
    long long cnt[K_COUNT];
};

void prof_begin(Prof* p, int kid, cudaStream_t s);
void prof_end(Prof* p, cudaStream_t s);

struct ProfScope {
    Prof* p;
    cudaStream_t s;
    ProfScope(Prof* p_, int kid, cudaStream_t s_) : p(p_), s(s_) { prof_begin(p, kid, s); }
    ~ProfScope() { prof_end(p, s); }
};

struct Work {
    void* work;        // C*G complex T: FFT intermediate
    void* work2;       // C*G complex T: projected directions / gradients
    double* partA;     // per-block partials
    double* partB;
    size_t part_cap;   // doubles in each of partA / partB
    double* scal;      // device scalar block (S_COUNT doubles)
    // FP64 handles in 2D and 3D: the densities of the latest gradient, dens_count(F)
    // planes of G doubles per instance ([B][q][G]), written by the gradient epilogue
    // and read by the Hessian epilogues at the same state; null otherwise
    double* dens;
    int num_sms;
    Prof* prof;
};

// out = (ca * scal[ia]) A + (cb * scal[ib]) B over the 2 C G reals of a field, with
// optional fused dots <out, D1>, <out, D2>; skipped (out left as is, dots of the
// old out) when scal[guard] == 0.
struct Lin {
    void* out;
    const void* A;
    const void* B;
    double ca, cb;
    int ia, ib;
    int ineg;
    const void* D1;
    const void* D2;
    int guard;
};

// Scalar-block slots of the modified CG (the solver's layout), for the fused CG kernels:
// kap, kap + 1 = <p,Hp>, <p,p>; alpha, alpha + 1 = the step and its guard; rr_now /
// rr_next = <r,r> before / after the update; beta, j, stop, maxin, cg, sest, cgneg, cghd
// as the solver documents them; skip_val = the S_SKIP value of an instance whose CG ended.
struct CgSlots {
    int kap, alpha, rr_now, rr_next, beta, j, stop, maxin, cg, sest, cgneg, cghd;
    double skip_val;
};

// per-precision entry points (implemented in sbec_kernels_f64.cu / _f32.cu)
template <typename T> struct Ops {
    static int lincomb(const Geom& g, const Work& w, const Lin& L, int dot_slot, cudaStream_t s);
    static int dot2(const Geom& g, const Work& w, const void* A, const void* B, const void* C, const void* D,
                    int slot, cudaStream_t s);
    static int bbdots(const Geom& g, const Work& w, const void* U, const void* UP, const void* Gv, const void* GP,
                      int slot, cudaStream_t s);
    static int ratio(const Geom& g, const Work& w, int dst, int num, int den, int guard_kap, int guard_pp,
                     double eps, cudaStream_t s, int mask = -1);
    // one modified-CG iteration after Hp = Hess p: cg_curv stores <p,Hp>, <p,p> and the
    // guarded step alpha = <r,r> / <p,Hp>; cg_update applies x += alpha p, r -= alpha Hp,
    // stores <r,r> and runs the CG control (iteration count, stopping tests, beta)
    static int cg_curv(const Geom& g, const Work& w, const void* p, const void* Hp, const CgSlots& cs,
                       cudaStream_t s);
    static int cg_update(const Geom& g, const Work& w, void* x, void* r, const void* p, const void* Hp,
                         const CgSlots& cs, cudaStream_t s);
    static int energy(const Geom& g, const Work& w, const void* X, cudaStream_t s);
    static int grad(const Geom& g, const Work& w, const void* X, void* Geuc, void* Griem, bool want_norm,
                    cudaStream_t s);
    // sigslot / tslot >= 0: sigma / t multiplied by each instance's scalar-block slot;
    // dens: the latest grad on w was at X (X unchanged since), so the Hessian epilogue
    // may read the densities it stored in w.dens instead of forming them again
    static int hessvec(const Geom& g, const Work& w, const void* X, const void* Z, double sigma, int riem,
                       void* HZ, cudaStream_t s, int sigslot = -1, bool dens = false);
    static int retract(const Geom& g, const Work& w, const void* U, const void* Xi, double t, int kind,
                       void* out, cudaStream_t s, int tslot = -1);
    static int prolongate(const Geom& gc, const Work& wc, const void* Xc, const Geom& gf, const Work& wf,
                          void* Xf, cudaStream_t s);
    static int init_tables(Geom& g, void* tw_storage, cudaStream_t s);
    static int harmonic_potential(const Geom& g, void* V, const double* lo, const double* hi, cudaStream_t s);
    static int convert_potential(const Geom& g, void* V, const double* Vd, cudaStream_t s);
    // partial-sum slots for the shapes of g.tune, or (any_shape) for every
    // shape tune_ok accepts
    static size_t partials_needed(const Geom& g, int num_sms, bool any_shape = true);
    // t is a valid set of launch shapes for g (0 fields: built-in choice)
    static bool tune_ok(const Geom& g, const Tune& t);
    // the launch shapes g resolves to (built-in choices filled in)
    static Tune resolved(const Geom& g, int num_sms);
};

}  // namespace sbec
