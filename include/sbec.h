/*
 * libsbec — C ABI of the GB300 (sm_103a) kernels for the spin-F BEC
 * ground-state problem of Tian, Cai, Wu & Wen, "Ground states and their
 * characterization of spin-F Bose-Einstein condensates" (arXiv:1907.01194).
 *
 * Problem (Sec. 3, Eq. minimize:discrete): minimise the Fourier-pseudospectral
 * Gross-Pitaevskii energy E_h(X) over X in C^{G x (2F+1)} subject to
 * tr(X^* X) = 1 and tr(X^* X D) = M, the manifold M of Sec. 4.
 *
 * State layout (all calls): X is the paper's scaled variable X = sqrt(dV) phi,
 * dV = prod_i h_i, stored component-major as [C][n_z][n_y][n_x] (x fastest),
 * components ordered l = F, F-1, ..., -F, interleaved complex: double2
 * (precision SBEC_FP64) or float2 (SBEC_MIXED).  Grid points are
 * x_j = lo + j (hi - lo) / n, j = 0..n-1, on each axis (Sec. 3).  n_i is a
 * power of two, 2 <= n_i <= 1024; missing axes of 1D/2D problems have n = 1.
 *
 * Pointers: every array argument may be a device pointer or a host pointer
 * (pageable or pinned); host arrays are staged through the handle's
 * workspace with copies on the handle's stream, except page-locked input
 * arrays of at most 1 MiB, which the kernels read in place over the CPU-GPU
 * link.  The caller owns all state
 * arrays; the library owns its workspace (allocated by sbec_create, freed by
 * sbec_destroy).  No other call allocates memory.
 *
 * Ordering and synchronisation: every call is ordered on the handle's stream.
 * A call that returns scalars through host pointers (non-NULL double* outputs)
 * or that reads/writes host arrays synchronises the stream before returning.
 * A call with only device arrays and NULL scalar outputs is asynchronous; its
 * scalar results stay in the handle's device scalar block (sbec_scalars) and
 * any device-side error is recorded there and reported by sbec_sync.
 *
 * Errors: every call returns SBEC_OK or one of the codes below; no call
 * aborts or throws across the ABI.
 */
#ifndef SBEC_H
#define SBEC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBEC_OK             0
#define SBEC_ERR_ARG        1  /* bad argument: |M| >= F, F not in {1,..,4}, bad n, NULL */
#define SBEC_ERR_DOMAIN     2  /* point outside the retraction's domain (Omega or S),
                                  u^T Gamma^2 u - M^2 <= 0, or root bracket failure */
#define SBEC_ERR_NONFINITE  3  /* NaN or Inf in a reduction */
#define SBEC_ERR_CUDA       4  /* a CUDA runtime call failed */
#define SBEC_ERR_TIMEOUT    5  /* a bounded device-side wait expired */
#define SBEC_ERR_NOCONV     6  /* solver hit its iteration cap; the state is still written */

#define SBEC_FP64   0          /* every step in double precision */
#define SBEC_MIXED  1          /* FFT and pointwise steps in float, reductions and
                                  retraction scalars in double (state is float2) */

/* Problem statement (Sec. 2-3).  beta[0..3] = (beta0, beta1, beta2, beta3):
 * density, spin, singlet (F >= 2) and quintet (F = 3) interaction strengths.
 * F = 4: the paper prints the energy for F <= 3 only; a spin-4 condensate is
 * modelled here with the density, spin and singlet-pair terms of the spin-2
 * form (angular-momentum matrices and singlet pair of spin 4; beta3 unused);
 * p, q: linear and quadratic Zeeman shifts (b_l = -p l + q l^2); M: the
 * magnetisation; lo/hi: the box per axis (x, y, z). */
typedef struct sbec_problem {
    int    F;            /* spin: 1, 2, 3 or 4 (C = 2F+1 components) */
    int    dim;          /* 1, 2 or 3 */
    int    n[3];         /* grid points per axis (x, y, z); unused axes: 1 */
    double lo[3], hi[3]; /* box per axis */
    double beta[4];
    double p, q;
    double M;
    int    precision;    /* SBEC_FP64 or SBEC_MIXED */
} sbec_problem;

typedef struct sbec_handle sbec_handle;

/* Create a handle for one problem on the calling thread's current device.
 * V: potential at the grid points, G doubles in [n_z][n_y][n_x] order (host or
 * device; copied), or NULL for the harmonic trap V = |x|^2 / 2.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Allocates the workspace (about 5 C G complex values plus V). */
int sbec_create(const sbec_problem* prob, const double* V, void* cuda_stream, sbec_handle** out);
int sbec_destroy(sbec_handle* h);

/* Batch handle: `count` problems that share F, dim, n, box, p, q and precision
 * and differ in beta and M.  Arrays of every call are then [count][C][G] (the
 * instances back to back, each in the state layout), V is [count][G] doubles or
 * NULL (harmonic), and host scalar outputs (E, rgrad_norm) receive `count`
 * values.  Every kernel launch covers all instances: blocks map to (instance,
 * tile) pairs, reductions and scalars are per instance. */
int sbec_create_batch(const sbec_problem* probs, int count, const double* V, void* cuda_stream,
                      sbec_handle** out);
int sbec_batch_size(const sbec_handle* h);

/* E_h(X), Eq. (3.7) with h -> dV.  E: host pointer or NULL (then the value is
 * left in the scalar block, slot SBEC_S_ENERGY). */
int sbec_energy(sbec_handle* h, const void* X, double* E);

/* Euclidean gradient nabla E_h(X) w.r.t. Re<.,.> (Eq. 3.12) into G_euc, and
 * the Riemannian gradient grad E = P_u nabla E (Eq. 4.6, Lemma 4.1) into
 * G_riem, with u the real stacking of X (Sec. 4).  Either output may be NULL.
 * E and rgrad_norm (||grad E||_2, the stopping norm of Sec. 7.1) are optional
 * host outputs.  The Lemma 4.1 coefficients are cached in the handle for the
 * next sbec_hessvec with riemannian != 0; FP64 handles in 2D and 3D also keep
 * the pointwise densities of X (rho, F_z, F_+, A00, A_2l; Sec. 2) for the
 * Hessian-vector products at the same X pointer. */
int sbec_grad(sbec_handle* h, const void* X, void* G_euc, void* G_riem, double* E,
              double* rgrad_norm);

/* Hessian-vector product.  riemannian == 0: HZ = nabla^2 E_h(X)[Z] + sigma Z
 * (Eq. 3.13).  riemannian != 0: HZ = Hess f(u)[xi] of Lemma 4.2 for
 * f = E + (sigma/2)||u - u_k||^2, i.e. P_u(nabla^2 E[xi] + sigma xi
 * - alpha_g xi - beta_g Gamma xi) with xi = P_u Z, using the alpha_g, beta_g
 * of the latest sbec_grad call at the same X pointer, host or device (the call
 * recomputes them when X differs from that call's pointer; after changing the
 * contents of X in place, call sbec_grad again).  Either form, at the X pointer
 * of the latest sbec_grad, reads the densities that call kept (FP64, 2D/3D)
 * instead of forming them again, and a host X that call staged is not copied
 * to the device again while no other call has used the staging field. */
int sbec_hessvec(sbec_handle* h, const void* X, const void* Z, double sigma, int riemannian,
                 void* HZ);

/* Retraction R_u(t xi) = psi(u + t xi) (Sec. 6, Eq. oretr0): kind 1 = projective
 * (Lemma 5.1), 2 = orthogonal (Lemma 5.3), 3 = closed form (Lemma 5.4).
 * out may alias U.  Returns SBEC_ERR_DOMAIN (synchronous calls) when u + t xi
 * is outside Omega (kinds 1, 2) or S (kind 3). */
int sbec_retract(sbec_handle* h, const void* U, const void* Xi, double t, int kind, void* out);

/* Ground-state solve (Sec. 5, Algorithm 1 on one mesh): the Riemannian
 * gradient method with BB step and nonmonotone search (RGBB) as a warm start,
 * then the adaptive regularised Newton method (ARNT) with the modified CG,
 * the curvilinear search and the sigma update of Sec. 7.1; or RGBB alone.
 * Readings where the paper is silent (constants of the modified CG and of the
 * searches) follow the library's design notes and match its CPU oracle. */
#define SBEC_ARNT 0
#define SBEC_RGBB 1

typedef struct sbec_solve_opts {
    int    method;           /* SBEC_ARNT (RGBB warm start, then ARNT) or SBEC_RGBB */
    int    retraction;       /* 1 (projective, the paper's choice), 2 or 3 */
    double tol;              /* stop when ||grad E||_2 <= tol (Sec. 7.1 uses 1e-6) */
    int    maxit;            /* iteration cap of the final method (Sec. 7.1: 10000) */
    double rgbb_tol;         /* warm-start tolerance inside ARNT (Sec. 7.1: 1e-2) */
    int    rgbb_maxit;       /* warm-start cap inside ARNT (Sec. 7.1: 2000) */
    int    project_initial;  /* 1: replace X by P_M(X) (Lemma 5.1) before iterating */
    int    cg_chunk;         /* modified-CG iterations run between two host reads of the
                                scalar block (>= 1; default 4).  The CG stopping tests run
                                on the device; an instance whose CG has ended leaves the
                                rest of its chunk untouched, so results do not depend on it */
    int    cuda_graphs;      /* 1 (default): every CG chunk is the replay of a CUDA graph
                                captured once per solve; 0: its kernels are launched one
                                by one.  Graphs are not used while sbec_profile is on */
    int    refine_cg_fp32;   /* sbec_solve_mixed on single handles: 1 (default): in the FP64
                                refinement the modified CG runs on the SBEC_MIXED handle
                                (FP32 Hessian-vector products at u rounded to float), while
                                the gradient, energy, model value, search, retraction and
                                the stopping test stay FP64; 0: every step in FP64.
                                Ignored by the other solvers */
} sbec_solve_opts;

typedef struct sbec_stats {
    double    energy;        /* E_h at the returned state */
    double    grad_norm;     /* ||grad E||_2 at the returned state */
    long long outer_iters;   /* ARNT (or RGBB-only) iterations */
    long long inner_iters;   /* modified-CG iterations in total */
    long long rgbb_iters;    /* RGBB iterations (warm start included) */
    long long n_grad, n_energy, n_hvp;
    int       converged;     /* grad_norm <= tol */
} sbec_stats;

/* Paper defaults: ARNT with R1, tol 1e-6, maxit 10000, RGBB warm start to 1e-2
 * or 2000 iterations, project_initial 1; cg_chunk 4, cuda_graphs 1,
 * refine_cg_fp32 1. */
void sbec_solve_defaults(sbec_solve_opts* opts);

/* Bytes of device workspace sbec_solve needs for the handle's problem (ten fields). */
int sbec_solve_workspace_bytes(const sbec_handle* h, size_t* bytes);

/* Minimise E_h over M from X (host or device array, overwritten with the
 * solution).  workspace: caller-owned device memory of at least
 * sbec_solve_workspace_bytes.  Returns SBEC_OK, SBEC_ERR_NOCONV (cap reached,
 * X holds the last iterate) or an error.  Synchronises the stream. */
int sbec_solve(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
               sbec_stats* stats);

/* sbec_solve for a batch handle: all instances iterate in lock step (one launch
 * per pass covers the batch); each instance takes the decisions sbec_solve
 * would take for it alone and stops when it converges.  X: device array of the
 * batch; stats: B entries.  Returns SBEC_ERR_NOCONV if any instance did not
 * reach the tolerance. */
int sbec_solve_batch(sbec_handle* h, void* X, const sbec_solve_opts* opts, void* workspace, size_t workspace_bytes,
                     sbec_stats* stats);

/* Device-driven solve (Algorithm 1 as one CUDA graph): the solve of every
 * instance of nh handles (single or batch handles of one precision on one
 * device, e.g. the grid-size classes of an uneven sweep), captured once and run
 * as ONE graph launch.  The decisions sbec_solve_batch takes on the host (RGBB
 * step and nonmonotone search, end of the modified CG, the direction of the
 * Newton step, the curvilinear search, the ratio test and the sigma update) are
 * taken per instance by one-block control kernels in the same formulas; the
 * loops are conditional WHILE nodes whose conditions those kernels set, and the
 * handles are parallel branches of the graph.  The host reads the scalar blocks
 * once, after the graph.  X[i]: device array of handle i (overwritten with its
 * ground states); workspaces[i]: at least sbec_solve_workspace_bytes of handle
 * i; stats[i]: B_i entries.  loop_cap: executions of any loop body of a branch
 * before the branch stops with SBEC_ERR_TIMEOUT (0: 10^6).  Returns SBEC_OK,
 * SBEC_ERR_NOCONV (some instance above the tolerance), SBEC_ERR_TIMEOUT or an
 * error.  Not available while sbec_profile is on (event timing cannot be
 * captured).  Synchronises the handles' streams. */
int sbec_solve_graph(sbec_handle* const* handles, int nh, void* const* X, const sbec_solve_opts* opts,
                     void* const* workspaces, const size_t* workspace_bytes, long long loop_cap,
                     sbec_stats* const* stats);

/* Mixed-precision solve with FP64 refinement: X (complex128, device) is cast to
 * float, solved on h32 (precision SBEC_MIXED, same problem and stream as h64)
 * to max(tol_mixed, opts->tol) or at most 300 iterations, cast back, projected
 * on M and refined on h64 (SBEC_FP64) to opts->tol.  Stats of both phases are
 * returned.  Batch handles
 * (the same instances in both) run both phases with sbec_solve_batch; the stats
 * arrays then have B entries.  workspace: device memory of at least
 * sbec_solve_mixed_workspace_bytes. */
int sbec_solve_mixed_workspace_bytes(const sbec_handle* h64, const sbec_handle* h32, size_t* bytes);
int sbec_solve_mixed(sbec_handle* h64, sbec_handle* h32, void* X, const sbec_solve_opts* opts, double tol_mixed,
                     void* workspace, size_t workspace_bytes, sbec_stats* st_mixed, sbec_stats* st_fp64);

/* Cascadic multigrid (Algorithm 1: solve on a coarse mesh, refine uniformly,
 * repeat).  sbec_prolongate maps a state of handle hc to the finer handle hf
 * (same spin, box, precision and stream; n_f >= n_c per axis): the coarse
 * spectrum is zero-padded (the coarse Nyquist coefficient split evenly between
 * +-n_c/2), transformed back, rescaled to keep X = sqrt(dV) phi and put on M
 * with R1 (Lemma 5.1).  sbec_solve_cascadic solves on levels[0..nlevels-1]
 * (coarse to fine) with X[j] the caller's state array of level j (X[0] holds
 * the initial data); coarse levels stop at max(tol_coarse, opts->tol)
 * (Sec. 7.1: 1e-5), the finest at opts->tol; stats are those of the finest
 * level.  workspace: at least sbec_solve_workspace_bytes of the finest handle. */
int sbec_prolongate(sbec_handle* hc, const void* Xc, sbec_handle* hf, void* Xf);
int sbec_solve_cascadic(sbec_handle* const* levels, int nlevels, void* const* X, const sbec_solve_opts* opts,
                        double tol_coarse, void* workspace, size_t workspace_bytes, sbec_stats* stats);

/* sbec_solve_cascadic with the mixed form on every level: levels64[j] (SBEC_FP64)
 * and levels32[j] (SBEC_MIXED) describe level j; each level runs
 * sbec_solve_mixed (tolerance max(tol_coarse, opts->tol) on coarse levels,
 * opts->tol on the finest) and its FP64 result is prolongated with
 * sbec_prolongate on the FP64 handles.  X[j]: complex128 device arrays.
 * workspace: at least sbec_solve_mixed_workspace_bytes of the finest pair.
 * Stats are those of the finest level's two phases. */
int sbec_solve_cascadic_mixed(sbec_handle* const* levels64, sbec_handle* const* levels32, int nlevels,
                              void* const* X, const sbec_solve_opts* opts, double tol_coarse, double tol_mixed,
                              void* workspace, size_t workspace_bytes, sbec_stats* st_mixed, sbec_stats* st_fp64);

/* Stream synchronisation; returns the first device-side error recorded since
 * the previous sbec_sync (and clears it), or SBEC_ERR_CUDA. */
int sbec_sync(sbec_handle* h);

/* Device pointer to the handle's scalar block (doubles, see SBEC_S_* slots). */
const double* sbec_scalars(const sbec_handle* h);

/* Launch shapes of the hot-path kernels (not in the paper: the paper's own
 * kernels are MATLAB's).  x_rows: grid rows (x lines, all C components) per
 * block of the x-axis FFT pass, a power of 2 dividing the rows of an
 * instance.  s_pencils[a], a = 1, 2: pencils (consecutive x columns) per
 * shared-memory tile of the FFT pass along axis a, a power of 2 <= n[0];
 * s_split[a]: butterflies per thread of that pass (1, 2, 4 or 8), or 16 for
 * the TMA pass (SBEC_MIXED handles of one instance, an axis of 128 or 256
 * points: tiles moved by cp.async.bulk.tensor, s_pencils[a] = 8, 16 or 32
 * columns per tile, n[0] a multiple of it; the built-in choice there, with
 * 8 columns on the last axis and 16 on the middle one of a 3D problem).
 * elem_per_sm: blocks per SM of the grid-stride elementwise and reduction
 * kernels (1..32); a kernel of which fewer blocks fit per SM gets whole waves
 * of the blocks that fit.  At most 16384 points per FFT block and 227 KB of shared
 * memory.  [0] entries and the entries of axes >= dim are 0.  In
 * sbec_set_tune a 0 field keeps the built-in choice. */
typedef struct sbec_tune {
    int    x_rows;
    int    s_pencils[3];
    int    s_split[3];
    int    elem_per_sm;
    double ms;     /* sbec_autotune: measured ms of one energy+gradient evaluation
                      plus one Riemannian Hessian-vector product; otherwise 0 */
} sbec_tune;

/* Autotuner: times one energy+gradient evaluation plus one Riemannian
 * Hessian-vector product at X (a device state of the handle, e.g. the initial
 * data; its values only need to be finite) with CUDA events on the handle's
 * stream, for each candidate of one field at a time (coordinate descent in the
 * order of the struct, starting from the built-in choices), keeps a candidate
 * that is more than 2% faster, and leaves the handle on the best shapes, which
 * it also writes to *out.  reps: timed repetitions per candidate (0: enough
 * for about 3 ms).  Uses the handle's staging arrays; synchronises the stream.
 * Results do not depend on the shapes beyond the order of the partial sums. */
int sbec_autotune(sbec_handle* h, const void* X, int reps, sbec_tune* out);
/* Set shapes (e.g. an earlier sbec_autotune result): SBEC_ERR_ARG if invalid
 * for the handle's problem.  sbec_get_tune: the shapes in use, the built-in
 * choices filled in. */
int sbec_set_tune(sbec_handle* h, const sbec_tune* t);
int sbec_get_tune(const sbec_handle* h, sbec_tune* out);

/* Launch bookkeeping (not in the paper: instrumentation of this library).
 * sbec_launch_count: number of library kernels launched on the handle so far.
 * sbec_profile(h, 1) starts recording a CUDA event pair around every kernel
 * launch on the handle's stream (at most 16384 launches; later ones are
 * counted but not timed); sbec_profile(h, 0) stops.  sbec_profile_read
 * synchronises the stream, adds the recorded device times per kernel and
 * returns up to `max` rows: names (NUL-terminated, 32 bytes each in
 * `names`), total milliseconds and launch counts; *rows receives the row
 * count.  Reading clears the recorded launches. */
long long sbec_launch_count(const sbec_handle* h);
int sbec_profile(sbec_handle* h, int enable);
int sbec_profile_read(sbec_handle* h, int max, char* names, double* ms, long long* counts, int* rows);

/* Arithmetic peak probe (not in the paper: instrumentation of this library).
 * Runs independent chains of fused multiply-adds in double (precision
 * SBEC_FP64) or float (SBEC_MIXED) on every SM of the current device, `iters`
 * steps per chain, on a private stream; *gflops receives the best of three
 * timed launches in GFLOP/s (2 per FMA).  The FP64 form of the hot path is
 * bound by this rate rather than by HBM bandwidth; it is the denominator of
 * its roofline.  Synchronises its stream; allocates nothing. */
int sbec_probe_fma_peak(int precision, int iters, double* gflops);

/* Allocation-free energy.  The paper has no counterpart: this is a service
 * of the library, not a step of the method.  It is for callers that must not
 * allocate device memory when they need the energy, for example a host
 * framework that owns all device memory through its own pool, or a
 * latency-critical loop that cannot afford cudaMalloc/cudaFree (which can
 * wait for the whole device to go idle).  It returns the same energy as
 * sbec_energy but needs no handle: every intermediate lives in one fixed
 * 8 MiB array of device memory inside the library image, which each GPU that
 * loads the library holds until the process exits.  prob must have precision
 * SBEC_FP64.  X (the state layout) and V (G doubles, or NULL for the harmonic
 * trap) must be device (or managed) memory of the current device: they are
 * read in place, and any other pointer is rejected with SBEC_ERR_ARG.  E is a
 * host pointer; the call runs on cuda_stream, synchronises it and reads E
 * back before returning.  The array holds 2^20 doubles: the transformed field
 * (2 C G doubles), the harmonic potential when V is NULL (G), and about
 * 40,000 doubles of tables and partial sums; a problem that needs more is
 * rejected with SBEC_ERR_ARG (spin-3 on 256 x 256 fits, spin-3 on 512 x 256
 * does not).  The first call on a device looks up the array's device
 * address, so make it before any stream capture.  All calls share the one
 * array and leave their intermediates in it: calls that overlap on the GPU
 * (other streams or host threads) race and must be serialised by the
 * caller. */
int sbec_energy_noalloc(const sbec_problem* prob, const double* V, const void* X, double* E,
                        void* cuda_stream);

#define SBEC_S_ENERGY      0   /* E_h of the latest energy / grad call */
#define SBEC_S_RGRAD_NORM2 1   /* ||grad E||^2 of the latest grad call */
#define SBEC_S_ALPHA_G     2   /* Lemma 4.2 alpha_g of the latest grad call */
#define SBEC_S_BETA_G      3   /* Lemma 4.2 beta_g */
#define SBEC_S_MASS        4   /* u^T u of the latest grad call */
#define SBEC_S_MAG         5   /* u^T Gamma u */
#define SBEC_S_STATUS      6   /* device-side error code (as double) */

const char* sbec_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SBEC_H */
