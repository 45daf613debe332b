// Pass kernels and their orchestration for one precision T (double or float).
// Included once per precision by sbec_kernels_f64.cu / sbec_kernels_f32.cu.
//
// Energy + gradient of a d-dimensional problem (Sec. 3) is d+1 passes over
// the C-component field, every FFT pencil staged through shared memory:
//   x pass, forward (all C components of one grid row per block)
//   strided passes along y (z) forward ... the last axis fused as
//       forward -> multiply by |k|^2 / G (Eq. 3.5, L = C^* Lambda C) -> inverse
//   strided inverse passes ... x pass inverse fused with the pointwise
//       gradient (Eq. 3.12), the energy density (Eq. 3.7) and the per-component
//       reductions u_l^T u_l, u_l^T g_l that Lemma 4.1 needs.
// The Hessian-vector product (Eq. 3.13) runs the same passes on Z with a
// Hessian epilogue; the energy alone needs only forward passes (Parseval).
#pragma once

#include <math.h>

#include <atomic>

#include "sbec_device.cuh"
#include "sbec_internal.h"

namespace sbec {

// instance `inst` of a batch is switched off by its scalar block (S_SKIP)
__device__ __forceinline__ bool skipped(const double* scal0, long long inst) {
    return scal0 != nullptr && scal0[inst * S_COUNT + S_SKIP] != 0.0;
}

// Launch slot -> instance of a batch: a launch covers the nl instances listed in
// imap (the running ones of a lock-step solve), or all of them when imap is null.
// Partial sums are laid out by slot, data and scalar blocks by instance.
__device__ __forceinline__ long long inst_of(const int* imap, long long slot) {
    return imap ? (long long)imap[slot] : slot;
}

// ---------------------------------------------------------------------------
// Finalize steps: fixed-order sums of the partials and the scalar algebra of
// Lemma 4.1 / 4.2 and of the retractions, run by one block per instance (the
// last block of the kernel that stored the partials, or a one-block kernel).
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void set_status(double* scal, int code) {
    if (scal[SBEC_S_STATUS] == 0.0) scal[SBEC_S_STATUS] = double(code);
}

// Block-parallel fixed-order sums of nq partial quantities.  With nw warps, each
// quantity gets wq = max(1, nw / nq) warps; warp j of quantity k sums the
// lane-strided elements part*32 + lane + i * wq * 32 (part = j) and a shuffle
// tree, then thread k adds the wq warp sums in order, so every sum has an order
// fixed by the block size.  Quantity q of instance b is partials[q * ntot + off ..
// off + cnt - 1] with off = b * cnt.  vals[k] is valid after the barrier.  Every
// block that calls it has a multiple of 32 threads (all launch shapes do).
// U loads of a lane are in flight at a time (the order of the sums is the same for
// every U).  U = 1 in the tail of k_dot_reduce: with U = 8 there, the FP32 spin-3
// kernel took 0.57 instead of 0.38 ms on 256^3 fields (its main loop, unchanged in
// the source, was compiled differently).
template <int U = 8>
__device__ __forceinline__ void warp_sums(const double* __restrict__ pa, int ntot, int off, int cnt, const int* qs,
                                          int nq, double* vals) {
    __shared__ double part_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int wq = nq < nw ? nw / nq : 1;
    for (int j = warp; j < nq * wq; j += nw) {
        const int k = j / wq, part = j - k * wq;
        const double* src = pa + (size_t)qs[k] * ntot + off;
        // sequential sum of the lane's elements, U loads in flight at a time
        const int st = wq * 32;
        int i = part * 32 + lane;
        double s = 0.0;
        if constexpr (U > 1) {
            for (; i + (U - 1) * st < cnt; i += U * st) {
                double t[U];
#pragma unroll
                for (int u = 0; u < U; ++u) t[u] = __ldcg(src + i + u * st);
#pragma unroll
                for (int u = 0; u < U; ++u) s += t[u];
            }
        }
        for (; i < cnt; i += st) s += __ldcg(src + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (wq == 1) vals[k] = s;
            else part_sums[j] = s;
        }
    }
    __syncthreads();
    if (wq > 1) {
        if ((int)threadIdx.x < nq) {
            double s = 0.0;
            for (int p = 0; p < wq; ++p) s += part_sums[threadIdx.x * wq + p];
            vals[threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// Finalize bodies: instance `inst` sits in launch slot b; its partials are the
// slice b * na_inst .. of na_inst blocks inside the na_tot blocks of the launch.

// Finalize fused into a producer: every block of instance `inst` stores its
// partials, then draws a ticket in the instance's scalar block; the block that
// draws the last one (nblk_slot - 1) runs the finalize on all of them.  Thread 0
// wrote the block's partials (block_reduce_store) and fences them before its
// ticket; the last block resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(double* scal, int nblk_slot) {
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();
        const double t = atomicAdd(scal + S_TICKET, 1.0);
        last = (t == double(nblk_slot - 1));
        if (last) scal[S_TICKET] = 0.0;
        __threadfence();
    }
    __syncthreads();
    return last != 0;
}

// energy: scal[E] = sum of partA quantities 0..nqa-1 (+ partB quantity 0)
__device__ __forceinline__ void fin_energy_body(const double* pa, int na_tot, int na_inst, int nqa, const double* pb,
                                                int nb_tot, int nb_inst, double* scal0, int b, long long inst) {
    __shared__ double va[4], vb[1];
    const int qa[4] = {0, 1, 2, 3}, qb[1] = {0};
    warp_sums(pa, na_tot, b * na_inst, na_inst, qa, nqa, va);
    if (pb) warp_sums(pb, nb_tot, b * nb_inst, nb_inst, qb, 1, vb);
    if (threadIdx.x == 0) {
        double* scal = scal0 + (size_t)inst * S_COUNT;
        double e = 0.0;
        for (int q = 0; q < nqa; ++q) e += va[q];
        if (pb) e += vb[0];
        scal[SBEC_S_ENERGY] = e;
        if (!isfinite(e)) set_status(scal, SBEC_ERR_NONFINITE);
    }
}

// gradient / projection coefficients (Lemma 4.1, Eq. ab) from n_l (q = qn + l) and
// t_l (q = qt + l): alpha_w = (c u^T w - M u^T Gamma w)/(c - M^2),
// beta_w = (u^T Gamma w - M u^T w)/(c - M^2), c = u^T Gamma^2 u.
struct FinProj {
    int on;                 // run by the producer's last block per instance
    int qe, qn, qt;         // partial quantities: energy (-1: none), n_l, t_l
    int slot_a, slot_b, write_grad_info;
    double M0;
    const double* Mb;
    double* scal0;          // scalar blocks (tickets and results)
};

// Energy finalize fused into the Parseval pass: pa holds the x pass's pointwise
// energy partials (one quantity), the pass's own partials the kinetic term.
struct FinEnergy {
    int on;
    const double* pa;
    int na_tot, na_inst;
    double* scal0;
};

template <int U = 8>
__device__ __forceinline__ void fin_proj_body(const double* pa, int na_tot, int na_inst, int F, int qe, int qn, int qt,
                                              double M0, const double* Mb, double* scal0, int slot_a, int slot_b,
                                              int write_grad_info, int b, long long inst) {
    const int C = 2 * F + 1;
    __shared__ double v[2 * kMaxC + 1];
    int qs[2 * kMaxC + 1];
    int nq = 0;
    for (int i = 0; i < C; ++i) qs[nq++] = qn + i;
    for (int i = 0; i < C; ++i) qs[nq++] = qt + i;
    if (qe >= 0) qs[nq++] = qe;
    warp_sums<U>(pa, na_tot, b * na_inst, na_inst, qs, nq, v);
    if (threadIdx.x == 0) {
        double* scal = scal0 + (size_t)inst * S_COUNT;
        const double M = Mb ? Mb[inst] : M0;
        double e = (qe >= 0) ? v[2 * C] : 0.0, a = 0.0, bb = 0.0, c = 0.0, ug = 0.0, uGg = 0.0;
        for (int i = 0; i < C; ++i) {
            const double l = double(F - i), nl = v[i], tl = v[C + i];
            a += nl; bb += l * nl; c += l * l * nl;
            ug += tl; uGg += l * tl;
        }
        const double au = c - M * M;
        const double al = (c * ug - M * uGg) / au;
        const double be = (uGg - M * ug) / au;
        if (!isfinite(c) || !isfinite(ug) || !isfinite(uGg) || !isfinite(e)) set_status(scal, SBEC_ERR_NONFINITE);
        if (!(au > 0.0)) set_status(scal, SBEC_ERR_DOMAIN);
        scal[slot_a] = al;
        scal[slot_b] = be;
        if (write_grad_info) {
            scal[SBEC_S_ENERGY] = e;
            scal[SBEC_S_MASS] = a;
            scal[SBEC_S_MAG] = bb;
            scal[S_C2] = c;
            if (!isfinite(e) || !isfinite(al) || !isfinite(be)) set_status(scal, SBEC_ERR_NONFINITE);
        }
    }
}

// one block per instance: the finalize of a producer that does not run it itself
static __global__ void k_fin_proj(const double* pa, int na_tot, int na_inst, int F, const FinProj fp,
                                  const int* imap) {
    const int b = blockIdx.x;
    const long long inst = inst_of(imap, b);
    if (skipped(fp.scal0, inst)) return;
    fin_proj_body(pa, na_tot, na_inst, F, fp.qe, fp.qn, fp.qt, fp.M0, fp.Mb, fp.scal0, fp.slot_a, fp.slot_b,
                  fp.write_grad_info, b, inst);
}

__device__ __forceinline__ void fin_norm_body(const double* pa, int na_tot, int na_inst, double* scal0, int slot,
                                              int b, long long inst) {
    __shared__ double v[1];
    const int q[1] = {0};
    warp_sums(pa, na_tot, b * na_inst, na_inst, q, 1, v);
    if (threadIdx.x == 0) {
        double* scal = scal0 + (size_t)inst * S_COUNT;
        scal[slot] = v[0];
        if (!isfinite(v[0])) set_status(scal, SBEC_ERR_NONFINITE);
    }
}

#define SBEC_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return SBEC_ERR_CUDA;          \
    } while (0)
#define SBEC_LAUNCH_CHECK() SBEC_CUDA_TRY(cudaGetLastError())

enum XMode {
    X_FWD = 0,         // forward x-FFT of every row
    X_FWD_EPW = 1,     // + pointwise energy partial (q0)
    X_INV_GRAD = 2,    // inverse x-FFT + gradient epilogue, partials E, n_l, t_l
    X_INV_HESS = 3,    // inverse x-FFT + Hessian epilogue, partials n_l, t_l
    X_FULL_GRAD = 4,   // 1D: fwd, |k|^2/G, inv, gradient epilogue
    X_FULL_ENERGY = 5, // 1D: pointwise energy + fwd + Parseval
    X_FULL_HESS = 6,   // 1D: fwd, |k|^2/G, inv, Hessian epilogue
    X_INV = 7          // inverse x-FFT of every row, stored
};

enum SMode { S_FWD = 0, S_INV = 1, S_K2 = 2, S_PARSEVAL = 3 };

template <int MODE, int C> struct XNQ {
    static constexpr int v = (MODE == X_INV_GRAD || MODE == X_FULL_GRAD) ? 1 + 2 * C
                           : (MODE == X_INV_HESS || MODE == X_FULL_HESS) ? 2 * C
                           : (MODE == X_FULL_ENERGY) ? 2
                           : (MODE == X_FWD_EPW) ? 1 : 1;
};

struct XArgs {
    const void* in;       // field to transform (X, Z or work)
    void* out;            // destination (work, or the gradient / Hessian output)
    const void* X;        // state (epilogues)
    const void* Zd;       // direction (Hessian epilogue, = in for FULL_HESS)
    const void* V;
    const void* tw;
    const double* lam2x;
    const void* k2x;      // T: lambda_p^2 / G along x (the precision of the pass)
    long long G;
    int logn;             // x length
    int rpb;              // row groups per block
    double invG;
    double sigma;         // Hessian shift
    const double* scal;   // device scalar block: Lemma 4.2 alpha_g, beta_g (riemannian epilogue)
    int riem;
    int sigslot;          // >= 0: sigma is multiplied by the instance's scal[sigslot]
    int zproj;            // Hessian of a Riemannian product: the direction read from `in` (x pass)
                          // or Zd (epilogue) is Z, and the pass uses xi = P_u Z = Z - (a + b l) X
                          // with a, b = the instance's scal[S_PA], scal[S_PB] (Lemma 4.1)
    double* partials;
    int nblk;
    PointParams pp;
    long long rpi;              // grid rows (x lines) per instance
    const PointParams* ppb;     // per-instance point parameters (batches) or null
    const double* skip;         // scalar blocks (S_SKIP flags) or null
    const int* imap;            // launch slot -> instance, or null (identity)
    FinProj fp;                 // fp.on: Lemma 4.1 finalize by the last block per instance
    int fe;                     // X_FULL_ENERGY: energy finalize by the last block per
                                // instance, into the scalar blocks fp.scal0
    double* dens;               // FP64 stand-alone epilogues: densities per point, stored by
                                // the gradient epilogue and read by the Hessian epilogue
                                // ([B][dens_count(F)][G]), or null
};

// Shift of the Hessian epilogue per component: sigma (times the instance's
// scal[sigslot] when sigslot >= 0), minus alpha_g + beta_g l in the Riemannian
// form (Lemma 4.2), in the pass precision.
template <int F, typename T>
__device__ __forceinline__ void hess_shift(const XArgs& a, const double* scal, T (&shift)[2 * F + 1]) {
#pragma unroll
    for (int c = 0; c < 2 * F + 1; ++c) {
        T s = T(a.sigslot >= 0 ? a.sigma * scal[a.sigslot] : a.sigma);
        if (a.riem) s -= T(scal[SBEC_S_ALPHA_G] + scal[SBEC_S_BETA_G] * double(F - c));
        shift[c] = s;
    }
}

template <typename T, int F, int MODE, int ITEMS>
__global__ void __launch_bounds__(512) k_xpass(const XArgs a) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    constexpr int NQ = XNQ<MODE, C>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* buf = reinterpret_cast<T2*>(smem_raw);
    const int logn = a.logn, n = 1 << logn;
    const int RPB = a.rpb, P = RPB * C;
    const int tid = threadIdx.x, nth = blockDim.x;
    // instance of this block (blocks never straddle instances) and its offsets
    const long long growrow = (long long)blockIdx.x * RPB;
    const long long slot = growrow / a.rpi;
    const long long inst = inst_of(a.imap, slot);
    const long long row0 = growrow - slot * a.rpi;
    const long long foff = inst * (long long)C * a.G;
    const T2* __restrict__ src = reinterpret_cast<const T2*>(a.in) + foff;
    const T2* __restrict__ tw = reinterpret_cast<const T2*>(a.tw);
    const T* __restrict__ Vp = reinterpret_cast<const T*>(a.V) + inst * a.G;
    const PPT<T> pp(a.ppb ? a.ppb[inst] : a.pp);
    const double* scal = a.scal ? a.scal + inst * S_COUNT : nullptr;
    const T* __restrict__ k2x = reinterpret_cast<const T*>(a.k2x);
    if (skipped(a.skip, inst)) return;

    for (int idx = tid; idx < P * n; idx += nth) {
        const int p = idx >> logn, e = idx & (n - 1);
        const int rg = p / C, c = p - rg * C;
        buf[smem_slot(idx)] = src[(long long)c * a.G + (row0 + rg) * n + e];
    }
    __syncthreads();

    Acc<T> acc[NQ];

    if (MODE == X_FWD_EPW || MODE == X_FULL_ENERGY) {
        for (int idx = tid; idx < RPB * n; idx += nth) {
            const int rg = idx >> logn, e = idx & (n - 1);
            T2 x[C];
#pragma unroll
            for (int c = 0; c < C; ++c) x[c] = buf[smem_slot((rg * C + c) * n + e)];
            Dens<F, T2> D;
            D.compute(x);
            acc[0].add(D.energy_density(x, Vp[(row0 + rg) * n + e], pp));
        }
        __syncthreads();
    }

    const bool fwd = (MODE == X_FWD || MODE == X_FWD_EPW || MODE == X_FULL_GRAD || MODE == X_FULL_ENERGY ||
                      MODE == X_FULL_HESS);
    if (fwd) fft_pencils<T2, false, ITEMS, false, true>(buf, logn, P, n, 1, tw, tid, nth);

    if (MODE == X_FULL_ENERGY) {
        // kinetic part by Parseval: (1/(2G)) sum |k|^2 |X^|^2
        for (int idx = tid; idx < P * n; idx += nth) {
            const int e = idx & (n - 1);
            if constexpr (sizeof(T) == 8) acc[1].add(0.5 * a.invG * a.lam2x[e] * cabs2(buf[smem_slot(idx)]));
            else acc[1].add(T(0.5) * k2x[e] * cabs2(buf[smem_slot(idx)]));
        }
    }
    if (MODE == X_FULL_GRAD || MODE == X_FULL_HESS) {
        for (int idx = tid; idx < P * n; idx += nth) {
            const int e = idx & (n - 1);
            buf[smem_slot(idx)] = cscale(buf[smem_slot(idx)], k2x[e]);
        }
        __syncthreads();
    }
    const bool inv = (MODE == X_INV_GRAD || MODE == X_INV_HESS || MODE == X_FULL_GRAD || MODE == X_FULL_HESS ||
                      MODE == X_INV);
    if (inv) fft_pencils<T2, true, ITEMS, false, true>(buf, logn, P, n, 1, tw, tid, nth);

    if (MODE == X_FWD || MODE == X_FWD_EPW || MODE == X_INV) {
        T2* __restrict__ dst = reinterpret_cast<T2*>(a.out) + foff;
        for (int idx = tid; idx < P * n; idx += nth) {
            const int p = idx >> logn, e = idx & (n - 1);
            const int rg = p / C, c = p - rg * C;
            dst[(long long)c * a.G + (row0 + rg) * n + e] = buf[smem_slot(idx)];
        }
    }

    if (MODE == X_INV_GRAD || MODE == X_FULL_GRAD) {
        const T2* __restrict__ Xp = reinterpret_cast<const T2*>(a.X) + foff;
        T2* __restrict__ dst = a.out ? reinterpret_cast<T2*>(a.out) + foff : nullptr;
        for (int idx = tid; idx < RPB * n; idx += nth) {
            const int rg = idx >> logn, e = idx & (n - 1);
            const long long pt = (row0 + rg) * n + e;
            T2 x[C], lx[C], g[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                x[c] = Xp[(long long)c * a.G + pt];
                lx[c] = buf[smem_slot((rg * C + c) * n + e)];
            }
            const T V = Vp[pt];
            Dens<F, T2> D;
            D.compute(x);
            grad_point<F, T2>(x, D, V, pp, lx, g);
            T ek = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) ek += x[c].x * lx[c].x + x[c].y * lx[c].y;
            acc[0].add(T(0.5) * ek + D.energy_density(x, V, pp));
#pragma unroll
            for (int c = 0; c < C; ++c) {
                acc[1 + c].add(cabs2(x[c]));
                acc[1 + C + c].add(x[c].x * g[c].x + x[c].y * g[c].y);
                if (dst) dst[(long long)c * a.G + pt] = g[c];
            }
        }
    }

    if (MODE == X_INV_HESS || MODE == X_FULL_HESS) {
        const T2* __restrict__ Xp = reinterpret_cast<const T2*>(a.X) + foff;
        const T2* __restrict__ Zp = reinterpret_cast<const T2*>(a.Zd) + foff;
        T2* __restrict__ dst = reinterpret_cast<T2*>(a.out) + foff;
        T shift[C];
        hess_shift<F, T>(a, scal, shift);
        for (int idx = tid; idx < RPB * n; idx += nth) {
            const int rg = idx >> logn, e = idx & (n - 1);
            const long long pt = (row0 + rg) * n + e;
            T2 x[C], z[C], lz[C], h[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                x[c] = Xp[(long long)c * a.G + pt];
                z[c] = Zp[(long long)c * a.G + pt];
                lz[c] = buf[smem_slot((rg * C + c) * n + e)];
            }
            const T V = Vp[pt];
            Dens<F, T2> D;
            D.compute(x);
            hess_point<F, T2>(x, z, D, V, pp, lz, h);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                caxpy(h[c], shift[c], z[c]);
                acc[c].add(cabs2(x[c]));
                acc[C + c].add(x[c].x * h[c].x + x[c].y * h[c].y);
                dst[(long long)c * a.G + pt] = h[c];
            }
        }
    }

    if (MODE != X_FWD && MODE != X_INV) {
        double v[NQ];
        acc_values(acc, v);
        block_reduce_store<NQ>(v, a.partials, a.nblk, blockIdx.x);
        // 1D passes: the finalize by the last block of the instance
        const int nb_inst = (int)(a.rpi / RPB);
        if (MODE == X_FULL_ENERGY && a.fe && last_block(a.fp.scal0 + inst * S_COUNT, nb_inst))
            fin_energy_body(a.partials, a.nblk, nb_inst, 2, nullptr, 0, 0, a.fp.scal0, (int)slot, inst);
        if (MODE != X_FULL_ENERGY && a.fp.on && last_block(a.fp.scal0 + inst * S_COUNT, nb_inst))
            fin_proj_body(a.partials, a.nblk, nb_inst, F, a.fp.qe, a.fp.qn, a.fp.qt, a.fp.M0, a.fp.Mb, a.fp.scal0,
                          a.fp.slot_a, a.fp.slot_b, a.fp.write_grad_info, (int)slot, inst);
    }
}

struct SArgs {
    const void* in;
    void* out;
    const void* tw;
    const double* lam2[3];
    const void* k2t[3];   // T: lambda_p^2 / G per axis (the precision of the pass)
    long long G;
    int axis;         // 1 = y, 2 = z
    int logn;         // axis length
    int W;            // pencils (consecutive x) per block
    int nx, ny, nz;
    int ntx;          // nx / W
    int nouter;       // nz for axis y, ny for axis z
    long long estride;
    double invG;
    double* partials;
    int nblk;
    int nblk_inst;        // blocks per instance
    int C;                // components (instance = pencil component / C)
    const double* skip;   // scalar blocks (S_SKIP flags) or null
    const int* imap;      // launch slot -> instance, or null (identity)
    FinEnergy fe;         // S_PARSEVAL, fe.on: energy finalize by the last block per instance
};

template <typename T, int MODE, int ITEMS>
__global__ void __launch_bounds__(512) k_spass(const SArgs a) {
    using T2 = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* buf = reinterpret_cast<T2*>(smem_raw);
    const int logn = a.logn, n = 1 << logn, W = a.W;
    const int tid = threadIdx.x, nth = blockDim.x;
    long long b = blockIdx.x;
    const int xt = (int)(b % a.ntx); b /= a.ntx;
    const int o = (int)(b % a.nouter);
    const int cs = (int)(b / a.nouter);                     // slot * C + component
    const long long inst = inst_of(a.imap, cs / a.C);
    const long long c = inst * a.C + (cs % a.C);
    if (skipped(a.skip, inst)) return;
    const long long obase = (a.axis == 1) ? (long long)o * a.ny * a.nx : (long long)o * a.nx;
    const long long base = (long long)c * a.G + obase + (long long)xt * W;
    const T2* __restrict__ src = reinterpret_cast<const T2*>(a.in);
    const T2* __restrict__ tw = reinterpret_cast<const T2*>(a.tw);

    for (int idx = tid; idx < W * n; idx += nth) {
        const int e = idx / W, w = idx - e * W;
        buf[idx] = src[base + e * a.estride + w];
    }
    __syncthreads();
    fft_pencils<T2, MODE == S_INV, ITEMS, true>(buf, logn, W, 1, W, tw, tid, nth);

    if (MODE == S_K2 || MODE == S_PARSEVAL) {
        Acc<T> acc[1];
        const T* __restrict__ k0 = reinterpret_cast<const T*>(a.k2t[0]);
        const T* __restrict__ k1 = reinterpret_cast<const T*>(a.k2t[1]);
        const T* __restrict__ k2t = reinterpret_cast<const T*>(a.k2t[2]);
        for (int idx = tid; idx < W * n; idx += nth) {
            const int e = idx / W, w = idx - e * W;
            // frequency indices: x and the pass axis from the tile, the third axis from o
            const int ix = xt * W + w;
            const int iy = (a.axis == 1) ? e : o;
            const int iz = (a.axis == 2) ? e : o;
            if constexpr (sizeof(T) == 8) {
                const double k2 = a.lam2[0][ix] + a.lam2[1][iy] + a.lam2[2][iz];
                if (MODE == S_K2) buf[idx] = cscale(buf[idx], T(k2 * a.invG));
                else acc[0].add(0.5 * a.invG * k2 * cabs2(buf[idx]));
            } else {
                // FP32: |k|^2 / G from the per-axis tables, no FP64 arithmetic per point
                const T f = k0[ix] + k1[iy] + k2t[iz];
                if (MODE == S_K2) buf[idx] = cscale(buf[idx], f);
                else acc[0].add(T(0.5) * f * cabs2(buf[idx]));
            }
        }
        if (MODE == S_PARSEVAL) {
            double v[1];
            acc_values(acc, v);
            block_reduce_store<1>(v, a.partials, a.nblk, blockIdx.x);
            const int slot = cs / a.C, nb_inst = a.nblk_inst;
            if (a.fe.on && last_block(a.fe.scal0 + inst * S_COUNT, nb_inst))
                fin_energy_body(a.fe.pa, a.fe.na_tot, a.fe.na_inst, 1, a.partials, a.nblk, nb_inst, a.fe.scal0, slot,
                                inst);
            return;
        }
        __syncthreads();
        fft_pencils<T2, true, ITEMS, true>(buf, logn, W, 1, W, tw, tid, nth);
    }
    T2* __restrict__ dst = reinterpret_cast<T2*>(a.out);
    for (int idx = tid; idx < W * n; idx += nth) {
        const int e = idx / W, w = idx - e * W;
        dst[base + e * a.estride + w] = buf[idx];
    }
}

// ---------------------------------------------------------------------------
// Passes with the two-level FFT (lengths n = 2^LOGN <= 256).  Level A reads its
// values straight from global memory and level A' writes them straight back;
// the level-B values of one k2 stay in registers, so the k-space scaling of
// S_K2 and the Parseval sum touch no shared memory.  The one exchange per
// transform goes through the block's shared-memory tile.
// ---------------------------------------------------------------------------

// Strided pass: W pencils (consecutive x) of one component along the pass axis;
// thread (w, q), w = tid mod W, blockDim.x = W N1 <= 256.  Exchange slot of element
// (e1, e2) of pencil w: sm[e2 * rs + e1 * W + w], rs = N1 W + pad; pad = W for
// W < 16 puts the level-B reads of a half-warp on distinct banks.
template <typename T, int MODE, int LOGN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_spass2(const SArgs a) {
    using T2 = typename C2<T>::t;
    constexpr int N1 = Split2<LOGN>::N1, N2 = Split2<LOGN>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* sm = reinterpret_cast<T2*>(smem_raw);
    const int W = a.W;
    const int w = threadIdx.x & (W - 1), q = threadIdx.x / W;
    long long b = blockIdx.x;
    const int xt = (int)(b % a.ntx); b /= a.ntx;
    const int o = (int)(b % a.nouter);
    const int cs = (int)(b / a.nouter);                     // slot * C + component
    const long long inst = inst_of(a.imap, cs / a.C);
    const long long c = inst * a.C + (cs % a.C);
    if (skipped(a.skip, inst)) return;
    const long long obase = (a.axis == 1) ? (long long)o * a.ny * a.nx : (long long)o * a.nx;
    const long long base = (long long)c * a.G + obase + (long long)xt * W + w;
    const T2* __restrict__ src = reinterpret_cast<const T2*>(a.in) + base;
    const T2* __restrict__ tw = reinterpret_cast<const T2*>(a.tw);
    const long long es = a.estride;
    const int rs = N1 * W + (W < 16 ? W : 0);
    T2 v[N1];
    if (MODE != S_INV) {
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = src[(long long)(q + N1 * j2) * es];
        level_a_fwd<T2, LOGN, false>(v, q, tw);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) sm[k2 * rs + q * W + w] = v[k2];
        __syncthreads();
        if (q < N2) {
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = sm[q * rs + j1 * W + w];
            RegDft<T2, N1, false>::run(v);            // v[k1] = X[q + N2 k1]
        }
    }
    if (MODE == S_FWD) {
        T2* __restrict__ dst = reinterpret_cast<T2*>(a.out) + base;
        if (q < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) dst[(long long)(q + N2 * k1) * es] = v[k1];
        }
        return;
    }
    if (MODE == S_K2 || MODE == S_PARSEVAL) {
        Acc<T> acc[1];
        if (q < N2) {
            const int ix = xt * W + w;
            const bool ya = (a.axis == 1);
            if constexpr (sizeof(T) == 8) {
                // |k|^2 = (lam_x + lam_y) + lam_z, the pass axis' term from the table
                const double lx = a.lam2[0][ix], lo = a.lam2[ya ? 2 : 1][o];
                const double* __restrict__ le = a.lam2[a.axis];
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    const double l = le[q + N2 * k1];
                    const double k2 = ya ? (lx + l) + lo : (lx + lo) + l;
                    if (MODE == S_K2) v[k1] = cscale(v[k1], T(k2 * a.invG));
                    else acc[0].add(0.5 * a.invG * k2 * cabs2(v[k1]));
                }
            } else {
                const T f0 = reinterpret_cast<const T*>(a.k2t[0])[ix] +
                             reinterpret_cast<const T*>(a.k2t[ya ? 2 : 1])[o];
                const T* __restrict__ fe = reinterpret_cast<const T*>(a.k2t[a.axis]);
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    const T f = f0 + fe[q + N2 * k1];
                    if (MODE == S_K2) v[k1] = cscale(v[k1], f);
                    else acc[0].add(T(0.5) * f * cabs2(v[k1]));
                }
            }
        }
        if (MODE == S_PARSEVAL) {
            double r[1];
            acc_values(acc, r);
            block_reduce_store<1>(r, a.partials, a.nblk, blockIdx.x);
            const int slot = cs / a.C, nb_inst = a.nblk_inst;
            if (a.fe.on && last_block(a.fe.scal0 + inst * S_COUNT, nb_inst))
                fin_energy_body(a.fe.pa, a.fe.na_tot, a.fe.na_inst, 1, a.partials, a.nblk, nb_inst, a.fe.scal0, slot,
                                inst);
            return;
        }
    }
    if (MODE == S_INV && q < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[(long long)(q + N2 * k1) * es];
    }
    // inverse: level B' (k2 = q; its slots are this thread's own), exchange, level A'
    if (q < N2) {
        level_b_inv<T2, LOGN>(v, q, tw);
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) sm[q * rs + j1 * W + w] = v[j1];
    }
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = sm[k2 * rs + q * W + w];
    RegDft<T2, N2, true>::run(v);                     // v[j2] = x[q + N1 j2]
    T2* __restrict__ dst = reinterpret_cast<T2*>(a.out) + base;
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) dst[(long long)(q + N1 * j2) * es] = v[j2];
}

}  // namespace sbec

// the TMA variant of the strided pass (uses SArgs, the pass modes and the finalize bodies above)
#include "sbec_tma.cuh"

namespace sbec {

// x pass of 2D / 3D problems (X_FWD, X_FWD_EPW, X_INV): rpb grid rows of all C
// components; pencil p = row group * C + component, thread (p, q) with
// q = tid mod N1 (threads with p >= P only join the barriers and sums).
// Exchange slot of element (e1, e2) of pencil p: sm[p * S + e2 (N1 + 1) + e1],
// S = N2 (N1 + 1); the +1 spreads the level-B reads over the banks.
template <typename T, int F, int MODE, int LOGN>
__global__ void __launch_bounds__(512) k_xpass2(const XArgs a) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    constexpr int N = 1 << LOGN, N1 = Split2<LOGN>::N1, N2 = Split2<LOGN>::N2;
    constexpr int S = N2 * (N1 + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* sm = reinterpret_cast<T2*>(smem_raw);
    const int RPB = a.rpb, P = RPB * C;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int p = tid / N1, q = tid & (N1 - 1);
    const bool on = p < P;
    const long long growrow = (long long)blockIdx.x * RPB;
    const long long slot = growrow / a.rpi;
    const long long inst = inst_of(a.imap, slot);
    const long long row0 = growrow - slot * a.rpi;
    const long long foff = inst * (long long)C * a.G;
    if (skipped(a.skip, inst)) return;
    const int rg = p / C, cc = p - rg * C;
    const long long roff = foff + (long long)cc * a.G + (row0 + rg) * N;
    const T2* __restrict__ row = reinterpret_cast<const T2*>(a.in) + (on ? roff : 0);
    T2* __restrict__ orow = reinterpret_cast<T2*>(a.out) + (on ? roff : 0);
    const T2* __restrict__ tw = reinterpret_cast<const T2*>(a.tw);
    T2* my = sm + p * S;
    Acc<T> acc[1];
    if (MODE == X_FWD_EPW) {
        // pointwise energy density of the block's input points (Eq. 3.7 without the kinetic term)
        const T2* __restrict__ src = reinterpret_cast<const T2*>(a.in) + foff;
        const T* __restrict__ Vp = reinterpret_cast<const T*>(a.V) + inst * a.G;
        const PPT<T> pp(a.ppb ? a.ppb[inst] : a.pp);
        for (int idx = tid; idx < RPB * N; idx += nth) {
            const long long pt = (row0 + (idx >> LOGN)) * N + (idx & (N - 1));
            T2 x[C];
#pragma unroll
            for (int c = 0; c < C; ++c) x[c] = src[(long long)c * a.G + pt];
            Dens<F, T2> D;
            D.compute(x);
            acc[0].add(D.energy_density(x, Vp[pt], pp));
        }
    }
    T2 v[N1];
    if (MODE != X_INV) {
        if (on) {
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) v[j2] = row[q + N1 * j2];
            if (MODE == X_FWD && a.zproj) {
                // xi = Z - (a + b l) X on the fly: the projected direction is never stored
                const double* sc = a.scal + inst * S_COUNT;
                const T cf = T(sc[S_PA] + sc[S_PB] * double(F - cc));
                const T2* __restrict__ xrow = reinterpret_cast<const T2*>(a.X) + roff;
#pragma unroll
                for (int j2 = 0; j2 < N2; ++j2) caxpy(v[j2], -cf, xrow[q + N1 * j2]);
            }
            level_a_fwd<T2, LOGN, false>(v, q, tw);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) my[k2 * (N1 + 1) + q] = v[k2];
        }
        __syncthreads();
        if (on && q < N2) {
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) v[j1] = my[q * (N1 + 1) + j1];
            RegDft<T2, N1, false>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) orow[q + N2 * k1] = v[k1];
        }
    } else {
        if (on && q < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = row[q + N2 * k1];
            level_b_inv<T2, LOGN>(v, q, tw);
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) my[q * (N1 + 1) + j1] = v[j1];
        }
        __syncthreads();
        if (on) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k2] = my[k2 * (N1 + 1) + q];
            RegDft<T2, N2, true>::run(v);
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) orow[q + N1 * j2] = v[j2];
        }
    }
    if (MODE == X_FWD_EPW) {
        double r[1];
        acc_values(acc, r);
        block_reduce_store<1>(r, a.partials, a.nblk, blockIdx.x);
    }
}

// ---------------------------------------------------------------------------
// Stand-alone epilogues (used when the inverse x pass only transforms): the
// gradient (Eq. 3.12) or Hessian-vector product (Eq. 3.13) of every grid point
// from L X (or L Z) in `lx`, with the same partial sums as the fused x pass.
// blockIdx.y is the instance; partials of instance b are blocks b*gridDim.x ...
//
// The inputs of a point (X, L X, Z: C values each, and V) reach shared memory by
// per-thread asynchronous copies (cp.async) one or two grid-stride steps ahead:
// while a thread computes point k, the copies of the next points are in flight,
// so the register-heavy pointwise algebra (one or two blocks per SM) overlaps the
// HBM traffic.  Each thread reads back only the slots it copied itself.
// ---------------------------------------------------------------------------
constexpr int kEpiThreads = 256;

// Epilogues whose last block per instance runs the Lemma 4.1 finalize.  The F = 3
// Hessian epilogue keeps a separate finalize launch: with the finalize in its tail
// ptxas allocated its registers differently (168 instead of 254 in FP32) and the
// epilogue ran 5-9% slower on the 128^3 (FP64) and 256^3 (FP32) spin-3 grids.
template <typename T, int F, bool HESS> struct EpiFusedFin { static constexpr bool v = !(HESS && F == 3); };

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int F, bool HESS>
__host__ __device__ constexpr size_t epi_stage_bytes() {
    return (size_t)(HESS ? 3 : 2) * (2 * F + 1) * kEpiThreads * sizeof(typename C2<T>::t) +
           (size_t)kEpiThreads * sizeof(T);
}
// Resident blocks per SM the epilogue is compiled for: two in FP32 (its pointwise
// algebra fits 128 registers), except the spin-3 Hessian, whose algebra spills at 128
// registers and runs faster as one block with three copy stages; one in FP64 (the
// FP64 pipe, not latency, bounds it)
template <typename T, int F, bool HESS> struct EpiBlocks {
    static constexpr int v = (sizeof(T) == 4 && !(HESS && F >= 3)) ? 2 : 1;
};

// copies in flight: points k + 1 and k + 2 while point k is computed, when three
// stages of every resident block fit in 200 KB of shared memory, else point k + 1 only
template <typename T, int F, bool HESS>
__host__ __device__ constexpr int epi_stages() {
    return 3 * EpiBlocks<T, F, HESS>::v * epi_stage_bytes<T, F, HESS>() <= 200 * 1024   ? 3
           : 2 * EpiBlocks<T, F, HESS>::v * epi_stage_bytes<T, F, HESS>() <= 200 * 1024 ? 2
                                                                              : 1;
}
template <typename T, int F, bool HESS>
__host__ __device__ constexpr size_t epi_smem() {
    return epi_stages<T, F, HESS>() * epi_stage_bytes<T, F, HESS>();
}

// The densities of a point in dens_count(F) planes of G doubles: rho, F_z, F_+, then
// A00 (F >= 2) and the quintet amplitudes A_{2l} (F = 3)
template <int F>
__device__ __forceinline__ void dens_store(const Dens<F, double2>& D, double* __restrict__ d, long long G) {
    d[0] = D.rho; d[G] = D.Fz; d[2 * G] = D.Fp.x; d[3 * G] = D.Fp.y;
    if (F >= 2) { d[4 * G] = D.A00.x; d[5 * G] = D.A00.y; }
    if (F == 3) {
#pragma unroll
        for (int k = 0; k < 5; ++k) { d[(6 + 2 * k) * G] = D.A2[k].x; d[(7 + 2 * k) * G] = D.A2[k].y; }
    }
}
template <int F>
__device__ __forceinline__ void dens_load(Dens<F, double2>& D, const double* __restrict__ d, long long G) {
    D.rho = __ldg(d); D.Fz = __ldg(d + G); D.Fp = make_double2(__ldg(d + 2 * G), __ldg(d + 3 * G));
    D.A00 = make_double2(0.0, 0.0);
    if (F >= 2) D.A00 = make_double2(__ldg(d + 4 * G), __ldg(d + 5 * G));
    if (F == 3) {
#pragma unroll
        for (int k = 0; k < 5; ++k) D.A2[k] = make_double2(__ldg(d + (6 + 2 * k) * G), __ldg(d + (7 + 2 * k) * G));
    }
}

// DC: 0 densities formed from X; 1 (FP64 gradient) formed and stored to a.dens;
// 2 (FP64 Hessian) read from a.dens, stored there by the gradient at the same X
template <typename T, int F, bool HESS, int DC>
__global__ void __launch_bounds__(kEpiThreads, EpiBlocks<T, F, HESS>::v) k_epilogue(const XArgs a, const void* lxp, long long G) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    constexpr int NQ = HESS ? 2 * C : 1 + 2 * C;
    constexpr int NA = HESS ? 3 : 2;                  // staged arrays X, L X (, Z)
    constexpr int P = kEpiThreads;
    constexpr int NS = epi_stages<T, F, HESS>();
    const long long inst = inst_of(a.imap, blockIdx.y);
    const long long foff = inst * (long long)C * G;
    const T2* __restrict__ LX = reinterpret_cast<const T2*>(lxp) + foff;
    const T2* __restrict__ Xp = reinterpret_cast<const T2*>(a.X) + foff;
    const T2* __restrict__ Zp = HESS ? reinterpret_cast<const T2*>(a.Zd) + foff : nullptr;
    T2* __restrict__ dst = a.out ? reinterpret_cast<T2*>(a.out) + foff : nullptr;
    const T* __restrict__ Vp = reinterpret_cast<const T*>(a.V) + inst * G;
    const PPT<T> pp(a.ppb ? a.ppb[inst] : a.pp);
    const double* scal = a.scal ? a.scal + inst * S_COUNT : nullptr;
    static_assert(DC == 0 || (sizeof(T) == 8 && (DC == 1) == !HESS), "density cache: FP64 gradient / Hessian");
    double* __restrict__ dens = DC ? a.dens + inst * (long long)dens_count(F) * G : nullptr;
    if (skipped(a.skip, inst)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* stg = reinterpret_cast<T2*>(smem_raw);                       // [NS][NA C][P]
    T* vst = reinterpret_cast<T*>(stg + NS * NA * C * P);            // [NS][P]
    const int tid = threadIdx.x;
    T shift[C], zcf[C];
    if (HESS) hess_shift<F, T>(a, scal, shift);
    if (HESS && a.zproj) {
        // Lemma 4.1 coefficients of Z, read before this launch's own finalize rewrites them
#pragma unroll
        for (int c = 0; c < C; ++c) zcf[c] = T(scal[S_PA] + scal[S_PB] * double(F - c));
    }
    Acc<T> acc[NQ];
    const long long stride = (long long)gridDim.x * P;
    // copies of point p into stage st (none past the end; the group is committed anyway)
    auto issue = [&](long long p, int st) {
        if (p < G) {
            T2* d = stg + (size_t)st * NA * C * P + tid;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                cp_async<sizeof(T2)>(d + c * P, Xp + c * G + p);
                cp_async<sizeof(T2)>(d + (C + c) * P, LX + c * G + p);
                if (HESS) cp_async<sizeof(T2)>(d + (2 * C + c) * P, Zp + c * G + p);
            }
            cp_async<sizeof(T)>(vst + st * P + tid, Vp + p);
        }
        cp_async_commit();
    };
    long long pt = (long long)blockIdx.x * P + tid;
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) issue(pt + k * stride, k);
    for (int k = 0; pt < G; ++k, pt += stride) {
        issue(pt + (NS - 1) * stride, (k + NS - 1) % NS);
        Dens<F, T2> Dl;                              // DC == 2: loads in flight during the wait
        if constexpr (DC == 2) dens_load<F>(Dl, dens + pt, G);
        cp_async_wait<NS - 1>();                     // this thread's copies of point pt are in
        const int sk = k % NS;
        const T2* sx = stg + (size_t)sk * NA * C * P + tid;
        T2 x[C], l[C], o[C];
#pragma unroll
        for (int c = 0; c < C; ++c) { x[c] = sx[c * P]; l[c] = sx[(C + c) * P]; }
        const T V = vst[sk * P + tid];
        Dens<F, T2> D;
        if constexpr (DC == 2) D = Dl;
        else D.compute(x);
        if constexpr (DC == 1) dens_store<F>(D, dens + pt, G);
        if (!HESS) {
            grad_point<F, T2>(x, D, V, pp, l, o);
            T ek = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) ek += x[c].x * l[c].x + x[c].y * l[c].y;
            acc[0].add(T(0.5) * ek + D.energy_density(x, V, pp));
#pragma unroll
            for (int c = 0; c < C; ++c) {
                acc[1 + c].add(cabs2(x[c]));
                acc[1 + C + c].add(x[c].x * o[c].x + x[c].y * o[c].y);
                if (dst) dst[c * G + pt] = o[c];
            }
        } else {
            T2 z[C];
#pragma unroll
            for (int c = 0; c < C; ++c) z[c] = sx[(2 * C + c) * P];
            if (a.zproj) {
#pragma unroll
                for (int c = 0; c < C; ++c) caxpy(z[c], -zcf[c], x[c]);
            }
            hess_point<F, T2>(x, z, D, V, pp, l, o);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                caxpy(o[c], shift[c], z[c]);
                acc[c].add(cabs2(x[c]));
                acc[C + c].add(x[c].x * o[c].x + x[c].y * o[c].y);
                dst[c * G + pt] = o[c];
            }
        }
    }
    cp_async_wait<0>();                              // no copy outlives the block
    double v[NQ];
    acc_values(acc, v);
    block_reduce_store<NQ>(v, a.partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    if constexpr (EpiFusedFin<T, F, HESS>::v) {
        if (a.fp.on && last_block(a.fp.scal0 + inst * S_COUNT, gridDim.x))
            fin_proj_body(a.partials, gridDim.x * gridDim.y, gridDim.x, F, a.fp.qe, a.fp.qn, a.fp.qt, a.fp.M0,
                          a.fp.Mb, a.fp.scal0, a.fp.slot_a, a.fp.slot_b, a.fp.write_grad_info, blockIdx.y, inst);
    }
}

// ---------------------------------------------------------------------------
// Elementwise kernels over grid points (grid-stride), all C components per point.
// ---------------------------------------------------------------------------

// Elementwise kernels: blockIdx.y is the instance of a batch, blockIdx.x strides
// over its G grid points; partials of instance b are blocks b*gridDim.x ...

// partials: n_l = |u_l|^2 (q = l index), t_l = <u_l, w_l> (q = C + l)
template <typename T, int F>
__global__ void __launch_bounds__(256) k_dot_reduce(const void* Up, const void* Wp, long long G, double* partials,
                                                    const double* skip, const int* imap, const FinProj fp) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(skip, inst)) return;
    const long long foff = inst * C * G;
    const T2* __restrict__ U = reinterpret_cast<const T2*>(Up) + foff;
    const T2* __restrict__ Wv = reinterpret_cast<const T2*>(Wp) + foff;
    Acc<T> acc[2 * C];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const T2 u = U[c * G + p], w = Wv[c * G + p];
            acc[c].add(cabs2(u));
            acc[C + c].add(u.x * w.x + u.y * w.y);
        }
    }
    double v[2 * C];
    acc_values(acc, v);
    block_reduce_store<2 * C>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    if (fp.on && last_block(fp.scal0 + inst * S_COUNT, gridDim.x))
        fin_proj_body<1>(partials, gridDim.x * gridDim.y, gridDim.x, F, fp.qe, fp.qn, fp.qt, fp.M0, fp.Mb, fp.scal0,
                      fp.slot_a, fp.slot_b, fp.write_grad_info, blockIdx.y, inst);
}

// out_l = W_l - (alpha + beta l) U_l with (alpha, beta) = scal[ia], scal[ib]; with
// NORM, |out|^2 into scal[norm_slot] (partials, summed by the last block per instance)
template <typename T, int F, bool NORM>
__global__ void __launch_bounds__(256) k_proj_apply(const void* Up, const void* Wp, void* Op, long long G,
                                                    double* scal0, int ia, int ib, double* partials,
                                                    const int* imap, int norm_slot) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(scal0, inst)) return;
    const long long foff = inst * C * G;
    const double* scal = scal0 + inst * S_COUNT;
    const T2* __restrict__ U = reinterpret_cast<const T2*>(Up) + foff;
    const T2* __restrict__ Wv = reinterpret_cast<const T2*>(Wp) + foff;
    T2* __restrict__ O = Op ? reinterpret_cast<T2*>(Op) + foff : nullptr;
    T coef[C];
#pragma unroll
    for (int c = 0; c < C; ++c) coef[c] = T(scal[ia] + scal[ib] * double(F - c));
    Acc<T> acc[1];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const T2 u = U[c * G + p];
            T2 w = Wv[c * G + p];
            caxpy(w, -coef[c], u);
            if (NORM) acc[0].add(cabs2(w));
            if (O) O[c * G + p] = w;
        }
    }
    if (NORM) {
        double v[1];
        acc_values(acc, v);
        block_reduce_store<1>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
        if (last_block(scal0 + inst * S_COUNT, gridDim.x))
            fin_norm_body(partials, gridDim.x * gridDim.y, gridDim.x, scal0, norm_slot, blockIdx.y, inst);
    }
}

// out_l *= scal[S_SIG + l]
template <typename T, int F>
__global__ void __launch_bounds__(256) k_scale(void* Op, long long G, const double* __restrict__ scal0,
                                               const int* imap) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(scal0, inst)) return;
    const long long foff = inst * C * G;
    const double* scal = scal0 + inst * S_COUNT;
    T2* __restrict__ O = reinterpret_cast<T2*>(Op) + foff;
    T s[C];
#pragma unroll
    for (int c = 0; c < C; ++c) s[c] = T(scal[S_SIG + c]);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) O[c * G + p] = cscale(O[c * G + p], s[c]);
    }
}

// Retraction scales sigma_l from m_l = |w_l|^2 (Sec. 6), one block per instance;
// warp 0 solves, lane i holding component i, so each Newton step costs one term
// per lane and a shuffle sum (lane 0's sum is broadcast: every lane takes the
// same decisions).
//  kind 1, Lemma 5.1: r is the zero of h1, increasing on (1/(f1-M), 1/(f2-M))
//    (Eq. hderi); safeguarded Newton from r = 0 (the zero for w on M), bisecting
//    whenever a Newton step leaves the current sign bracket.
//  kind 2, Lemma 5.3: r is the positive zero of h3 = h2 t^{-f1-F}, h3(0) < 0 and
//    h3' > 0 at the zero; bracket from t = 1 by doubling, then the same
//    safeguarded Newton.
//  kind 3, Lemma 5.4: closed form.
// Both iterations stop when h is at the rounding floor of its own terms
// (|h| <= 8 eps sum |terms|: r is the zero to working precision, and further
// steps would only move it within the noise), when the step is below 4 ulps of
// r, or after 200 steps.
__device__ __forceinline__ double warp_sum_bcast(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// three warp sums in one shuffle tree, every lane gets the totals
__device__ __forceinline__ void warp_sum3_bcast(double& a, double& b, double& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    a = __shfl_sync(0xffffffffu, a, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    c = __shfl_sync(0xffffffffu, c, 0);
}

constexpr double kEps = 2.220446049250313e-16;   // 2^-52

__device__ __forceinline__ void retract_solve_body(const double* pa, int na_tot, int na_inst, int F, double M0,
                                                   const double* Mb, int kind, double* scal0, int b, long long inst) {
    __shared__ double m[kMaxC];
    const int C = 2 * F + 1;
    int qs[kMaxC];
    for (int i = 0; i < kMaxC; ++i) qs[i] = i;
    warp_sums(pa, na_tot, b * na_inst, na_inst, qs, C, m);
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double* scal = scal0 + (size_t)inst * S_COUNT;
    const double M = Mb ? Mb[inst] : M0;
    // f2 = largest l with w_l != 0 (component index i1), f1 = smallest (index i2)
    int i1 = -1, i2 = -1;
    for (int i = 0; i < C; ++i)
        if (m[i] > 0.0) { if (i1 < 0) i1 = i; i2 = i; }
    bool ok = (i1 >= 0);
    const double f2 = ok ? double(F - i1) : 0.0, f1 = ok ? double(F - i2) : 0.0;
    const bool mine = lane < C;
    const double ml = mine ? m[lane] : 0.0;
    const double l = double(F - lane);
    double sig = 0.0;
    if (kind == 3) {
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < C; ++i) { const double li = double(F - i); a += m[i]; b += li * m[i]; c += li * li * m[i]; }
        const double den = a * c - b * b;
        const double num = c - (M + l) * b + M * l * a;
        const bool good = !mine || (num > 0.0 && den > 0.0);
        ok = ok && (__all_sync(0xffffffffu, good) != 0);
        if (ok && mine) sig = sqrt(num / den);
    } else if (ok && f1 < M && M < f2) {
        const bool act = mine && lane >= i1 && lane <= i2;
        if (kind == 1) {
            const double d = l - M;
            double lo = 1.0 / (f1 - M), hi = 1.0 / (f2 - M);   // h1(lo+) = -inf, h1(hi-) = +inf
            double r = 0.0;
            for (int it = 0; it < 200; ++it) {
                double h = 0.0, dh = 0.0, habs = 0.0;
                if (act) {
                    const double iq = 1.0 / (1.0 - d * r);
                    h = d * ml * iq * iq;
                    dh = 2.0 * d * h * iq;
                    habs = fabs(h);
                }
                warp_sum3_bcast(h, dh, habs);
                if (fabs(h) <= 8.0 * kEps * habs) break;
                if (h < 0.0) lo = r; else if (h > 0.0) hi = r; else break;
                // a Newton step below 4 ulps of r ends the iteration (tested before the
                // bracket, which a converged step may no longer clear)
                const double dr = (dh > 0.0) ? h / dh : 0.0;
                if (dh > 0.0 && fabs(dr) <= 4.0 * kEps * fmax(fabs(r), 1e-300)) {
                    r -= dr;
                    break;
                }
                double rn = (dh > 0.0) ? r - dr : 0.5 * (lo + hi);
                if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
                const double step = fabs(rn - r);
                r = rn;
                if (step <= 4.0 * kEps * fmax(fabs(r), 1e-300)) break;
            }
            const double q = 1.0 - d * r;
            const double sv = warp_sum_bcast(act ? ml / (q * q) : 0.0);
            if (act) sig = 1.0 / (sqrt(sv) * q);
        } else {
            // h3(t) = sum_j (j + f1 - M) m_{f1+j} t^j, j = l - f1, over the components in [f1, f2]
            const int j = int(l - f1);
            const double cf = act ? (double(j) + f1 - M) * ml : 0.0;
            // h3(t), h3'(t) and sum |terms| in habs
            auto h3 = [&](double t, double* dh, double* habs) {
                double tp = 1.0, tpm = 0.0;          // t^j and t^(j-1)
                for (int k = 0; k < j; ++k) { tpm = tp; tp *= t; }
                double v = act ? cf * tp : 0.0;
                *dh = act && j > 0 ? double(j) * cf * tpm : 0.0;
                *habs = fabs(v);
                warp_sum3_bcast(v, *dh, *habs);
                return v;
            };
            double dh, habs;
            double lo = 0.0, hi = 1.0;
            int guard = 0;
            if (h3(1.0, &dh, &habs) < 0.0) {
                lo = 1.0; hi = 2.0;
                while (h3(hi, &dh, &habs) < 0.0 && guard++ < 2000) { lo = hi; hi *= 2.0; }
            }
            if (guard >= 2000) ok = false;
            double r = (lo > 0.0) ? lo : 1.0;
            for (int it = 0; it < 200 && ok; ++it) {
                const double h = h3(r, &dh, &habs);
                if (fabs(h) <= 8.0 * kEps * habs) break;
                if (h < 0.0) lo = r; else if (h > 0.0) hi = r; else break;
                if (dh > 0.0 && fabs(h / dh) <= 4.0 * kEps * r) {
                    r -= h / dh;
                    break;
                }
                double rn = (dh > 0.0) ? r - h / dh : 0.5 * (lo + hi);
                if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
                const double step = fabs(rn - r);
                r = rn;
                if (step <= 4.0 * kEps * r) break;
            }
            // sigma_0^2 = 1 / sum_l m_l r^l, sigma_l = sigma_0 r^{l/2}
            const int L = F - lane;
            const int al = L > 0 ? L : -L;
            const double base = L > 0 ? r : 1.0 / r, sbase = L > 0 ? sqrt(r) : 1.0 / sqrt(r);
            double p = 1.0, ps = 1.0;
            for (int k = 0; k < al; ++k) { p *= base; ps *= sbase; }
            const double ssum = warp_sum_bcast(mine ? ml * p : 0.0);
            if (mine) sig = sqrt(1.0 / ssum) * ps;
        }
    } else {
        ok = false;
    }
    const bool fin = !mine || isfinite(sig);
    ok = ok && (__all_sync(0xffffffffu, fin) != 0);
    if (lane < kMaxC) scal[S_SIG + lane] = mine ? sig : 0.0;
    if (lane == 0 && !ok) set_status(scal, SBEC_ERR_DOMAIN);
}

// w = U + t Xi into out; partials m_l = |w_l|^2, from which the last block per
// instance solves for the retraction scales sigma_l (retract_solve_body)
template <typename T, int F>
__global__ void __launch_bounds__(256) k_retract_w(const void* Up, const void* Xp, double t, void* Op, long long G,
                                                   double* partials, double* scal0, int tslot, const int* imap,
                                                   int kind, double M0, const double* Mb) {
    using T2 = typename C2<T>::t;
    constexpr int C = 2 * F + 1;
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(scal0, inst)) return;
    const long long foff = inst * C * G;
    if (tslot >= 0) t *= scal0[(size_t)inst * S_COUNT + tslot];
    const T2* __restrict__ U = reinterpret_cast<const T2*>(Up) + foff;
    const T2* __restrict__ Xi = reinterpret_cast<const T2*>(Xp) + foff;
    T2* __restrict__ O = reinterpret_cast<T2*>(Op) + foff;
    Acc<T> acc[C];
    const T tt = T(t);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            T2 w = U[c * G + p];
            caxpy(w, tt, Xi[c * G + p]);
            acc[c].add(cabs2(w));
            O[c * G + p] = w;
        }
    }
    double v[C];
    acc_values(acc, v);
    block_reduce_store<C>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    if (last_block(scal0 + inst * S_COUNT, gridDim.x))
        retract_solve_body(partials, gridDim.x * gridDim.y, gridDim.x, F, M0, Mb, kind, scal0, blockIdx.y, inst);
}


// ---------------------------------------------------------------------------
// Tangent-vector BLAS-1 (Sec. 4 inner product <xi, zeta>_u = xi^T zeta on the real
// stacking, Eq. prod): fields are treated as 2 C G reals.  Dots go to per-block
// partials (fixed order); coefficients are read from the scalar block so that a
// sequence of updates needs no host round trip.
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_lincomb(const Lin L, long long N, const double* __restrict__ scal0,
                                                 double* partials, const int* imap) {
    // out may alias A, B, D1 or D2 (same index only), so no __restrict__ here;
    // blockIdx.y is the launch slot of the instance, N the reals per instance
    const long long inst = inst_of(imap, blockIdx.y);
    const long long off = inst * N;
    const double* scal = scal0 + (size_t)inst * S_COUNT;
    if (skipped(scal0, inst)) return;
    const T* A = reinterpret_cast<const T*>(L.A) + off;
    const T* B = L.B ? reinterpret_cast<const T*>(L.B) + off : nullptr;
    const T* D1 = L.D1 ? reinterpret_cast<const T*>(L.D1) + off : nullptr;
    const T* D2 = L.D2 ? reinterpret_cast<const T*>(L.D2) + off : nullptr;
    T* O = reinterpret_cast<T*>(L.out) + off;
    const bool self1 = (L.D1 == L.out), self2 = (L.D2 == L.out);
    double ca = L.ca, cb = L.cb;
    if (L.ia >= 0) ca *= scal[L.ia];
    if (L.ib >= 0) cb *= scal[L.ib];
    const bool upd = (L.guard < 0) || (scal[L.guard] != 0.0);
    const T a = T(ca), b = T(cb);
    Acc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        T v;
        if (upd) {
            v = a * A[i];
            if (B) v += b * B[i];
            O[i] = v;
        } else {
            v = O[i];
        }
        if (D1) acc[0].add(v * (self1 ? v : D1[i]));
        if (D2) acc[1].add(v * (self2 ? v : D2[i]));
    }
    if (partials) {
        double r[2];
        acc_values(acc, r);
        block_reduce_store<2>(r, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    }
}

// partials q0 = <A, B>, q1 = <C, D> (C null: skip)
template <typename T>
__global__ void __launch_bounds__(256) k_dot2(const void* Ap, const void* Bp, const void* Cp, const void* Dp,
                                              long long N, double* partials, const double* skip, const int* imap) {
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(skip, inst)) return;
    const long long off = inst * N;
    const T* __restrict__ A = reinterpret_cast<const T*>(Ap) + off;
    const T* __restrict__ B = reinterpret_cast<const T*>(Bp) + off;
    const T* __restrict__ Cv = Cp ? reinterpret_cast<const T*>(Cp) + off : nullptr;
    const T* __restrict__ D = Dp ? reinterpret_cast<const T*>(Dp) + off : nullptr;
    Acc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        acc[0].add(A[i] * B[i]);
        if (Cv) acc[1].add(Cv[i] * D[i]);
    }
    double v[2];
    acc_values(acc, v);
    block_reduce_store<2>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// partials q0 = <u - up, g - gp>, q1 = |g - gp|^2 (the BB quantities s^T v, v^T v)
template <typename T>
__global__ void __launch_bounds__(256) k_bbdots(const void* Up, const void* UPp, const void* Gp, const void* GPp,
                                                long long N, double* partials, const double* skip, const int* imap) {
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(skip, inst)) return;
    const long long off = inst * N;
    const T* __restrict__ U = reinterpret_cast<const T*>(Up) + off;
    const T* __restrict__ UP = reinterpret_cast<const T*>(UPp) + off;
    const T* __restrict__ G = reinterpret_cast<const T*>(Gp) + off;
    const T* __restrict__ GP = reinterpret_cast<const T*>(GPp) + off;
    Acc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const T sv = U[i] - UP[i];
        const T vv = G[i] - GP[i];
        acc[0].add(sv * vv);
        acc[1].add(vv * vv);
    }
    double v[2];
    acc_values(acc, v);
    block_reduce_store<2>(v, partials, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// scal[slot + q] = sum of partial quantity q, q = 0..nq-1 (nq <= 2), per instance
static __global__ void k_fin_sums(const double* pa, int na_tot, int na_inst, int nq, double* scal0, int slot,
                                  const int* imap) {
    const long long inst = inst_of(imap, blockIdx.x);
    if (skipped(scal0, inst)) return;
    __shared__ double v[2];
    const int qs[2] = {0, 1};
    warp_sums(pa, na_tot, blockIdx.x * na_inst, na_inst, qs, nq, v);
    if (threadIdx.x == 0) {
        double* scal = scal0 + (size_t)inst * S_COUNT;
        for (int q = 0; q < nq; ++q) {
            scal[slot + q] = v[q];
            if (!isfinite(v[q])) set_status(scal, SBEC_ERR_NONFINITE);
        }
    }
}

// Modified-CG iteration, fused (Sec. 5, Eq. prob-lsub, the CG of the ARNT subproblem).
// k_cg_curv: partials <p, Hp>, <p, p>; the last block per instance stores them and the
// guarded step alpha = <r,r> / <p,Hp> (alpha = 0 and guard 0 when <p,Hp> <= 1e-12 <p,p>).
template <typename T>
__global__ void __launch_bounds__(256) k_cg_curv(const void* Pp, const void* Hpp, long long N, double* partials,
                                                 double* scal0, const int* imap, const CgSlots cs) {
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(scal0, inst)) return;
    const long long off = inst * N;
    const T* __restrict__ P = reinterpret_cast<const T*>(Pp) + off;
    const T* __restrict__ H = reinterpret_cast<const T*>(Hpp) + off;
    Acc<T> acc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const T pi = P[i];
        acc[0].add(pi * H[i]);
        acc[1].add(pi * pi);
    }
    double v[2];
    acc_values(acc, v);
    const int ntot = gridDim.x * gridDim.y;
    block_reduce_store<2>(v, partials, ntot, blockIdx.y * gridDim.x + blockIdx.x);
    double* scal = scal0 + (size_t)inst * S_COUNT;
    if (!last_block(scal, gridDim.x)) return;
    __shared__ double sums[2];
    const int qs[2] = {0, 1};
    warp_sums(partials, ntot, blockIdx.y * gridDim.x, gridDim.x, qs, 2, sums);
    if (threadIdx.x == 0) {
        const double kap = sums[0], pp = sums[1];
        scal[cs.kap] = kap;
        scal[cs.kap + 1] = pp;
        if (!isfinite(kap) || !isfinite(pp)) set_status(scal, SBEC_ERR_NONFINITE);
        const bool ok = kap > 1e-12 * pp;
        scal[cs.alpha] = ok ? scal[cs.rr_now] / kap : 0.0;
        scal[cs.alpha + 1] = ok ? 1.0 : 0.0;
    }
}

// k_cg_update: x += alpha p and r -= alpha Hp (when the step's guard holds), partials
// <r,r>; the last block per instance stores <r,r> and takes the CG's decision: count
// the iteration; end the CG on curvature <p,Hp> <= 1e-12 <p,p> (recording sigma_est =
// |<p,Hp>| / <p,p> and which direction Eq. (xi) takes), on ||r|| <= the threshold or at
// the iteration cap; otherwise beta = <r',r'> / <r,r>.  An instance whose CG ends is
// switched off (S_SKIP), so the rest of its chunk leaves it alone.
template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(void* Xp, void* Rp, const void* Pp, const void* Hpp, long long N,
                                                   double* partials, double* scal0, const int* imap,
                                                   const CgSlots cs) {
    const long long inst = inst_of(imap, blockIdx.y);
    if (skipped(scal0, inst)) return;
    const long long off = inst * N;
    double* scal = scal0 + (size_t)inst * S_COUNT;
    T* __restrict__ X = reinterpret_cast<T*>(Xp) + off;
    T* __restrict__ R = reinterpret_cast<T*>(Rp) + off;
    const T* __restrict__ P = reinterpret_cast<const T*>(Pp) + off;
    const T* __restrict__ H = reinterpret_cast<const T*>(Hpp) + off;
    const bool upd = scal[cs.alpha + 1] != 0.0;
    const T a = T(scal[cs.alpha]), na = T(-scal[cs.alpha]);
    Acc<T> acc[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        T ri = R[i];
        if (upd) {
            X[i] = fma(a, P[i], X[i]);
            ri = fma(na, H[i], ri);
            R[i] = ri;
        }
        acc[0].add(ri * ri);
    }
    double v[1];
    acc_values(acc, v);
    const int ntot = gridDim.x * gridDim.y;
    block_reduce_store<1>(v, partials, ntot, blockIdx.y * gridDim.x + blockIdx.x);
    if (!last_block(scal, gridDim.x)) return;
    __shared__ double sums[1];
    const int qs[1] = {0};
    warp_sums(partials, ntot, blockIdx.y * gridDim.x, gridDim.x, qs, 1, sums);
    if (threadIdx.x == 0) {
        const double rrn = sums[0];
        scal[cs.rr_next] = rrn;
        if (!isfinite(rrn)) set_status(scal, SBEC_ERR_NONFINITE);
        const double kap = scal[cs.kap], pp = scal[cs.kap + 1];
        const double j = scal[cs.j] + 1.0;
        scal[cs.j] = j;
        bool done;
        if (kap <= 1e-12 * pp) {
            scal[cs.sest] = fabs(kap) / pp;
            if (j == 1.0) scal[cs.cgneg] = 1.0;
            else if (kap < -1e-12 * pp) scal[cs.cghd] = 1.0;
            done = true;
        } else if (sqrt(rrn) <= scal[cs.stop]) {
            done = true;
        } else {
            scal[cs.beta] = rrn / scal[cs.rr_now];
            done = j >= scal[cs.maxin];
        }
        if (done) {
            scal[cs.cg] = 0.0;
            scal[S_SKIP] = cs.skip_val;
        }
    }
}

// scal[dst] = scal[num] / scal[den] when the guard holds, else 0  (CG alpha), per
// instance; scal[dst + 1] is the guard flag of the guarded updates
static __global__ void k_ratio(double* scal0, int dst, int num, int den, int guard_kap, int guard_pp, double eps,
                               int mask, const int* imap) {
    const long long inst = inst_of(imap, blockIdx.x);
    if (threadIdx.x != 0 || skipped(scal0, inst)) return;
    double* scal = scal0 + (size_t)inst * S_COUNT;
    bool ok = (mask < 0) || (scal[mask] != 0.0);
    if (guard_kap >= 0) ok = ok && scal[guard_kap] > eps * scal[guard_pp];
    scal[dst] = ok ? scal[num] / scal[den] : 0.0;
    scal[dst + 1] = ok ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// Cascadic prolongation (Algorithm 1, "refine uniformly"): the coarse spectrum
// is zero-padded to the fine grid; the coarse Nyquist coefficient (p = -n_c/2)
// is split evenly between p = +-n_c/2 of the fine grid on every refined axis.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad_map(int i_f, int nc, int nf, double* wgt) {
    if (nc == nf) { *wgt = 1.0; return i_f; }
    const int h = nc >> 1;
    if (i_f < h) { *wgt = 1.0; return i_f; }
    if (i_f == h || i_f == nf - h) { *wgt = 0.5; return h; }
    if (i_f > nf - h) { *wgt = 1.0; return i_f - nf + nc; }
    *wgt = 0.0;
    return 0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_pad(const void* srcp, void* dstp, int C, int ncx, int ncy, int ncz,
                                             int nfx, int nfy, int nfz, double scale) {
    using T2 = typename C2<T>::t;
    const T2* __restrict__ src = reinterpret_cast<const T2*>(srcp);
    T2* __restrict__ dst = reinterpret_cast<T2*>(dstp);
    const long long Gf = (long long)nfx * nfy * nfz, Gc = (long long)ncx * ncy * ncz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)C * Gf;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / Gf);
        const long long p = i - (long long)c * Gf;
        const int ix = (int)(p % nfx), iy = (int)((p / nfx) % nfy), iz = (int)(p / ((long long)nfx * nfy));
        double wx, wy, wz;
        const int jx = pad_map(ix, ncx, nfx, &wx), jy = pad_map(iy, ncy, nfy, &wy), jz = pad_map(iz, ncz, nfz, &wz);
        const double wgt = wx * wy * wz * scale;
        T2 v = mk<T2>(0, 0);
        if (wgt != 0.0) v = cscale(src[(long long)c * Gc + ((long long)jz * ncy + jy) * ncx + jx], T(wgt));
        dst[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_twiddles(void* twp, int n) {
    using T2 = typename C2<T>::t;
    T2* tw = reinterpret_cast<T2*>(twp);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * double(m) / double(n), &s, &c);
        tw[m] = mk<T2>(T(c), T(s));
    }
}

template <typename T>
__global__ void k_harmonic(void* Vp, int nx, int ny, int nz, double x0, double hx, double y0, double hy, double z0,
                           double hz, int dim) {
    T* V = reinterpret_cast<T*>(Vp);
    const long long G = (long long)nx * ny * nz;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
        const int ix = int(p % nx), iy = int((p / nx) % ny), iz = int(p / ((long long)nx * ny));
        const double x = x0 + hx * ix, y = y0 + hy * iy, z = z0 + hz * iz;
        double v = x * x;
        if (dim >= 2) v += y * y;
        if (dim >= 3) v += z * z;
        V[p] = T(0.5 * v);
    }
}

template <typename T>
__global__ void k_convert(void* Vp, const double* Vd, long long G) {
    T* V = reinterpret_cast<T*>(Vp);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x)
        V[p] = T(Vd[p]);
}

// ---------------------------------------------------------------------------
// Launch configuration
// ---------------------------------------------------------------------------
// two: the pass runs the two-level FFT kernel (k_xpass2 / k_spass2) of length 2^logn
struct XCfg { int rpb, nth, items, nblk, nblk_inst, two, logn; size_t smem; };
struct SCfg { int W, nth, items, nblk, nblk_inst, two, logn; size_t smem; };
constexpr int kMaxLogn2 = 8;   // longest two-level FFT: 256 points

// Limits of the launch shapes: at most 4096 butterflies per block (512 threads x 8
// items) and the opt-in dynamic shared memory of one block.
constexpr int kMaxPointsPerBlock = 16384;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr int kMaxElemPerSm = 32;

template <typename T>
static size_t xsmem(int P, int n) {
    return (size_t)(P * n + ((P * n) >> 3) + 1) * sizeof(typename C2<T>::t);   // padded slots (smem_slot)
}

// x pass: one block = rpb grid rows (x lines) of all C components of one instance
template <typename T>
static XCfg xcfg(const Geom& g) {
    const int n = g.n[0];
    const long long rows_inst = g.G / n;
    if (g.dim > 1 && g.logn[0] >= 1 && g.logn[0] <= kMaxLogn2) {
        // two-level FFT: N1 threads per row, all C components of rpb rows per block
        const int lg = g.logn[0];
        const int N1 = 1 << ((lg + 1) / 2), N2 = n / N1;
        int rpb = 1;
        if (g.tune.x_rows > 0) {
            rpb = g.tune.x_rows;
        } else {
            while ((long long)rpb * 2 * g.C * N1 <= 256 && rows_inst % (rpb * 2) == 0) rpb *= 2;
        }
        XCfg c;
        c.two = 1; c.logn = lg; c.rpb = rpb; c.items = 0;
        c.nth = ((rpb * g.C * N1 + 31) / 32) * 32;
        c.nblk_inst = (int)(rows_inst / rpb);
        c.nblk = c.nblk_inst * g.nl;
        c.smem = (size_t)rpb * g.C * N2 * (N1 + 1) * sizeof(typename C2<T>::t);
        return c;
    }
    int rpb = 1;
    if (g.tune.x_rows > 0) {
        rpb = g.tune.x_rows;
    } else {
        while ((long long)rpb * 2 * g.C * n <= 2048 && rows_inst % (rpb * 2) == 0) rpb *= 2;
    }
    const int P = rpb * g.C;
    const int bfly = (n >= 4) ? P * n / 4 : P;
    int nth = ((bfly + 31) / 32) * 32;
    if (nth > 512) nth = 512;
    if (nth < 64) nth = 64;
    int items = (bfly + nth - 1) / nth;
    int it2 = 1;
    while (it2 < items) it2 *= 2;
    XCfg c;
    c.two = 0; c.logn = g.logn[0];
    c.rpb = rpb; c.nth = nth; c.items = it2;
    c.nblk_inst = (int)(rows_inst / rpb);
    c.nblk = c.nblk_inst * g.nl;
    c.smem = xsmem<T>(P, n);
    return c;
}

// strided pass: one block = W consecutive x columns of one component of one instance
template <typename T>
static SCfg scfg(const Geom& g, int axis, int num_sms) {
    using T2 = typename C2<T>::t;
    const int n = g.n[axis];
    const int nx = g.n[0];
    const long long outer = (axis == 1) ? g.n[2] : g.n[1];
    int W = (sizeof(T) == 8) ? 8 : 16;
    if (g.tune.s_pencils[axis] > 0) {
        W = g.tune.s_pencils[axis];
    } else {
        if (W > nx) W = nx;
        // prefer at least 4 blocks per SM when the grid is small
        while (W > 2 && (long long)g.B * g.C * outer * (nx / W) < 4LL * num_sms) W >>= 1;
    }
    const int lg = g.logn[axis];
    if (lg >= 1 && lg <= kMaxLogn2) {
        // two-level FFT: N1 threads per pencil, whole warps, at most 256 threads
        // (k_spass2's launch bound: two such blocks per SM)
        const int N1 = 1 << ((lg + 1) / 2), N2 = n / N1;
        if ((W * N1) % 32 == 0 && W * N1 <= 256) {
            SCfg c;
            c.two = 1; c.logn = lg; c.W = W; c.nth = W * N1; c.items = 0;
            c.nblk_inst = (int)((long long)g.C * outer * (nx / W));
            c.nblk = c.nblk_inst * g.nl;
            c.smem = (size_t)N2 * (N1 * W + (W < 16 ? W : 0)) * sizeof(T2);
            return c;
        }
    }
    const int bfly = (n >= 4) ? W * n / 4 : W;
    const int split = g.tune.s_split[axis] > 0 ? g.tune.s_split[axis] : 1;
    int nth = ((bfly / split + 31) / 32) * 32;
    if (nth > 512) nth = 512;
    if (nth < 64) nth = 64;
    int items = (bfly + nth - 1) / nth;
    int it2 = 1;
    while (it2 < items) it2 *= 2;
    SCfg c;
    c.two = 0; c.logn = lg;
    c.W = W; c.nth = nth; c.items = it2;
    c.nblk_inst = (int)((long long)g.C * outer * (nx / W));
    c.nblk = c.nblk_inst * g.nl;
    c.smem = (size_t)W * n * sizeof(T2);
    return c;
}

// blocks per instance of the grid-stride elementwise kernels (from the batch size B,
// not from the number of instances a launch covers, so that every instance's
// partial sums have the same order whichever instances run alongside it)
static int elem_blocks(long long G, int num_sms, int B = 1, int per_sm = 0) {
    long long b = (G + 255) / 256;
    long long cap = (long long)(per_sm > 0 ? per_sm : 8) * num_sms / (B > 0 ? B : 1);
    if (cap < 1) cap = 1;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// Resident 256-thread blocks per SM of a grid-stride kernel, asked once per
// kernel (cache: a static of the call site); -1 when the runtime cannot tell.
template <typename K>
static int resident_256(K kern, std::atomic<int>& cache) {
    int n = cache.load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, 0) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = -1;
        }
        cache.store(n, std::memory_order_relaxed);
    }
    return n;
}

// Grid of a grid-stride kernel over n points per instance: elem_blocks, rounded
// down to whole waves of the kernel's resident blocks when it spans more than one
// (8 blocks per SM over a kernel of which 6 fit would run a second, one-third-full
// wave: 6 are launched).  Measured on the 256^3 FP32 fields: the one-third wave
// cost the projection 25%; a kernel of which 4 fit keeps its two full waves, which
// took 40% less time than one wave of blocks with twice the work each.
static int elem_grid(long long n, const Geom& g, const Work& w, int resident) {
    const int nb = elem_blocks(n, w.num_sms, g.B, g.tune.elem_per_sm);
    if (resident <= 0) return nb;
    const long long wave = (long long)resident * w.num_sms / (g.B > 0 ? g.B : 1);
    if (wave < 1 || nb <= wave) return nb;
    return (int)((nb / wave) * wave);
}
#define SBEC_ELEM_GRID(n, kern)                                         \
    [&]() {                                                             \
        static std::atomic<int> occ_{0};                                \
        return elem_grid((n), g, w, resident_256(kern, occ_));          \
    }()

static PointParams point_params(const Geom& g) {
    PointParams pp;
    for (int i = 0; i < kMaxC; ++i) pp.bz[i] = g.bz[i];
    pp.g0 = g.g0; pp.g1 = g.g1; pp.g2 = g.g2; pp.g3 = g.g3;
    pp.e0 = g.e0; pp.e1 = g.e1; pp.e2 = g.e2; pp.e3 = g.e3;
    return pp;
}

// Dynamic shared memory above the default carve-out needs an opt-in per kernel;
// the static shared memory of the reductions comes on top, so opt in above
// 32 KB.  `granted` is the caller's per-kernel record of the size already set.
template <typename K>
static int ensure_smem(K kern, size_t bytes, size_t& granted) {
    if (bytes > 32 * 1024 && bytes > granted) {
        SBEC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        granted = bytes;
    }
    return SBEC_OK;
}

template <int MODE> struct XKid {
    static constexpr int v = MODE == X_FWD ? K_X_FWD : MODE == X_FWD_EPW ? K_X_FWD_EPW
                           : MODE == X_INV_GRAD ? K_X_INV_GRAD : MODE == X_INV_HESS ? K_X_INV_HESS
                           : MODE == X_FULL_GRAD ? K_X_FULL_GRAD : MODE == X_FULL_ENERGY ? K_X_FULL_ENERGY
                           : MODE == X_FULL_HESS ? K_X_FULL_HESS : K_X_INV;
};
template <int MODE> struct SKid {
    static constexpr int v = MODE == S_FWD ? K_S_FWD : MODE == S_INV ? K_S_INV : MODE == S_K2 ? K_S_K2 : K_S_PARSEVAL;
};

template <typename T, int F, int MODE, int ITEMS>
static int launch_x_items(const XCfg& c, const XArgs& a, const Work& w, cudaStream_t s) {
    auto kern = k_xpass<T, F, MODE, ITEMS>;
    static size_t granted = 0;
    if (int st = ensure_smem(kern, c.smem, granted)) return st;
    ProfScope ps(w.prof, XKid<MODE>::v, s);
    kern<<<c.nblk, c.nth, c.smem, s>>>(a);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T, int F, int MODE, int LOGN>
static int launch_x2(const XCfg& c, const XArgs& a, const Work& w, cudaStream_t s) {
    auto kern = k_xpass2<T, F, MODE, LOGN>;
    static size_t granted = 0;
    if (int st = ensure_smem(kern, c.smem, granted)) return st;
    ProfScope ps(w.prof, XKid<MODE>::v, s);
    kern<<<c.nblk, c.nth, c.smem, s>>>(a);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T, int F, int MODE>
static int launch_x(const XCfg& c, const XArgs& a, const Work& w, cudaStream_t s) {
    if constexpr (MODE == X_FWD || MODE == X_FWD_EPW || MODE == X_INV) {
        if (c.two) {
            switch (c.logn) {
                case 1: return launch_x2<T, F, MODE, 1>(c, a, w, s);
                case 2: return launch_x2<T, F, MODE, 2>(c, a, w, s);
                case 3: return launch_x2<T, F, MODE, 3>(c, a, w, s);
                case 4: return launch_x2<T, F, MODE, 4>(c, a, w, s);
                case 5: return launch_x2<T, F, MODE, 5>(c, a, w, s);
                case 6: return launch_x2<T, F, MODE, 6>(c, a, w, s);
                case 7: return launch_x2<T, F, MODE, 7>(c, a, w, s);
                case 8: return launch_x2<T, F, MODE, 8>(c, a, w, s);
                default: return SBEC_ERR_ARG;
            }
        }
    } else {
        if (c.two) return SBEC_ERR_ARG;
    }
    switch (c.items) {
        case 1: return launch_x_items<T, F, MODE, 1>(c, a, w, s);
        case 2: return launch_x_items<T, F, MODE, 2>(c, a, w, s);
        case 4: return launch_x_items<T, F, MODE, 4>(c, a, w, s);
        case 8: return launch_x_items<T, F, MODE, 8>(c, a, w, s);
        default: return SBEC_ERR_ARG;
    }
}

template <typename T, int MODE, int ITEMS>
static int launch_s_items(const SCfg& c, const SArgs& a, const Work& w, cudaStream_t s) {
    auto kern = k_spass<T, MODE, ITEMS>;
    static size_t granted = 0;
    if (int st = ensure_smem(kern, c.smem, granted)) return st;
    ProfScope ps(w.prof, SKid<MODE>::v, s);
    kern<<<c.nblk, c.nth, c.smem, s>>>(a);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T, int MODE, int LOGN>
static int launch_s2(const SCfg& c, const SArgs& a, const Work& w, cudaStream_t s) {
    auto kern = k_spass2<T, MODE, LOGN>;
    static size_t granted = 0;
    if (int st = ensure_smem(kern, c.smem, granted)) return st;
    ProfScope ps(w.prof, SKid<MODE>::v, s);
    kern<<<c.nblk, c.nth, c.smem, s>>>(a);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T, int MODE>
static int launch_s(const SCfg& c, const SArgs& a, const Work& w, cudaStream_t s) {
    if (c.two) {
        switch (c.logn) {
            case 1: return launch_s2<T, MODE, 1>(c, a, w, s);
            case 2: return launch_s2<T, MODE, 2>(c, a, w, s);
            case 3: return launch_s2<T, MODE, 3>(c, a, w, s);
            case 4: return launch_s2<T, MODE, 4>(c, a, w, s);
            case 5: return launch_s2<T, MODE, 5>(c, a, w, s);
            case 6: return launch_s2<T, MODE, 6>(c, a, w, s);
            case 7: return launch_s2<T, MODE, 7>(c, a, w, s);
            case 8: return launch_s2<T, MODE, 8>(c, a, w, s);
            default: return SBEC_ERR_ARG;
        }
    }
    switch (c.items) {
        case 1: return launch_s_items<T, MODE, 1>(c, a, w, s);
        case 2: return launch_s_items<T, MODE, 2>(c, a, w, s);
        case 4: return launch_s_items<T, MODE, 4>(c, a, w, s);
        case 8: return launch_s_items<T, MODE, 8>(c, a, w, s);
        default: return SBEC_ERR_ARG;
    }
}

// ---------------------------------------------------------------------------
// TMA strided passes (FP32 single-instance fields, pass axis of 128 or 256 points)
// ---------------------------------------------------------------------------
// cuTensorMapEncodeTiled fetched from the driver at run time (the library links
// the runtime only); null when the driver does not provide it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tma_encoder() {
    static std::atomic<int> state{0};            // 0 unknown, 1 available, -1 unavailable
    static std::atomic<EncodeTiledFn> fn{nullptr};
    int st = state.load(std::memory_order_acquire);
    if (st == 0) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p) {
            fn.store(reinterpret_cast<EncodeTiledFn>(p), std::memory_order_release);
            st = 1;
        } else {
            cudaGetLastError();
            st = -1;
        }
        state.store(st, std::memory_order_release);
    }
    return st == 1 ? fn.load(std::memory_order_acquire) : nullptr;
}

// The field at `base` as a 4D float tensor [C][n_z][n_y][2 n_x] with a box of one
// tile of the pass along `axis` (2W floats along x, the whole axis).
static bool tma_map(CUtensorMap* m, const void* base, const Geom& g, int axis, int W) {
    EncodeTiledFn enc = tma_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t nx2 = 2ull * (cuuint64_t)g.n[0];
    const cuuint64_t dims[4] = {nx2, (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)g.C};
    const cuuint64_t strides[3] = {nx2 * 4, nx2 * g.n[1] * 4, nx2 * g.n[1] * g.n[2] * 4};
    const cuuint32_t box[4] = {2u * (cuuint32_t)W, axis == 1 ? (cuuint32_t)g.n[1] : 1u,
                               axis == 2 ? (cuuint32_t)g.n[2] : 1u, 1u};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA tile width of a pass with launch shapes t (0: not a TMA shape): s_split =
// kTmaSplit with s_pencils 8, 16 or 32, or both 0 (the built-in choice: 8 columns
// on the last axis, whose fused fwd·|k|²·inv and Parseval passes were measured
// fastest at four blocks per SM, 16 on the middle axis of a 3D problem)
static int tma_width(const Tune& t, int axis, int dim) {
    const int W = t.s_pencils[axis], sp = t.s_split[axis];
    const int wdef = axis == dim - 1 ? 8 : 16;
    if (W == 0 && sp == 0) return wdef;
    if (sp != kTmaSplit) return 0;
    return (W == 8 || W == 16 || W == 32) ? W : (W == 0 ? wdef : 0);
}

// the pass's TMA tile width, or 0 where the pass does not run on the TMA kernel:
// FP32, one instance, a TMA shape, a pass axis of 128 or 256 points and x a
// multiple of the tile width
template <typename T>
static int tma_pass(const Geom& g, int axis) {
    if (sizeof(T) != 4 || g.B != 1 || g.nl != 1 || g.imap || g.dim < 2) return 0;
    if (g.n[axis] != 128 && g.n[axis] != 256) return 0;
    const int W = tma_width(g.tune, axis, g.dim);
    if (W == 0 || g.n[0] % W != 0) return 0;
    return tma_encoder() != nullptr ? W : 0;
}

template <int MODE, int LOGN, int W>
static int launch_tma_n(const Geom& g, const SArgs& a, const Work& w, cudaStream_t s) {
    auto kern = k_spass_tma<MODE, LOGN, W>;
    constexpr size_t smem = tma_smem_bytes<LOGN, W>();
    constexpr int nth = W * Split2<LOGN>::N1;
    static size_t granted = 0;
    if (int st = ensure_smem(kern, smem, granted)) return st;
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nth, smem) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        occ.store(per_sm, std::memory_order_relaxed);
    }
    CUtensorMap mi, mo;
    if (!tma_map(&mi, a.in, g, a.axis, W)) return SBEC_ERR_CUDA;
    if (!tma_map(&mo, a.out ? a.out : a.in, g, a.axis, W)) return SBEC_ERR_CUDA;
    TmaArgs ta;
    ta.s = a;
    ta.ntiles = (long long)g.C * a.nouter * a.ntx;
    ta.status = w.scal;
    long long grid = (long long)w.num_sms * per_sm;
    if (grid > ta.ntiles) grid = ta.ntiles;
    ProfScope ps(w.prof, SKid<MODE>::v, s);
    kern<<<(int)grid, nth, smem, s>>>(ta, mi, mo);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

// strided pass along a.axis: the TMA kernel where it applies, else the
// two-level / Stockham kernels
template <typename T, int MODE>
static int launch_pass(const Geom& g, const SCfg& c, const SArgs& a, const Work& w, cudaStream_t s) {
    if (const int W = tma_pass<T>(g, a.axis)) {
        SArgs b = a;
        b.W = W;
        b.ntx = g.n[0] / W;
        const bool n256 = g.n[a.axis] == 256;
        switch (W) {
            case 8: return n256 ? launch_tma_n<MODE, 8, 8>(g, b, w, s) : launch_tma_n<MODE, 7, 8>(g, b, w, s);
            case 16: return n256 ? launch_tma_n<MODE, 8, 16>(g, b, w, s) : launch_tma_n<MODE, 7, 16>(g, b, w, s);
            default: return n256 ? launch_tma_n<MODE, 8, 32>(g, b, w, s) : launch_tma_n<MODE, 7, 32>(g, b, w, s);
        }
    }
    return launch_s<T, MODE>(c, a, w, s);
}

// launch of an elementwise / finalize kernel with bookkeeping
#define SBEC_LAUNCH(kid, kern, grid, block, ...)            \
    do {                                                    \
        ProfScope ps_(w.prof, kid, s);                      \
        kern<<<grid, block, 0, s>>>(__VA_ARGS__);           \
        SBEC_LAUNCH_CHECK();                                \
    } while (0)

template <typename T, int F, bool HESS, int DC>
static int launch_epi_dc(const Geom& g, const Work& w, const XArgs& a, int ne, cudaStream_t s) {
    auto kern = k_epilogue<T, F, HESS, DC>;
    constexpr size_t smem = epi_smem<T, F, HESS>();
    static size_t granted = 0;
    if (int st = ensure_smem(kern, smem, granted)) return st;
    ProfScope ps(w.prof, HESS ? K_X_INV_HESS : K_X_INV_GRAD, s);
    kern<<<dim3(ne, g.nl), kEpiThreads, smem, s>>>(a, w.work, g.G);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

// a.dens set (FP64 only): the gradient epilogue stores the densities, the Hessian
// epilogue reads them
template <typename T, int F, bool HESS>
static int launch_epi(const Geom& g, const Work& w, const XArgs& a, int ne, cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
        if (a.dens) return launch_epi_dc<T, F, HESS, HESS ? 2 : 1>(g, w, a, ne, s);
    }
    return launch_epi_dc<T, F, HESS, 0>(g, w, a, ne, s);
}

template <typename T>
static SArgs sargs(const Geom& g, const SCfg& c, int axis, const void* in, void* out, double* part) {
    SArgs a;
    a.in = in; a.out = out; a.tw = g.tw[axis];
    for (int i = 0; i < 3; ++i) { a.lam2[i] = g.lam2[i]; a.k2t[i] = g.k2s[i]; }
    a.G = g.G; a.axis = axis; a.logn = g.logn[axis]; a.W = c.W;
    a.nx = g.n[0]; a.ny = g.n[1]; a.nz = g.n[2];
    a.ntx = g.n[0] / c.W;
    a.nouter = (axis == 1) ? g.n[2] : g.n[1];
    a.estride = (axis == 1) ? (long long)g.n[0] : (long long)g.n[0] * g.n[1];
    a.invG = g.invG;
    a.partials = part; a.nblk = c.nblk; a.nblk_inst = c.nblk_inst;
    a.C = g.C;
    a.skip = g.skip;
    a.imap = g.imap;
    a.fe = FinEnergy{};
    return a;
}

template <typename T>
static XArgs xargs(const Geom& g, const XCfg& c, const void* in, void* out, double* part) {
    XArgs a;
    a.in = in; a.out = out; a.X = nullptr; a.Zd = nullptr; a.V = g.V; a.tw = g.tw[0];
    a.lam2x = g.lam2[0]; a.k2x = g.k2s[0]; a.G = g.G; a.logn = g.logn[0]; a.rpb = c.rpb; a.invG = g.invG;
    a.sigma = 0.0; a.scal = nullptr; a.riem = 0; a.sigslot = -1; a.zproj = 0;
    a.partials = part; a.nblk = c.nblk;
    a.pp = point_params(g);
    a.rpi = g.G / g.n[0];
    a.ppb = reinterpret_cast<const PointParams*>(g.ppb);
    a.skip = g.skip;
    a.imap = g.imap;
    a.fp = FinProj{};
    a.fe = 0;
    a.dens = nullptr;
    return a;
}

// Lemma 4.1 finalize run by the producer's last block per instance
static FinProj fin_proj(const Geom& g, const Work& w, int qe, int qn, int qt, int slot_a, int slot_b,
                        int write_grad_info) {
    FinProj f;
    f.on = 1;
    f.qe = qe; f.qn = qn; f.qt = qt;
    f.slot_a = slot_a; f.slot_b = slot_b; f.write_grad_info = write_grad_info;
    f.M0 = g.M; f.Mb = g.Mb; f.scal0 = w.scal;
    return f;
}

// Forward transforms of every axis but x after the x pass, then the fused
// k-space pass on the last axis, then the inverse passes back to (but not
// including) x.  in = out = w.work on entry (x pass already done).
template <typename T>
static int middle_passes(const Geom& g, const Work& w, cudaStream_t s) {
    const int d = g.dim;
    if (d == 2) {
        const SCfg c = scfg<T>(g, 1, w.num_sms);
        return launch_pass<T, S_K2>(g, c, sargs<T>(g, c, 1, w.work, w.work, nullptr), w, s);
    }
    // d == 3
    const SCfg cy = scfg<T>(g, 1, w.num_sms), cz = scfg<T>(g, 2, w.num_sms);
    int st = launch_pass<T, S_FWD>(g, cy, sargs<T>(g, cy, 1, w.work, w.work, nullptr), w, s);
    if (st) return st;
    st = launch_pass<T, S_K2>(g, cz, sargs<T>(g, cz, 2, w.work, w.work, nullptr), w, s);
    if (st) return st;
    return launch_pass<T, S_INV>(g, cy, sargs<T>(g, cy, 1, w.work, w.work, nullptr), w, s);
}

template <typename T, int F>
static int grad_F(const Geom& g, const Work& w, const void* X, void* Geuc, void* Griem, bool want_norm,
                  cudaStream_t s) {
    constexpr int C = 2 * F + 1;
    const XCfg c = xcfg<T>(g);
    if ((size_t)c.nblk * (1 + 2 * C) > w.part_cap) return SBEC_ERR_ARG;
    void* gout = Geuc ? Geuc : ((Griem || want_norm) ? w.work2 : nullptr);
    int st;
    // the Lemma 4.1 coefficients alpha_g, beta_g and E, mass, magnetisation: finalized
    // by the last block per instance of the pass that stores the partials
    const FinProj fg = fin_proj(g, w, 0, 1, 1 + C, SBEC_S_ALPHA_G, SBEC_S_BETA_G, 1);
    if (g.dim == 1) {
        XArgs a = xargs<T>(g, c, X, gout, w.partA);
        a.X = X;
        a.fp = fg;
        st = launch_x<T, F, X_FULL_GRAD>(c, a, w, s);
        if (st) return st;
    } else {
        st = launch_x<T, F, X_FWD>(c, xargs<T>(g, c, X, w.work, nullptr), w, s);
        if (st) return st;
        st = middle_passes<T>(g, w, s);
        if (st) return st;
        // In 2D and 3D the inverse x pass only transforms and a separate kernel applies
        // the nonlinear epilogue: fused, the epilogue's registers cap the pass at one
        // block per SM; measured, the split form is as fast on 256^2 and faster on 128^3
        // in FP64, and 4x faster on 256^3 in FP32.  1D problems keep the fused kernel.
        st = launch_x<T, F, X_INV>(c, xargs<T>(g, c, w.work, w.work, nullptr), w, s);
        if (st) return st;
        const int ne = elem_blocks(g.G, w.num_sms, g.B, g.tune.elem_per_sm);
        XArgs a = xargs<T>(g, c, nullptr, gout, w.partA);
        a.X = X;
        a.fp = fg;
        a.dens = w.dens;
        st = launch_epi<T, F, false>(g, w, a, ne, s);
        if (st) return st;
    }
    if (Griem || want_norm) {
        const int nb = SBEC_ELEM_GRID(g.G, (k_proj_apply<T, F, true>));
        SBEC_LAUNCH(K_PROJ, (k_proj_apply<T, F, true>), dim3(nb, g.nl), 256, X, gout, Griem, g.G, w.scal,
                    SBEC_S_ALPHA_G, SBEC_S_BETA_G, w.partB, g.imap, SBEC_S_RGRAD_NORM2);
    }
    return SBEC_OK;
}

template <typename T, int F>
static int energy_F(const Geom& g, const Work& w, const void* X, cudaStream_t s) {
    const XCfg c = xcfg<T>(g);
    int st;
    // E (Eq. 3.7) finalized by the last block per instance of the last pass
    if (g.dim == 1) {
        XArgs a = xargs<T>(g, c, X, nullptr, w.partA);
        a.fe = 1;
        a.fp.scal0 = w.scal;
        return launch_x<T, F, X_FULL_ENERGY>(c, a, w, s);
    }
    st = launch_x<T, F, X_FWD_EPW>(c, xargs<T>(g, c, X, w.work, w.partA), w, s);
    if (st) return st;
    const int axis = g.dim == 2 ? 1 : 2;
    if (g.dim == 3) {
        const SCfg cy = scfg<T>(g, 1, w.num_sms);
        st = launch_pass<T, S_FWD>(g, cy, sargs<T>(g, cy, 1, w.work, w.work, nullptr), w, s);
        if (st) return st;
    }
    const SCfg cl = scfg<T>(g, axis, w.num_sms);
    SArgs a = sargs<T>(g, cl, axis, w.work, nullptr, w.partB);
    a.fe.on = 1;
    a.fe.pa = w.partA; a.fe.na_tot = c.nblk; a.fe.na_inst = c.nblk_inst;
    a.fe.scal0 = w.scal;
    return launch_pass<T, S_PARSEVAL>(g, cl, a, w, s);
}

template <typename T, int F>
static int hess_F(const Geom& g, const Work& w, const void* X, const void* Z, double sigma, int riem, void* HZ,
                  cudaStream_t s, int sigslot, bool dens) {
    constexpr int C = 2 * F + 1;
    const int nb = SBEC_ELEM_GRID(g.G, (k_proj_apply<T, F, false>));
    const void* zin = Z;
    // P_u coefficients (Lemma 4.1) into S_PA, S_PB by the last block per instance
    const FinProj fpz = fin_proj(g, w, -1, 0, C, S_PA, S_PB, 0);
    const XCfg c = xcfg<T>(g);
    // 2D/3D with the two-level x pass: xi = P_u Z is formed where Z is read (the x pass
    // and the epilogue), so it is never stored; otherwise it is stored first
    const bool fuse = riem && g.dim > 1 && c.two;
    if (riem) {
        // the Lemma 4.1 coefficients of Z
        const int nd = SBEC_ELEM_GRID(g.G, (k_dot_reduce<T, F>));
        SBEC_LAUNCH(K_DOT, (k_dot_reduce<T, F>), dim3(nd, g.nl), 256, X, Z, g.G, w.partB, w.scal, g.imap, fpz);
        if (!fuse) {
            SBEC_LAUNCH(K_PROJ, (k_proj_apply<T, F, false>), dim3(nb, g.nl), 256, X, Z, w.work2, g.G, w.scal, S_PA,
                        S_PB, nullptr, g.imap, -1);
            zin = w.work2;
        }
    }
    // the Lemma 4.2 coefficients alpha_g, beta_g are read by the epilogue from the
    // scalar block written by the latest gradient at X
    int st;
    if (g.dim == 1) {
        XArgs a = xargs<T>(g, c, zin, HZ, w.partA);
        a.X = X; a.Zd = zin; a.sigma = sigma; a.riem = riem; a.scal = w.scal; a.sigslot = sigslot;
        if (riem) a.fp = fpz;
        st = launch_x<T, F, X_FULL_HESS>(c, a, w, s);
        if (st) return st;
    } else {
        XArgs ax = xargs<T>(g, c, zin, w.work, nullptr);
        if (fuse) { ax.X = X; ax.scal = w.scal; ax.zproj = 1; }
        st = launch_x<T, F, X_FWD>(c, ax, w, s);
        if (st) return st;
        st = middle_passes<T>(g, w, s);
        if (st) return st;
        XArgs a = xargs<T>(g, c, w.work, HZ, w.partA);
        a.X = X; a.Zd = zin; a.sigma = sigma; a.riem = riem; a.scal = w.scal; a.sigslot = sigslot;
        a.zproj = fuse ? 1 : 0;
        if (dens) a.dens = w.dens;
        if (riem) a.fp = fpz;
        // inverse x-FFT in place, then the Hessian epilogue (split as in grad_F)
        st = launch_x<T, F, X_INV>(c, xargs<T>(g, c, w.work, w.work, nullptr), w, s);
        if (st) return st;
        const int ne = elem_blocks(g.G, w.num_sms, g.B, g.tune.elem_per_sm);
        st = launch_epi<T, F, true>(g, w, a, ne, s);
        if (st) return st;
        if (riem && !EpiFusedFin<T, F, true>::v)
            SBEC_LAUNCH(K_FIN, k_fin_proj, g.nl, 256, w.partA, ne * g.nl, ne, F, fpz, g.imap);
    }
    if (riem)
        SBEC_LAUNCH(K_PROJ, (k_proj_apply<T, F, false>), dim3(nb, g.nl), 256, X, HZ, HZ, g.G, w.scal, S_PA, S_PB,
                    nullptr, g.imap, -1);
    return SBEC_OK;
}

template <typename T, int F>
static int retract_F(const Geom& g, const Work& w, const void* U, const void* Xi, double t, int kind, void* out,
                     cudaStream_t s, int tslot = -1) {
    const int nb = SBEC_ELEM_GRID(g.G, (k_retract_w<T, F>));
    const int ns = SBEC_ELEM_GRID(g.G, (k_scale<T, F>));
    SBEC_LAUNCH(K_RETW, (k_retract_w<T, F>), dim3(nb, g.nl), 256, U, Xi, t, out, g.G, w.partB, w.scal, tslot, g.imap,
                kind, g.M, g.Mb);
    SBEC_LAUNCH(K_SCALE, (k_scale<T, F>), dim3(ns, g.nl), 256, out, g.G, w.scal, g.imap);
    return SBEC_OK;
}

#define SBEC_DISPATCH_F(expr_tmpl)                 \
    switch (g.F) {                                 \
        case 1: return expr_tmpl(1);               \
        case 2: return expr_tmpl(2);               \
        case 3: return expr_tmpl(3);               \
        case 4: return expr_tmpl(4);               \
        default: return SBEC_ERR_ARG;              \
    }

template <typename T>
int Ops<T>::energy(const Geom& g, const Work& w, const void* X, cudaStream_t s) {
#define E_(F) energy_F<T, F>(g, w, X, s)
    SBEC_DISPATCH_F(E_)
#undef E_
}

template <typename T>
int Ops<T>::grad(const Geom& g, const Work& w, const void* X, void* Geuc, void* Griem, bool want_norm,
                 cudaStream_t s) {
#define G_(F) grad_F<T, F>(g, w, X, Geuc, Griem, want_norm, s)
    SBEC_DISPATCH_F(G_)
#undef G_
}

template <typename T>
int Ops<T>::hessvec(const Geom& g, const Work& w, const void* X, const void* Z, double sigma, int riem, void* HZ,
                    cudaStream_t s, int sigslot, bool dens) {
#define H_(F) hess_F<T, F>(g, w, X, Z, sigma, riem, HZ, s, sigslot, dens)
    SBEC_DISPATCH_F(H_)
#undef H_
}

template <typename T>
int Ops<T>::retract(const Geom& g, const Work& w, const void* U, const void* Xi, double t, int kind, void* out,
                    cudaStream_t s, int tslot) {
#define R_(F) retract_F<T, F>(g, w, U, Xi, t, kind, out, s, tslot)
    SBEC_DISPATCH_F(R_)
#undef R_
}

template <typename T>
int Ops<T>::lincomb(const Geom& g, const Work& w, const Lin& L, int dot_slot, cudaStream_t s) {
    const long long N = 2LL * g.C * g.G;
    const int nb = SBEC_ELEM_GRID(N / 2, k_lincomb<T>);
    const bool dots = (L.D1 || L.D2);
    SBEC_LAUNCH(K_LIN, k_lincomb<T>, dim3(nb, g.nl), 256, L, N, w.scal, dots ? w.partB : nullptr, g.imap);
    if (dots) SBEC_LAUNCH(K_FIN, k_fin_sums, g.nl, 256, w.partB, nb * g.nl, nb, 2, w.scal, dot_slot, g.imap);
    return SBEC_OK;
}

template <typename T>
int Ops<T>::dot2(const Geom& g, const Work& w, const void* A, const void* B, const void* C, const void* D, int slot,
                 cudaStream_t s) {
    const long long N = 2LL * g.C * g.G;
    const int nb = SBEC_ELEM_GRID(N / 2, k_dot2<T>);
    SBEC_LAUNCH(K_DOT, k_dot2<T>, dim3(nb, g.nl), 256, A, B, C, D, N, w.partB, w.scal, g.imap);
    SBEC_LAUNCH(K_FIN, k_fin_sums, g.nl, 256, w.partB, nb * g.nl, nb, C ? 2 : 1, w.scal, slot, g.imap);
    return SBEC_OK;
}

template <typename T>
int Ops<T>::bbdots(const Geom& g, const Work& w, const void* U, const void* UP, const void* Gv, const void* GP,
                   int slot, cudaStream_t s) {
    const long long N = 2LL * g.C * g.G;
    const int nb = SBEC_ELEM_GRID(N / 2, k_bbdots<T>);
    SBEC_LAUNCH(K_DOT, k_bbdots<T>, dim3(nb, g.nl), 256, U, UP, Gv, GP, N, w.partB, w.scal, g.imap);
    SBEC_LAUNCH(K_FIN, k_fin_sums, g.nl, 256, w.partB, nb * g.nl, nb, 2, w.scal, slot, g.imap);
    return SBEC_OK;
}

template <typename T>
int Ops<T>::ratio(const Geom& g, const Work& w, int dst, int num, int den, int guard_kap, int guard_pp, double eps,
                  cudaStream_t s, int mask) {
    SBEC_LAUNCH(K_FIN, k_ratio, g.nl, 32, w.scal, dst, num, den, guard_kap, guard_pp, eps, mask, g.imap);
    return SBEC_OK;
}

template <typename T>
int Ops<T>::cg_curv(const Geom& g, const Work& w, const void* p, const void* Hp, const CgSlots& cs, cudaStream_t s) {
    const long long N = 2LL * g.C * g.G;
    const int nb = SBEC_ELEM_GRID(N / 2, k_cg_curv<T>);
    SBEC_LAUNCH(K_DOT, k_cg_curv<T>, dim3(nb, g.nl), 256, p, Hp, N, w.partB, w.scal, g.imap, cs);
    return SBEC_OK;
}

template <typename T>
int Ops<T>::cg_update(const Geom& g, const Work& w, void* x, void* r, const void* p, const void* Hp,
                      const CgSlots& cs, cudaStream_t s) {
    const long long N = 2LL * g.C * g.G;
    const int nb = SBEC_ELEM_GRID(N / 2, k_cg_update<T>);
    SBEC_LAUNCH(K_LIN, k_cg_update<T>, dim3(nb, g.nl), 256, x, r, p, Hp, N, w.partB, w.scal, g.imap, cs);
    return SBEC_OK;
}

template <typename T, int F>
static int prolongate_F(const Geom& gc, const Work& wc, const void* Xc, const Geom& gf, const Work& wf, void* Xf,
                        cudaStream_t s) {
    if (gc.B != 1 || gf.B != 1) return SBEC_ERR_ARG;
    // coarse forward transform into the coarse scratch
    {
        const Work& w = wc;
        const XCfg c = xcfg<T>(gc);
        int st = launch_x<T, F, X_FWD>(c, xargs<T>(gc, c, Xc, wc.work, nullptr), w, s);
        if (st) return st;
        for (int ax = 1; ax < gc.dim; ++ax) {
            const SCfg sc = scfg<T>(gc, ax, wc.num_sms);
            st = launch_s<T, S_FWD>(sc, sargs<T>(gc, sc, ax, wc.work, wc.work, nullptr), w, s);
            if (st) return st;
        }
    }
    const Work& w = wf;
    // zero-pad into the fine scratch; 1/G_c undoes the coarse forward DFT's scale on
    // inversion and sqrt(dV_f / dV_c) keeps X = sqrt(dV) phi
    const double scale = sqrt(gf.dV / gc.dV) / (double)gc.G;
    SBEC_LAUNCH(K_PROLONG, k_pad<T>, elem_blocks((long long)gf.C * gf.G, wf.num_sms), 256, wc.work, wf.work, gc.C,
                gc.n[0], gc.n[1], gc.n[2], gf.n[0], gf.n[1], gf.n[2], scale);
    for (int ax = gf.dim - 1; ax >= 1; --ax) {
        const SCfg sc = scfg<T>(gf, ax, wf.num_sms);
        int st = launch_s<T, S_INV>(sc, sargs<T>(gf, sc, ax, wf.work, wf.work, nullptr), w, s);
        if (st) return st;
    }
    const XCfg c = xcfg<T>(gf);
    int st = launch_x<T, F, X_INV>(c, xargs<T>(gf, c, wf.work, Xf, nullptr), w, s);
    if (st) return st;
    // back onto M with the projective retraction (Lemma 5.1)
    return retract_F<T, F>(gf, wf, Xf, Xf, 0.0, 1, Xf, s);
}

template <typename T>
int Ops<T>::prolongate(const Geom& gc, const Work& wc, const void* Xc, const Geom& gf, const Work& wf, void* Xf,
                       cudaStream_t s) {
    const Geom& g = gf;
#define P_(F) prolongate_F<T, F>(gc, wc, Xc, gf, wf, Xf, s)
    SBEC_DISPATCH_F(P_)
#undef P_
}

template <typename T>
int Ops<T>::init_tables(Geom& g, void* tw_storage, cudaStream_t s) {
    using T2 = typename C2<T>::t;
    T2* base = reinterpret_cast<T2*>(tw_storage);
    size_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        const int n = g.n[ax];
        g.tw[ax] = base + off;
        k_twiddles<T><<<(n + 255) / 256, 256, 0, s>>>(base + off, n);
        SBEC_LAUNCH_CHECK();
        off += n;
    }
    return SBEC_OK;
}

template <typename T>
int Ops<T>::harmonic_potential(const Geom& g, void* V, const double* lo, const double* hi, cudaStream_t s) {
    const double hx = (hi[0] - lo[0]) / g.n[0], hy = (hi[1] - lo[1]) / g.n[1], hz = (hi[2] - lo[2]) / g.n[2];
    k_harmonic<T><<<1024, 256, 0, s>>>(V, g.n[0], g.n[1], g.n[2], lo[0], hx, lo[1], hy, lo[2], hz, g.dim);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T>
int Ops<T>::convert_potential(const Geom& g, void* V, const double* Vd, cudaStream_t s) {
    k_convert<T><<<1024, 256, 0, s>>>(V, Vd, g.G);
    SBEC_LAUNCH_CHECK();
    return SBEC_OK;
}

template <typename T>
size_t Ops<T>::partials_needed(const Geom& g, int num_sms, bool any_shape) {
    // any_shape: the most blocks an accepted shape launches (one grid row per
    // x-pass block, one pencil per strided tile, kMaxElemPerSm blocks per SM)
    Geom h = g;
    if (any_shape) {
        h.tune = Tune{};
        h.tune.x_rows = 1;
        h.tune.elem_per_sm = kMaxElemPerSm;
        for (int ax = 1; ax < g.dim; ++ax) h.tune.s_pencils[ax] = 1;
    }
    const XCfg c = xcfg<T>(h);
    size_t need = (size_t)c.nblk * (1 + 2 * g.C);
    const size_t e = (size_t)elem_blocks(g.G, num_sms, g.B, h.tune.elem_per_sm) * g.B * (1 + 2 * g.C);
    if (e > need) need = e;
    for (int ax = 1; ax < g.dim; ++ax) {
        const SCfg sc = scfg<T>(h, ax, num_sms);
        if ((size_t)sc.nblk > need) need = sc.nblk;
    }
    return need;
}

template <typename T>
bool Ops<T>::tune_ok(const Geom& g, const Tune& t) {
    auto pow2 = [](int v) { return v >= 1 && (v & (v - 1)) == 0; };
    if (t.x_rows != 0) {
        const long long rows_inst = g.G / g.n[0];
        if (!pow2(t.x_rows) || rows_inst % t.x_rows != 0) return false;
        Geom h = g;
        h.tune = t;
        const XCfg c = xcfg<T>(h);
        if (c.two) {
            if (c.nth > 512 || c.smem > kMaxSmem) return false;
        } else {
            const long long pts = (long long)t.x_rows * g.C * g.n[0];
            if (pts > kMaxPointsPerBlock || xsmem<T>(t.x_rows * g.C, g.n[0]) > kMaxSmem) return false;
        }
    }
    if (t.s_pencils[0] != 0 || t.s_split[0] != 0) return false;
    for (int ax = 1; ax < 3; ++ax) {
        const int W = t.s_pencils[ax], sp = t.s_split[ax];
        if (ax >= g.dim && (W != 0 || sp != 0)) return false;
        if (sp == kTmaSplit) {
            // the TMA pass: a width it has, on a pass it runs
            if (W != 0 && W != 8 && W != 16 && W != 32) return false;
            Geom h = g;
            h.tune = t;
            if (!tma_pass<T>(h, ax)) return false;
            continue;
        }
        if (sp != 0 && sp != 1 && sp != 2 && sp != 4 && sp != 8) return false;
        if (W == 0) continue;
        if (!pow2(W) || W > g.n[0]) return false;
        Geom h = g;
        h.tune = t;
        const SCfg c = scfg<T>(h, ax, 1);
        if (c.two) {
            if (c.nth > 512 || c.smem > kMaxSmem) return false;
            continue;
        }
        const long long pts = (long long)W * g.n[ax];
        if (pts > kMaxPointsPerBlock || (size_t)pts * sizeof(typename C2<T>::t) > kMaxSmem) return false;
    }
    if (t.elem_per_sm < 0 || t.elem_per_sm > kMaxElemPerSm) return false;
    return true;
}

template <typename T>
Tune Ops<T>::resolved(const Geom& g, int num_sms) {
    Tune t{};
    t.x_rows = xcfg<T>(g).rpb;
    for (int ax = 1; ax < g.dim; ++ax) {
        // the TMA pass (its tile width, and s_split = kTmaSplit) where it runs
        if (const int W = tma_pass<T>(g, ax)) {
            t.s_pencils[ax] = W;
            t.s_split[ax] = kTmaSplit;
            continue;
        }
        t.s_pencils[ax] = scfg<T>(g, ax, num_sms).W;
        t.s_split[ax] = g.tune.s_split[ax] > 0 ? g.tune.s_split[ax] : 1;
    }
    t.elem_per_sm = g.tune.elem_per_sm > 0 ? g.tune.elem_per_sm : 8;
    return t;
}

}  // namespace sbec
