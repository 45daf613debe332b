// Device building blocks of libsbec: complex arithmetic, deterministic block
// reductions, the shared-memory Stockham FFT used by every pass, and the
// per-grid-point spin-F terms of the discrete energy (Sec. 3, Eq. 3.7), its
// gradient (Eq. 3.12) and Hessian-vector product (Eq. 3.13).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbec_internal.h"

namespace sbec {

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename T2> __device__ __forceinline__ T2 mk(decltype(T2::x) a, decltype(T2::x) b) {
    T2 r; r.x = a; r.y = b; return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
    return mk<T2>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { return mk<T2>(a.x, -a.y); }
template <typename T2> __device__ __forceinline__ T2 cscale(T2 a, decltype(T2::x) s) { return mk<T2>(a.x * s, a.y * s); }
template <typename T2> __device__ __forceinline__ decltype(T2::x) cabs2(T2 a) { return a.x * a.x + a.y * a.y; }
// a += s * b
template <typename T2> __device__ __forceinline__ void caxpy(T2& a, decltype(T2::x) s, T2 b) { a.x += s * b.x; a.y += s * b.y; }
// a += b * c (complex)
template <typename T2> __device__ __forceinline__ void cfma(T2& a, T2 b, T2 c) {
    a.x += b.x * c.x - b.y * c.y; a.y += b.x * c.y + b.y * c.x;
}

// FP32 complex additions, subtractions and real scalings as paired-float instructions
// (add/sub/mul/fma.rn.f32x2, sm_100 family): one instruction per complex value where the
// scalar form takes two.  Each lane is rounded as the scalar instruction would round it,
// so the results are the same bits.
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 f2_of(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(r);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(r);
}
template <> __device__ __forceinline__ float2 cscale<float2>(float2 a, float s) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(make_float2(s, s))));
    return f2_of(r);
}
template <> __device__ __forceinline__ void caxpy<float2>(float2& a, float s, float2 b) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(b)), "l"(f2_bits(make_float2(s, s))), "l"(f2_bits(a)));
    a = f2_of(r);
}

// ---------------------------------------------------------------------------
// Per-thread running sums of the reductions.  FP64 form: a double.  Mixed form:
// a float sum whose rounding error is carried in a second float (the error-free
// transformation TwoSum of Moller and Knuth, then cascaded as in Neumaier's
// compensated summation), so that the FP32 kernels keep about twice float
// precision in their partials without FP64 arithmetic per point (on this GPU the
// FP64 pipe runs at 1/64 of the FP32 rate, below what HBM bandwidth needs).
// value() hands the partial to the FP64 block reduction.
// ---------------------------------------------------------------------------
template <typename T> struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        const float bv = t - s;
        c += (s - (t - bv)) + (v - bv);
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

template <int NQ, typename T>
__device__ __forceinline__ void acc_values(const Acc<T> (&a)[NQ], double (&v)[NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = a[q].value();
}

// ---------------------------------------------------------------------------
// Deterministic reductions.  Each block reduces NQ doubles in a fixed order
// (warp shuffles, then warp 0 over the per-warp results) and writes them to
// partials[q * nblk + blk]; reduce_partials sums those in a fixed order too,
// so every result is bitwise reproducible for a given launch configuration.
// ---------------------------------------------------------------------------
template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&v)[NQ], double* __restrict__ partials,
                                                   int nblk, int blk) {
    __shared__ double red[NQ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = lane < nwarp ? red[q][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) partials[(size_t)q * nblk + blk] = s;
        }
    }
    __syncthreads();
}

// Sum of partials[q * nblk + 0 .. nblk-1] by one block, fixed order; result
// returned to every thread of the block.
__device__ __forceinline__ double block_sum_partials(const double* __restrict__ partials, int q, int nblk) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partials[(size_t)q * nblk + i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (warp == 0) {
        s = lane < nwarp ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Stockham autosort FFT of P pencils of length n = 2^logn held in shared
// memory: element e of pencil p lives at buf[p * ps + e * es].  Radix-4 stages
// (sub-transform length Ns = 1, 4, 16, ...) with a radix-2 stage last when
// logn is odd.  Stage with radix R at length Ns: butterfly j reads elements
// j + r n/R, multiplies element r by W_{R Ns}^{(j mod Ns) r}, applies the
// R-point DFT and writes output r to (j - j mod Ns) R + (j mod Ns) + r Ns.
// The radix-4 stages are in place: every thread holds its ITEMS butterflies in
// registers across a barrier, so ITEMS * nth >= P n / 4 is required.  The
// radix-2 stage touches only its own two slots and needs no staging.
// tw[m] = exp(-2 pi i m / n), m = 0..n-1; INV uses the conjugate twiddles and
// the conjugate DFT (unnormalised both ways).
// ---------------------------------------------------------------------------
// PFAST: consecutive threads take consecutive pencils (for tiles stored element-major,
// buf[e * P + p], so that a warp's accesses are unit-stride); otherwise consecutive
// threads take consecutive butterflies of one pencil (rows stored pencil-major).
// PAD: logical slot i lives at i + i/8 (smem_slot), which spreads the stride-4
// Stockham writes of pencil-major rows over all banks.
__device__ __forceinline__ int smem_slot(int i) { return i + (i >> 3); }

template <typename T2, bool INV, int ITEMS, bool PFAST = false, bool PAD = false>
__device__ __forceinline__ void fft_pencils(T2* buf, int logn, int P, int ps, int es,
                                            const T2* __restrict__ tw, int tid, int nth) {
#define SLOT(i) (PAD ? smem_slot(i) : (i))
    const int n = 1 << logn;
    int Ns = 1;
    if (logn >= 2) {
        const int nb = n >> 2;
        const int lognb = logn - 2;
        const int total = P * nb;
        for (int s = 0; s + 2 <= logn; s += 2) {
            const int twstep = n / (Ns << 2);
            T2 v[ITEMS][4];
            int dst[ITEMS];
#pragma unroll
            for (int it = 0; it < ITEMS; ++it) {
                const int idx = tid + it * nth;
                if (idx < total) {
                    const int p = PFAST ? (idx & (P - 1)) : (idx >> lognb);
                    const int j = PFAST ? (idx / P) : (idx & (nb - 1));
                    const int pb = p * ps;
                    T2 a0 = buf[SLOT(pb + j * es)], a1 = buf[SLOT(pb + (j + nb) * es)],
                       a2 = buf[SLOT(pb + (j + 2 * nb) * es)], a3 = buf[SLOT(pb + (j + 3 * nb) * es)];
                    const int k = j & (Ns - 1);
                    if (k != 0) {
                        T2 w1 = tw[k * twstep], w2 = tw[2 * k * twstep], w3 = tw[3 * k * twstep];
                        if (INV) { w1 = cconj(w1); w2 = cconj(w2); w3 = cconj(w3); }
                        a1 = cmul(a1, w1); a2 = cmul(a2, w2); a3 = cmul(a3, w3);
                    }
                    const T2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
                    const T2 d = csub(a1, a3);
                    // forward: (a1 - a3) * (-i); inverse: (a1 - a3) * (+i)
                    const T2 t3 = INV ? mk<T2>(-d.y, d.x) : mk<T2>(d.y, -d.x);
                    v[it][0] = cadd(t0, t2);
                    v[it][1] = cadd(t1, t3);
                    v[it][2] = csub(t0, t2);
                    v[it][3] = csub(t1, t3);
                    dst[it] = p * ps + (((j - k) << 2) + k) * es;
                }
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < ITEMS; ++it) {
                const int idx = tid + it * nth;
                if (idx < total) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) buf[SLOT(dst[it] + r * Ns * es)] = v[it][r];
                }
            }
            __syncthreads();
            Ns <<= 2;
        }
    }
    if (logn & 1) {
        // last stage, Ns = n/2: out[j] = a0 + w a1, out[j + n/2] = a0 - w a1, w = W_n^j
        const int half = n >> 1;
        const int total = P * half;
        for (int idx = tid; idx < total; idx += nth) {
            const int p = PFAST ? (idx & (P - 1)) : (idx >> (logn - 1));
            const int j = PFAST ? (idx / P) : (idx & (half - 1));
            const int i0 = SLOT(p * ps + j * es), i1 = SLOT(p * ps + (j + half) * es);
            const T2 a0 = buf[i0];
            T2 a1 = buf[i1];
            if (j != 0) {
                T2 w = tw[j];
                if (INV) w = cconj(w);
                a1 = cmul(a1, w);
            }
            buf[i0] = cadd(a0, a1);
            buf[i1] = csub(a0, a1);
        }
        __syncthreads();
    }
#undef SLOT
}

// ---------------------------------------------------------------------------
// Register DFTs of length L = 1, 2, 4, 8, 16 (natural order in and out,
// unnormalised; INV: the conjugate transform), built from 4-point butterflies.
// W16[e] = exp(-2 pi i e / 16) is exact to double rounding: cos and sin of
// multiples of pi/8 are 1, sqrt(1/2), cos(pi/8) = sqrt(2 + sqrt 2)/2 and
// sin(pi/8) = sqrt(2 - sqrt 2)/2.
// ---------------------------------------------------------------------------
constexpr double kC8 = 0.92387953251128675613;   // cos(pi/8)
constexpr double kS8 = 0.38268343236508977173;   // sin(pi/8)
constexpr double kR2 = 0.70710678118654752440;   // sqrt(1/2)

// a * W16^E (forward) or a * conj(W16^E) (inverse)
template <typename T2, bool INV, int E>
__device__ __forceinline__ T2 mul_w16(T2 a) {
    using T = decltype(T2::x);
    constexpr int e = E & 15;
    if constexpr (e == 0) {
        return a;
    } else if constexpr (e == 4) {
        return INV ? mk<T2>(-a.y, a.x) : mk<T2>(a.y, -a.x);        // -i (forward)
    } else if constexpr (e == 8) {
        return mk<T2>(-a.x, -a.y);
    } else if constexpr (e == 12) {
        return INV ? mk<T2>(a.y, -a.x) : mk<T2>(-a.y, a.x);        // +i (forward)
    } else {
        constexpr double cs[16] = {1, kC8, kR2, kS8, 0, -kS8, -kR2, -kC8, -1, -kC8, -kR2, -kS8, 0, kS8, kR2, kC8};
        constexpr double sn[16] = {0, kS8, kR2, kC8, 1, kC8, kR2, kS8, 0, -kS8, -kR2, -kC8, -1, -kC8, -kR2, -kS8};
        const T c = T(cs[e]), sg = T(INV ? -sn[e] : sn[e]);
        // (a.x + i a.y)(c - i sg)
        return mk<T2>(a.x * c + a.y * sg, a.y * c - a.x * sg);
    }
}

template <typename T2, bool INV>
__device__ __forceinline__ void dft4(T2& a0, T2& a1, T2& a2, T2& a3) {
    const T2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
    const T2 t3 = mul_w16<T2, INV, 4>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <typename T2, int L, bool INV> struct RegDft;
template <typename T2, bool INV> struct RegDft<T2, 1, INV> {
    __device__ static __forceinline__ void run(T2*) {}
};
template <typename T2, bool INV> struct RegDft<T2, 2, INV> {
    __device__ static __forceinline__ void run(T2* v) {
        const T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <typename T2, bool INV> struct RegDft<T2, 4, INV> {
    __device__ static __forceinline__ void run(T2* v) { dft4<T2, INV>(v[0], v[1], v[2], v[3]); }
};
// 8 = 2 x 4: X[k] = E[k] + W8^k O[k], X[k + 4] = E[k] - W8^k O[k]
template <typename T2, bool INV> struct RegDft<T2, 8, INV> {
    __device__ static __forceinline__ void run(T2* v) {
        T2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<T2, INV>(e0, e1, e2, e3);
        dft4<T2, INV>(o0, o1, o2, o3);
        o1 = mul_w16<T2, INV, 2>(o1);
        o2 = mul_w16<T2, INV, 4>(o2);
        o3 = mul_w16<T2, INV, 6>(o3);
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};
// 16 = 4 x 4: j = j1 + 4 j2, k = k2 + 4 k1; DFT4 over j2, times W16^{j1 k2},
// DFT4 over j1
template <typename T2, bool INV> struct RegDft<T2, 16, INV> {
    __device__ static __forceinline__ void run(T2* v) {
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) dft4<T2, INV>(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12]);
        // v[j1 + 4 k2] *= W16^{j1 k2}
        v[5] = mul_w16<T2, INV, 1>(v[5]);
        v[9] = mul_w16<T2, INV, 2>(v[9]);
        v[13] = mul_w16<T2, INV, 3>(v[13]);
        v[6] = mul_w16<T2, INV, 2>(v[6]);
        v[10] = mul_w16<T2, INV, 4>(v[10]);
        v[14] = mul_w16<T2, INV, 6>(v[14]);
        v[7] = mul_w16<T2, INV, 3>(v[7]);
        v[11] = mul_w16<T2, INV, 6>(v[11]);
        v[15] = mul_w16<T2, INV, 9>(v[15]);
        T2 r[16];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            T2 a0 = v[4 * k2], a1 = v[4 * k2 + 1], a2 = v[4 * k2 + 2], a3 = v[4 * k2 + 3];
            dft4<T2, INV>(a0, a1, a2, a3);
            r[k2] = a0; r[k2 + 4] = a1; r[k2 + 8] = a2; r[k2 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = r[i];
    }
};

// FP64 16-point DFT with the stage-2 twiddles folded into the butterflies.  A
// twiddle w = wr + i wi is written w = m (1 + i r) (r = wi / wr, |wr| >= |wi|) or
// w = m (r + i) (r = wr / wi, otherwise), so that b w = m b' with b' = b (1 + i r)
// or b (r + i) two FMAs; the real factor m then enters the butterfly's additions
// as FMAs (a0 +- m2 b2', and m1 b1' +- m3 b3' from one product).  With |r| <= 1
// every FMA has a bounded coefficient (the tangent / cotangent form of Linzer and
// Feig's FMA butterflies).  Per row of four outputs this takes 24 FP64
// instructions instead of 28 (three complex products and eight additions); the
// FP64 passes are bound by the FP64 pipe, where instructions are the cost.
template <bool INV, int E> struct W16Fold {
    static constexpr double cs[16] = {1, kC8, kR2, kS8, 0, -kS8, -kR2, -kC8, -1, -kC8, -kR2, -kS8, 0, kS8, kR2, kC8};
    static constexpr double sn[16] = {0, kS8, kR2, kC8, 1, kC8, kR2, kS8, 0, -kS8, -kR2, -kC8, -1, -kC8, -kR2, -kS8};
    static constexpr double wr = cs[E & 15];
    static constexpr double wi = INV ? sn[E & 15] : -sn[E & 15];
    static constexpr bool tangent = (wr < 0 ? -wr : wr) >= (wi < 0 ? -wi : wi);
    static constexpr double m = tangent ? wr : wi;
    static constexpr double r = tangent ? wi / wr : wr / wi;
};
// b' with b w = m b'
template <bool INV, int E>
__device__ __forceinline__ double2 fold_w16(double2 b) {
    using W = W16Fold<INV, E>;
    if constexpr (W::tangent)
        return make_double2(fma(-W::r, b.y, b.x), fma(W::r, b.x, b.y));      // b (1 + i r)
    else
        return make_double2(fma(W::r, b.x, -b.y), fma(W::r, b.y, b.x));      // b (r + i)
}
// one stage-2 row: DFT4 of (a0, b1 w^E1, b2 w^E2, b3 w^E3) in place, E2 = 2 E1, E3 = 3 E1
template <bool INV, int E1>
__device__ __forceinline__ void dft4_folded(double2& a0, double2& b1, double2& b2, double2& b3) {
    constexpr int E2 = 2 * E1, E3 = 3 * E1;
    using W1 = W16Fold<INV, E1>;
    using W2 = W16Fold<INV, E2>;
    using W3 = W16Fold<INV, E3>;
    double2 t0, t1;
    if constexpr ((E2 & 15) == 4 || (E2 & 15) == 12) {
        const double2 a2 = mul_w16<double2, INV, E2>(b2);                   // +-i: no arithmetic
        t0 = cadd(a0, a2);
        t1 = csub(a0, a2);
    } else {
        const double2 c2 = fold_w16<INV, E2>(b2);
        t0 = make_double2(fma(W2::m, c2.x, a0.x), fma(W2::m, c2.y, a0.y));
        t1 = make_double2(fma(-W2::m, c2.x, a0.x), fma(-W2::m, c2.y, a0.y));
    }
    const double2 c1 = fold_w16<INV, E1>(b1), c3 = fold_w16<INV, E3>(b3);
    const double2 p = make_double2(W1::m * c1.x, W1::m * c1.y);
    const double2 t2 = make_double2(fma(W3::m, c3.x, p.x), fma(W3::m, c3.y, p.y));
    const double2 t3 = mul_w16<double2, INV, 4>(make_double2(fma(-W3::m, c3.x, p.x), fma(-W3::m, c3.y, p.y)));
    a0 = cadd(t0, t2);
    b2 = csub(t0, t2);
    b1 = cadd(t1, t3);
    b3 = csub(t1, t3);
}
// FP64 8-point DFT, radix 2 x 4 with the W8 twiddles folded the same way
template <bool INV, int E>
__device__ __forceinline__ void bfly_folded(double2& e, double2& o) {
    using W = W16Fold<INV, E>;
    const double2 c = fold_w16<INV, E>(o);
    o = make_double2(fma(-W::m, c.x, e.x), fma(-W::m, c.y, e.y));
    e = make_double2(fma(W::m, c.x, e.x), fma(W::m, c.y, e.y));
}
template <bool INV> struct RegDft<double2, 8, INV> {
    __device__ static __forceinline__ void run(double2* v) {
        double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<double2, INV>(e0, e1, e2, e3);
        dft4<double2, INV>(o0, o1, o2, o3);
        o2 = mul_w16<double2, INV, 4>(o2);
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        bfly_folded<INV, 2>(e1, o1);
        bfly_folded<INV, 6>(e3, o3);
        v[1] = e1; v[5] = o1;
        v[3] = e3; v[7] = o3;
    }
};
template <bool INV> struct RegDft<double2, 16, INV> {
    __device__ static __forceinline__ void run(double2* v) {
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) dft4<double2, INV>(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12]);
        // row k2 holds v[4 k2 + j1], j1 = 0..3, whose twiddle is W16^{j1 k2}
        double2 r[16];
        {
            double2 a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
            dft4<double2, INV>(a0, a1, a2, a3);
            r[0] = a0; r[4] = a1; r[8] = a2; r[12] = a3;
        }
        {
            double2 a0 = v[4], a1 = v[5], a2 = v[6], a3 = v[7];
            dft4_folded<INV, 1>(a0, a1, a2, a3);
            r[1] = a0; r[5] = a1; r[9] = a2; r[13] = a3;
        }
        {
            double2 a0 = v[8], a1 = v[9], a2 = v[10], a3 = v[11];
            dft4_folded<INV, 2>(a0, a1, a2, a3);
            r[2] = a0; r[6] = a1; r[10] = a2; r[14] = a3;
        }
        {
            double2 a0 = v[12], a1 = v[13], a2 = v[14], a3 = v[15];
            dft4_folded<INV, 3>(a0, a1, a2, a3);
            r[3] = a0; r[7] = a1; r[11] = a2; r[15] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = r[i];
    }
};

// ---------------------------------------------------------------------------
// Two-level FFT of length N = N1 N2 (N <= 256): with j = j1 + N1 j2 and
// k = k2 + N2 k1,
//   X[k2 + N2 k1] = sum_j1 W_N1^{j1 k1} W_N^{j1 k2} sum_j2 W_N2^{j2 k2} x[j1 + N1 j2].
// Level A: one thread per j1 holds x[j1 + N1 j2] (j2 < N2) in registers, applies
// DFT_N2 and the twiddles W_N^{j1 k2}; one exchange through shared memory; level
// B: one thread per k2 holds the N1 values of its k2 and applies DFT_N1.  The
// inverse runs the levels backwards with conjugate twiddles.  Each level is a
// register computation; the only shared-memory traffic is the exchange.
// ---------------------------------------------------------------------------
template <int LOGN> struct Split2 {
    static constexpr int N = 1 << LOGN;
    static constexpr int N1 = 1 << ((LOGN + 1) / 2);   // level-B length (>= N2)
    static constexpr int N2 = N / N1;                   // level-A length
};

// level A forward: v[0..N2) = x[j1 + N1 j2] -> v[k2] = W_N^{j1 k2} DFT_N2(x)[k2]
template <typename T2, int LOGN, bool INV>
__device__ __forceinline__ void level_a_fwd(T2* v, int j1, const T2* __restrict__ tw) {
    constexpr int N2 = Split2<LOGN>::N2;
    RegDft<T2, N2, INV>::run(v);
    if (j1 != 0) {
#pragma unroll
        for (int k2 = 1; k2 < N2; ++k2) {
            T2 w = tw[j1 * k2];
            if (INV) w = cconj(w);
            v[k2] = cmul(v[k2], w);
        }
    }
}

// level B' (inverse start): v[0..N1) = X[k2 + N2 k1] -> v[j1] = W_N^{-j1 k2} IDFT_N1(X)[j1]
template <typename T2, int LOGN>
__device__ __forceinline__ void level_b_inv(T2* v, int k2, const T2* __restrict__ tw) {
    constexpr int N1 = Split2<LOGN>::N1;
    RegDft<T2, N1, true>::run(v);
    if (k2 != 0) {
#pragma unroll
        for (int j1 = 1; j1 < N1; ++j1) v[j1] = cmul(v[j1], cconj(tw[j1 * k2]));
    }
}

// ---------------------------------------------------------------------------
// Spin-F constants in ladder / pair form (an independent restatement of the
// Sec. 2 matrices).  Component index i = 0..2F holds l = F - i.
//   LAD[i]  = sqrt(F(F+1) - (l-1) l) couples i and i+1:  F_+ = sum_i LAD[i] conj(x_i) x_{i+1}
//             (f_+ raises l-1 -> l; Sec. 2 explicit F_+ of the spin-3 case).
//   SGL[i]  = (-1)^i / sqrt(2F+1): A00 = sum_i SGL[i] x_i x_{2F-i} (Sec. 2 singlet).
//   QNT[k][i], k = 0..4 for l = 2, 1, 0, -1, -2 (F = 3): A_{2l} = sum_i QNT[k][i] x_i x_{2F-l-i},
//             the symmetric matrix entry (A_l)_{i, 2F-l-i} (Sec. 2 quintet; explicit
//             pair formulas split evenly over the ordered pairs).
// ---------------------------------------------------------------------------
template <int F> struct Spin;

// 1 / sqrt(2F + 1), the singlet normalisation (a literal: a device sqrt of a
// constant is not folded at compile time and would cost an FP64 square root and
// division per grid point)
template <int C> struct InvSqrtC;
template <> struct InvSqrtC<3> { static constexpr double v = 0.57735026918962576451; };
template <> struct InvSqrtC<5> { static constexpr double v = 0.44721359549995793928; };
template <> struct InvSqrtC<7> { static constexpr double v = 0.37796447300922722721; };
template <> struct InvSqrtC<9> { static constexpr double v = 0.33333333333333333333; };

template <> struct Spin<1> {
    static constexpr int C = 3;
    __device__ static constexpr double lad(int i) { return 1.4142135623730950488; }
};
template <> struct Spin<2> {
    static constexpr int C = 5;
    __device__ static constexpr double lad(int i) {
        return (i == 0 || i == 3) ? 2.0 : 2.4494897427831780982;   // 2, sqrt6, sqrt6, 2
    }
};
template <> struct Spin<3> {
    static constexpr int C = 7;
    __device__ static constexpr double lad(int i) {
        return (i == 0 || i == 5) ? 2.4494897427831780982            // sqrt6
             : (i == 1 || i == 4) ? 3.1622776601683793320            // sqrt10
                                  : 3.4641016151377545871;           // sqrt12
    }
};

// F = 4 (and any higher F): the same ladder constants sqrt(F(F+1) - (l-1) l),
// l = F - i; the paper prints the spin matrices up to F = 3 only, and a spin-4
// condensate is modelled with the density, spin and singlet-pair terms
template <> struct Spin<4> {
    static constexpr int C = 9;
    __device__ static constexpr double lad(int i) {
        return (i == 0 || i == 7) ? 2.8284271247461900976            // sqrt8
             : (i == 1 || i == 6) ? 3.7416573867739413856            // sqrt14
             : (i == 2 || i == 5) ? 4.2426406871192851464            // sqrt18
                                  : 4.4721359549995793928;           // sqrt20
    }
};

__device__ __forceinline__ constexpr double qnt_entry(int k, int i) {
    // 1/sqrt21 and its multiples
    constexpr double r21 = 0.21821789023599238127;       // 1/sqrt(21)
    constexpr double a5 = 2.5 * r21;                     // 5/(2 sqrt21)
    constexpr double a3 = -1.5 * r21;                    // -3/(2 sqrt21)
    constexpr double s2 = 1.4142135623730950488 * r21;   // sqrt2/sqrt21
    constexpr double h2 = 0.5 * s2;                      // sqrt2/(2 sqrt21)
    constexpr double h15 = -0.5 * 3.8729833462074168852 * r21;  // -sqrt15/(2 sqrt21)
    constexpr double h10 = 0.5 * 3.1622776601683793320 * r21;   // sqrt10/(2 sqrt21)
    constexpr double h20 = -0.5 * 4.4721359549995793928 * r21;  // -sqrt20/(2 sqrt21)
    constexpr double s6 = 2.4494897427831780982 * r21;          // sqrt6/sqrt21
    switch (k) {
        case 0:  // l = 2: partner 4 - i
            return i == 0 ? h10 : i == 1 ? h20 : i == 2 ? s6 : i == 3 ? h20 : i == 4 ? h10 : 0.0;
        case 1:  // l = 1: partner 5 - i
            return i == 0 ? a5 : i == 1 ? h15 : i == 2 ? h2 : i == 3 ? h2 : i == 4 ? h15 : i == 5 ? a5 : 0.0;
        case 2:  // l = 0: partner 6 - i
            return i == 0 ? a5 : i == 1 ? 0.0 : i == 2 ? a3 : i == 3 ? s2 : i == 4 ? a3 : i == 5 ? 0.0 : a5;
        case 3:  // l = -1: partner 7 - i
            return i == 1 ? a5 : i == 2 ? h15 : i == 3 ? h2 : i == 4 ? h2 : i == 5 ? h15 : i == 6 ? a5 : 0.0;
        default: // l = -2: partner 8 - i
            return i == 2 ? h10 : i == 3 ? h20 : i == 4 ? s6 : i == 5 ? h20 : i == 6 ? h10 : 0.0;
    }
}
__device__ __forceinline__ constexpr int qnt_l(int k) { return 2 - k; }


// PointParams in the arithmetic type of the pointwise code (converted once per
// thread, so that the FP32 kernels do no FP64 arithmetic per point).
template <typename T> struct PPT {
    T bz[kMaxC], g0, g1, g2, g3, e0, e1, e2, e3;
    __device__ __forceinline__ explicit PPT(const PointParams& p) {
#pragma unroll
        for (int i = 0; i < kMaxC; ++i) bz[i] = T(p.bz[i]);
        g0 = T(p.g0); g1 = T(p.g1); g2 = T(p.g2); g3 = T(p.g3);
        e0 = T(p.e0); e1 = T(p.e1); e2 = T(p.e2); e3 = T(p.e3);
    }
};

// Densities at one grid point (Sec. 3): rho, F_z, F_+, A00, A_{2l}.
template <int F, typename T2>
struct Dens {
    using T = decltype(T2::x);
    T rho, Fz;
    T2 Fp, A00, A2[5];

    __device__ __forceinline__ void compute(const T2 (&x)[2 * F + 1]) {
        constexpr int C = 2 * F + 1;
        rho = 0; Fz = 0;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const T a = cabs2(x[i]);
            rho += a;
            Fz += T(F - i) * a;
        }
        Fp = mk<T2>(0, 0);
#pragma unroll
        for (int i = 0; i < C - 1; ++i) {
            const T2 t = cmulc(x[i], x[i + 1]);
            caxpy(Fp, T(Spin<F>::lad(i)), t);
        }
        A00 = mk<T2>(0, 0);
        if (F >= 2) {
            const T sg = T(InvSqrtC<C>::v);
#pragma unroll
            for (int i = 0; i < F; ++i) caxpy(A00, T((i & 1) ? -2.0 : 2.0) * sg, cmul(x[i], x[C - 1 - i]));
            caxpy(A00, T((F & 1) ? -1.0 : 1.0) * sg, cmul(x[F], x[F]));
        }
        if (F == 3) {
            // A_{2l} is a symmetric bilinear form: each unordered pair (i, ip) once,
            // off-diagonal pairs with twice the entry
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int l = qnt_l(k);
                T2 s = mk<T2>(0, 0);
#pragma unroll
                for (int i = 0; i < C; ++i) {
                    const int ip = 2 * F - l - i;
                    if (ip >= i && ip < C && qnt_entry(k, i) != 0.0)
                        caxpy(s, T((ip > i ? 2.0 : 1.0) * qnt_entry(k, i)), cmul(x[i], x[ip]));
                }
                A2[k] = s;
            }
        }
    }

    // interaction + potential + Zeeman energy density (kinetic part excluded), in T
    __device__ __forceinline__ T energy_density(const T2 (&x)[2 * F + 1], T V, const PPT<T>& pp) const {
        constexpr int C = 2 * F + 1;
        T e = V * rho;
#pragma unroll
        for (int i = 0; i < C; ++i) e += pp.bz[i] * cabs2(x[i]);
        T inter = pp.e0 * rho * rho + pp.e1 * (Fz * Fz + cabs2(Fp));
        if (F >= 2) inter += pp.e2 * cabs2(A00);
        if (F == 3) {
            T q = 0;
#pragma unroll
            for (int k = 0; k < 5; ++k) q += cabs2(A2[k]);
            inter += pp.e3 * q;
        }
        return e + inter;
    }
};

// Gradient (Eq. 3.12) at one grid point, component k, given the Laplacian term lx_k.
// The interaction prefactors are applied to the densities once per point (g1/2 F_-,
// g2 A00 / sqrt(2F+1), g3 A_{2l}), so that each component's terms are plain complex
// products with the compile-time ladder / pair constants.
template <int F, typename T2>
__device__ __forceinline__ void grad_point(const T2 (&x)[2 * F + 1], const Dens<F, T2>& D, decltype(T2::x) V,
                                           const PPT<decltype(T2::x)>& pp, const T2 (&lx)[2 * F + 1],
                                           T2 (&g)[2 * F + 1]) {
    using T = decltype(T2::x);
    constexpr int C = 2 * F + 1;
    const T gr = T(2) * V + pp.g0 * D.rho;          // 2 V + g0 rho
    const T gFz = pp.g1 * D.Fz;
    const T2 hFm = cscale(cconj(D.Fp), T(0.5) * pp.g1);
    T2 gA00 = mk<T2>(0, 0);
    if (F >= 2) gA00 = cscale(D.A00, pp.g2 * T(InvSqrtC<C>::v));
    T2 gA2[5];
    if (F == 3) {
#pragma unroll
        for (int q = 0; q < 5; ++q) gA2[q] = cscale(D.A2[q], pp.g3);
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
        T2 r = lx[k];
        caxpy(r, gr + T(2) * pp.bz[k] + T(F - k) * gFz, x[k]);
        // (g1/2) (F_- (f_+ x)_k + F_+ (f_- x)_k)
        if (k + 1 < C) cfma(r, cscale(hFm, T(Spin<F>::lad(k))), x[k + 1]);
        if (k >= 1) cfma(r, cscale(cconj(hFm), T(Spin<F>::lad(k - 1))), x[k - 1]);
        if (F >= 2) {
            const T2 t = cmul(gA00, cconj(x[C - 1 - k]));
            if (k & 1) r = csub(r, t); else r = cadd(r, t);
        }
        if (F == 3) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const int l = qnt_l(q);
                const int kp = 2 * F - l - k;
                if (kp >= 0 && kp < C && qnt_entry(q, k) != 0.0)
                    cfma(r, cscale(gA2[q], T(qnt_entry(q, k))), cconj(x[kp]));
            }
        }
        g[k] = r;
    }
}

// Hessian-vector product (Eq. 3.13) at one grid point, given lz_k = (L Z)_k.  As in
// grad_point the prefactors are applied to the densities and to their directional
// derivatives once per point; each coupling of component k is then
// c (D z_j + dD x_j) with one complex product, one complex FMA and one scaling.
template <int F, typename T2>
__device__ __forceinline__ void hess_point(const T2 (&x)[2 * F + 1], const T2 (&z)[2 * F + 1],
                                           const Dens<F, T2>& D, decltype(T2::x) V,
                                           const PPT<decltype(T2::x)>& pp, const T2 (&lz)[2 * F + 1],
                                           T2 (&hz)[2 * F + 1]) {
    using T = decltype(T2::x);
    constexpr int C = 2 * F + 1;
    // directional derivatives of the densities
    T drho = 0, dFz = 0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const T re = x[i].x * z[i].x + x[i].y * z[i].y;   // Re(conj(x) z)
        drho += re;
        dFz += T(F - i) * re;
    }
    T2 dFp = mk<T2>(0, 0);
#pragma unroll
    for (int i = 0; i < C - 1; ++i) {
        const T2 t = cadd(cmulc(z[i], x[i + 1]), cmulc(x[i], z[i + 1]));
        caxpy(dFp, T(Spin<F>::lad(i)), t);
    }
    // dA00 = 2 z^T A x and dA_{2l} = 2 z^T A_l x (directional derivatives of x^T A x)
    T2 dA00 = mk<T2>(0, 0);
    if (F >= 2) {
#pragma unroll
        for (int i = 0; i < C; ++i)
            caxpy(dA00, T(((i & 1) ? -2.0 : 2.0) * InvSqrtC<C>::v), cmul(z[i], x[C - 1 - i]));
    }
    T2 dA2[5];
    if (F == 3) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int l = qnt_l(q);
            T2 s = mk<T2>(0, 0);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int ip = 2 * F - l - i;
                if (ip >= 0 && ip < C && qnt_entry(q, i) != 0.0) caxpy(s, T(2.0 * qnt_entry(q, i)), cmul(z[i], x[ip]));
            }
            dA2[q] = s;
        }
    }
    // prefactors applied once: (g1/2) F_-, (g1/2) dF_-, g2 A00 / sqrt(2F+1),
    // g2 dA00 / sqrt(2F+1), g3 A_{2l}, g3 dA_{2l}; the scalar terms
    // 2V + g0 rho + g1 m F_z and 2 g0 Re(x^* z) + 2 g1 m Re(x^* f_z z)
    const T gr = T(2) * V + pp.g0 * D.rho;
    const T gFz = pp.g1 * D.Fz;
    const T gdr = T(2) * pp.g0 * drho, gdFz = T(2) * pp.g1 * dFz;
    const T2 hFm = cscale(cconj(D.Fp), T(0.5) * pp.g1), hdFm = cscale(cconj(dFp), T(0.5) * pp.g1);
    T2 gA00 = mk<T2>(0, 0), gdA00 = mk<T2>(0, 0);
    if (F >= 2) {
        const T sg = pp.g2 * T(InvSqrtC<C>::v);
        gA00 = cscale(D.A00, sg);
        gdA00 = cscale(dA00, sg);
    }
    T2 gA2[5];
    if (F == 3) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            gA2[q] = cscale(D.A2[q], pp.g3);
            dA2[q] = cscale(dA2[q], pp.g3);
        }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
        T2 r = lz[k];
        const T m = T(F - k);
        caxpy(r, gr + T(2) * pp.bz[k] + m * gFz, z[k]);
        caxpy(r, gdr + m * gdFz, x[k]);
        if (k + 1 < C) {
            T2 t = cmul(hFm, z[k + 1]);
            cfma(t, hdFm, x[k + 1]);
            caxpy(r, T(Spin<F>::lad(k)), t);
        }
        if (k >= 1) {
            T2 t = cmul(cconj(hFm), z[k - 1]);
            cfma(t, cconj(hdFm), x[k - 1]);
            caxpy(r, T(Spin<F>::lad(k - 1)), t);
        }
        if (F >= 2) {
            T2 t = cmul(gA00, cconj(z[C - 1 - k]));
            cfma(t, gdA00, cconj(x[C - 1 - k]));
            if (k & 1) r = csub(r, t); else r = cadd(r, t);
        }
        if (F == 3) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const int l = qnt_l(q);
                const int kp = 2 * F - l - k;
                if (kp >= 0 && kp < C && qnt_entry(q, k) != 0.0) {
                    T2 t = cmul(gA2[q], cconj(z[kp]));
                    cfma(t, dA2[q], cconj(x[kp]));
                    caxpy(r, T(qnt_entry(q, k)), t);
                }
            }
        }
        hz[k] = r;
    }
}

}  // namespace sbec
