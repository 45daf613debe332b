// Strided FFT passes with tensor-memory-accelerator (TMA) tiles, FP32 fields.
//
// The y and z passes of a 3D problem (the y pass of a 2D one) transform pencils
// whose consecutive elements lie n_x (y) or n_x n_y (z) complex values apart.  A
// tile of W consecutive x columns of one component along the whole pass axis is
// one cp.async.bulk.tensor load (a 4D tensor map over [C][n_z][n_y][2 n_x]
// floats, box [1][n][1][2W] or [1][1][n][2W]); the tile lands in shared memory as
// [e][w], e the pass-axis index, and the two-level FFT of every pencil runs from
// there.  Results are written back into the tile's own stage and stored by one
// cp.async.bulk.tensor store.  Each block is persistent over tiles with two
// stages: while it computes one tile, the load of the next is in flight, and the
// stage a store has finished reading is refilled at the start of the next tile
// (cp.async.bulk.wait_group.read), so the DMA engine keeps HBM busy while the
// block computes.  The tile width W (8, 16 or 32 columns: rows of 64, 128 or
// 256 contiguous bytes per pass-axis index) sets 4, 2 or 1 resident blocks per
// SM of the same 16 warps in all: with narrower tiles the blocks wait at their
// barriers independently, and one block's exchange overlaps another's loads and
// arithmetic (measured on the 256^3 z fwd·|k|²·inv pass: 0.49, 0.38 and 0.34 ms per
// launch for W = 32, 16, 8).
// The tensor maps cover this GPU's own memory; no cluster multicast is used.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the encoder is fetched from the driver at run time)

#include "sbec_device.cuh"

namespace sbec {

constexpr int kTmaStagesIn = 2;     // tiles in flight per block; results go back into the consumed stage
// polls of an mbarrier before a block gives up (the wait then records
// SBEC_ERR_TIMEOUT and the block returns); far beyond any real load latency
constexpr long long kTmaWaitLimit = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// one poll of phase `parity`: true once that phase has completed
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kTmaWaitLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3, const void* src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

struct TmaArgs {
    SArgs s;              // pass geometry, tables, partials, energy finalize
    long long ntiles;     // C * nouter * ntx tiles of one instance
    double* status;       // scalar block of the instance: SBEC_S_STATUS receives a timeout
};

// exchange row of the two-level FFT: N1 W slots, padded by 8 for W = 8 so that the
// four quarter-warps of a level-B read (four rows) fall on two bank halves
template <int LOGN, int W>
__host__ __device__ constexpr int tma_rs() { return Split2<LOGN>::N1 * W + (W < 16 ? 8 : 0); }
template <int LOGN, int W>
__host__ __device__ constexpr size_t tma_smem_bytes() {
    constexpr int N = 1 << LOGN;
    return (size_t)kTmaStagesIn * N * W * sizeof(float2) +
           (size_t)Split2<LOGN>::N2 * tma_rs<LOGN, W>() * sizeof(float2) + 128;   // + alignment slack
}

// Tile t -> tensor-map coordinates {2 x0, y0, z0, component} and the tile's x
// block and outer index.
template <int W>
__device__ __forceinline__ void tma_tile(const SArgs& a, long long t, int* c, int* xt, int* o) {
    *xt = (int)(t % a.ntx);
    const long long r = t / a.ntx;
    *o = (int)(r % a.nouter);
    const int comp = (int)(r / a.nouter);
    c[0] = 2 * *xt * W;
    c[1] = (a.axis == 2) ? *o : 0;
    c[2] = (a.axis == 2) ? 0 : *o;
    c[3] = comp;
}

template <int MODE, int LOGN, int W>
__global__ void __launch_bounds__(W * Split2<LOGN>::N1, 32 / W)
    k_spass_tma(const TmaArgs ta, const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout) {
    using T = float;
    using T2 = float2;
    constexpr int N = 1 << LOGN, N1 = Split2<LOGN>::N1, N2 = Split2<LOGN>::N2;
    static_assert(W == 8 || W == 16 || W == 32, "TMA tile width");
    constexpr int NS = kTmaStagesIn;
    constexpr int TILE = N * W;
    constexpr uint32_t TILE_BYTES = TILE * sizeof(T2);
    constexpr int RS = tma_rs<LOGN, W>();            // exchange row
    const SArgs& a = ta.s;
    // dynamic shared memory, rounded up to a 128-byte boundary for the TMA tiles
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* in = reinterpret_cast<T2*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));   // [NS][N][W]
    T2* ex = in + NS * TILE;                         // [N2][RS]
    __shared__ __align__(8) uint64_t bar[NS];
    // the pass's twiddles W_N^j and (S_K2, S_PARSEVAL) its axis's k-space factors,
    // read by every tile: in shared memory once per block (a warp shares one q, so
    // each read is a broadcast) instead of a global load per element and tile
    __shared__ T2 tw[N];
    __shared__ T fe[N];
    const int tid = threadIdx.x, w = tid & (W - 1), q = tid / W;
    const long long stride = gridDim.x;
    for (int j = tid; j < N; j += blockDim.x) {
        tw[j] = reinterpret_cast<const T2*>(a.tw)[j];
        if (MODE == S_K2 || MODE == S_PARSEVAL) fe[j] = reinterpret_cast<const T*>(a.k2t[a.axis])[j];
    }

    // thread 0's bookkeeping: loads issued into / consumed from each stage (the
    // pending load of stage s completes phase (consumed[s] & 1) of its mbarrier),
    // and the stage whose refill waits for its store to finish reading it
    int issued[NS], consumed[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) issued[s] = consumed[s] = 0;
    int refill = -1;
    long long refill_tile = 0;
    auto load = [&](int s, long long t) {
        int c[4], xt, o;
        tma_tile<W>(a, t, c, &xt, &o);
        fence_proxy_async();
        mbar_expect_tx(&bar[s], TILE_BYTES);
        tma_load_4d(in + s * TILE, &tin, c[0], c[1], c[2], c[3], &bar[s]);
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if (k == s) ++issued[k];
    };
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        fence_proxy_async();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            const long long t = blockIdx.x + s * stride;
            if (t < ta.ntiles) load(s, t);
        }
    }
    Acc<T> acc[1];
    bool timed_out = false;
    int it = 0;
    for (long long t = blockIdx.x; t < ta.ntiles; t += stride, ++it) {
        const int s = it % NS;
        // the previous tile's store has read its stage: that stage takes its next tile
        if (tid == 0 && refill >= 0) {
            bulk_wait_read<0>();
            load(refill, refill_tile);
            refill = -1;
        }
        const uint32_t parity = (uint32_t)((it / NS) & 1);
        const bool got = mbar_wait_bounded(&bar[s], parity);
        if (!__syncthreads_and(got)) {
            timed_out = true;
            break;
        }
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if (k == s) ++consumed[k];
        int c[4], xt, o;
        tma_tile<W>(a, t, c, &xt, &o);
        T2* tile = in + s * TILE;
        T2 v[N1];
        if (MODE != S_INV) {
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) v[j2] = tile[(q + N1 * j2) * W + w];
            level_a_fwd<T2, LOGN, false>(v, q, tw);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) ex[k2 * RS + q * W + w] = v[k2];
            __syncthreads();                           // exchange written; every read of the tile done
            if (q < N2) {
#pragma unroll
                for (int j1 = 0; j1 < N1; ++j1) v[j1] = ex[q * RS + j1 * W + w];
                RegDft<T2, N1, false>::run(v);          // v[k1] = X[q + N2 k1]
            }
        } else {
            if (q < N2) {
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) v[k1] = tile[(q + N2 * k1) * W + w];
            }
            __syncthreads();                           // every read of the tile done
        }
        if (MODE == S_K2 || MODE == S_PARSEVAL) {
            if (q < N2) {
                const int ix = xt * W + w;
                const bool ya = (a.axis == 1);
                const T f0 = reinterpret_cast<const T*>(a.k2t[0])[ix] +
                             reinterpret_cast<const T*>(a.k2t[ya ? 2 : 1])[o];
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    const T f = f0 + fe[q + N2 * k1];
                    if (MODE == S_K2) v[k1] = cscale(v[k1], f);
                    else acc[0].add(T(0.5) * f * cabs2(v[k1]));
                }
            }
        }
        // results go back into the tile's own stage (its reads ended at the barrier above)
        if (MODE == S_FWD && q < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) tile[(q + N2 * k1) * W + w] = v[k1];
        }
        if (MODE == S_K2 || MODE == S_INV) {
            // inverse: level B' (k2 = q; its exchange slots are this thread's own), exchange, level A'
            if (q < N2) {
                level_b_inv<T2, LOGN>(v, q, tw);
#pragma unroll
                for (int j1 = 0; j1 < N1; ++j1) ex[q * RS + j1 * W + w] = v[j1];
            }
            __syncthreads();
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k2] = ex[k2 * RS + q * W + w];
            RegDft<T2, N2, true>::run(v);              // v[j2] = x[q + N1 j2]
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) tile[(q + N1 * j2) * W + w] = v[j2];
        }
        if (MODE != S_PARSEVAL) fence_proxy_async();
        __syncthreads();                               // results written, exchange reads done
        if (tid == 0) {
            const long long tn = t + NS * stride;
            if (MODE != S_PARSEVAL) {
                tma_store_4d(&tout, c[0], c[1], c[2], c[3], tile);
                bulk_commit();
                if (tn < ta.ntiles) { refill = s; refill_tile = tn; }    // after the store has read the stage
            } else if (tn < ta.ntiles) {
                load(s, tn);
            }
        }
    }
    if (tid == 0) {
        bulk_wait<0>();                                // no store outlives the block
        if (timed_out) {
            // loads still in flight land in this block's shared memory: wait for them
            // (bounded) before the block exits, and record the timeout
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (issued[s] > consumed[s]) mbar_wait_bounded(&bar[s], (uint32_t)(consumed[s] & 1));
            if (ta.status && ta.status[SBEC_S_STATUS] == 0.0) ta.status[SBEC_S_STATUS] = double(SBEC_ERR_TIMEOUT);
        }
    }
    if (MODE == S_PARSEVAL) {
        __syncthreads();
        double r[1];
        acc_values(acc, r);
        block_reduce_store<1>(r, a.partials, gridDim.x, blockIdx.x);
        if (a.fe.on && last_block(a.fe.scal0, gridDim.x))
            fin_energy_body(a.fe.pa, a.fe.na_tot, a.fe.na_inst, 1, a.partials, gridDim.x, gridDim.x, a.fe.scal0, 0, 0);
    }
}

}  // namespace sbec
