// Allocation-free energy entry point.
//
// Some callers cannot allocate device memory at the point where they need an
// energy value: a host framework that owns every byte of device memory through
// its own pool and forbids allocations behind its back, or a latency-critical
// loop that must not pay for cudaMalloc/cudaFree, which can block until the
// whole device is idle.  sbec_energy_noalloc serves them: it takes the problem,
// the potential and the state from the caller and does all of its intermediate
// work (FFT tables, the transformed field, per-block partial sums, the scalar
// block) in one fixed array of device memory that is part of the library
// image, so it needs no handle and allocates nothing.
#include <math.h>

#include <atomic>

#include <cuda_runtime.h>

#include "sbec.h"
#include "sbec_internal.h"

namespace {

// 2^20 doubles = 8 MiB.  Every GPU that loads the library keeps this array
// until the process exits.
constexpr size_t kScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of g_noalloc_scratch per device ordinal; in host code the
// array's name only stands in for the symbol, it is not a device address.
// Atomic entries: host threads may make their first calls concurrently (they
// would store the same address, but plain stores would still race).
constexpr int kMaxDevices = 64;
static std::atomic<double*> g_scratch_addr[kMaxDevices];

// lambda_p^2 = (2 pi p / (b - a))^2 per axis, p the signed DFT frequency (Eq. 3.6);
// unused axes (n = 1) get 0.
__global__ void k_noalloc_lam2(double* lam, int n0, int n1, int n2, double L0, double L1, double L2) {
    const int total = n0 + n1 + n2;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        int ax = 0, i = j, n = n0;
        double L = L0;
        if (i >= n0) { i -= n0; ax = 1; n = n1; L = L1; }
        if (ax == 1 && i >= n1) { i -= n1; ax = 2; n = n2; L = L2; }
        const int p = (i < n / 2) ? i : i - n;
        const double lp = (n > 1) ? 2.0 * M_PI * (double)p / L : 0.0;
        lam[j] = lp * lp;
    }
}

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }
int lg2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }
size_t up256(size_t doubles) { return (doubles + 31) & ~size_t(31); }   // 256-byte slots

// Once per device, with that device current: look up the array's device address.
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SBEC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return SBEC_ERR_ARG;
    double* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SBEC_ERR_CUDA;
        }
        addr = static_cast<double*>(p);
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    *out = addr;
    return SBEC_OK;
}

// p is memory of the current device that kernels may read: device or managed
// memory of device `dev`.  The kernels of this entry point read X and V in place
// (there is no staging area to copy host arrays into), so a host or peer-device
// pointer is rejected here instead of being dereferenced on the GPU.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    if (at.type == cudaMemoryTypeManaged) return at.device == dev || at.device < 0;
    return false;
}

}  // namespace

extern "C" int sbec_energy_noalloc(const sbec_problem* prob, const double* V, const void* X, double* E,
                                   void* cuda_stream) {
    if (!prob || !X || !E) return SBEC_ERR_ARG;
    const sbec_problem& P = *prob;
    if (P.F < 1 || P.F > sbec::kMaxF || P.dim < 1 || P.dim > 3) return SBEC_ERR_ARG;
    if (P.precision != SBEC_FP64) return SBEC_ERR_ARG;
    if (!(fabs(P.M) < (double)P.F)) return SBEC_ERR_ARG;
    for (int ax = 0; ax < 3; ++ax) {
        if (ax < P.dim) {
            if (!pow2(P.n[ax]) || P.n[ax] < 2 || P.n[ax] > 1024 || !(P.hi[ax] > P.lo[ax])) return SBEC_ERR_ARG;
        } else if (P.n[ax] != 1) {
            return SBEC_ERR_ARG;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* base = nullptr;
    if (int st = scratch_for_current_device(&base)) return st;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (!on_device(X, dev) || (V && !on_device(V, dev))) return SBEC_ERR_ARG;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // geometry and parameters of the problem (Sec. 3 with h -> dV)
    sbec::Geom g = {};
    g.F = P.F; g.C = 2 * P.F + 1; g.dim = P.dim;
    g.B = 1;
    g.nl = 1;
    g.imap = nullptr;
    double dV = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        g.n[ax] = P.n[ax];
        g.logn[ax] = lg2(P.n[ax]);
        if (ax < P.dim) dV *= (P.hi[ax] - P.lo[ax]) / P.n[ax];
    }
    g.G = (long long)P.n[0] * P.n[1] * P.n[2];
    g.dV = dV; g.invG = 1.0 / (double)g.G; g.M = P.M;
    for (int i = 0; i < sbec::kMaxC; ++i) {
        const double l = (double)(P.F - i);
        g.bz[i] = (i < g.C) ? (-P.p * l + P.q * l * l) : 0.0;
    }
    const double b0 = P.beta[0], b1 = P.beta[1];
    const double b2 = P.F >= 2 ? P.beta[2] : 0.0, b3 = P.F == 3 ? P.beta[3] : 0.0;
    g.g0 = 2 * b0 / dV; g.g1 = 2 * b1 / dV; g.g2 = 2 * b2 / dV; g.g3 = 2 * b3 / dV;
    g.e0 = b0 / (2 * dV); g.e1 = b1 / (2 * dV); g.e2 = b2 / (2 * dV); g.e3 = b3 / (2 * dV);

    // carve the fixed array: twiddles, lambda^2, potential (when V is NULL), the
    // transformed field, two partial-sum areas and the scalar block
    const size_t ntw = (size_t)P.n[0] + P.n[1] + P.n[2];
    const size_t part = sbec::Ops<double>::partials_needed(g, sms > 0 ? sms : 1, false);
    size_t off = 0;
    const size_t o_tw = off;   off += up256(2 * ntw);
    const size_t o_lam = off;  off += up256(ntw);
    const size_t o_V = off;    off += V ? 0 : up256((size_t)g.G);
    const size_t o_work = off; off += up256(2 * (size_t)g.C * (size_t)g.G);
    const size_t o_pa = off;   off += up256(part);
    const size_t o_pb = off;   off += up256(part);
    const size_t o_sc = off;   off += up256(sbec::S_COUNT);
    if (off > kScratchDoubles) return SBEC_ERR_ARG;   // problem too large for the fixed 8 MiB array

    // Only FP64 reaches the kernels here: their FP64 branches read lam2 and invG,
    // never the lambda^2 / G tables of the FP32 passes (g.k2s), which this entry
    // point does not build and leaves null.
    sbec::Work w = {};
    w.work = base + o_work;
    w.work2 = nullptr;
    w.partA = base + o_pa;
    w.partB = base + o_pb;
    w.part_cap = part;
    w.scal = base + o_sc;
    w.num_sms = sms > 0 ? sms : 1;
    w.prof = nullptr;
    double* lam = base + o_lam;
    for (int ax = 0, acc = 0; ax < 3; ++ax) { g.lam2[ax] = lam + acc; acc += P.n[ax]; }

    // the array keeps the previous call's contents: the scalar block (status
    // slot included) must start at zero; everything else is rewritten below
    if (cudaMemsetAsync(w.scal, 0, sbec::S_COUNT * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return SBEC_ERR_CUDA;
    }
    const double L0 = P.hi[0] - P.lo[0];
    const double L1 = P.dim > 1 ? P.hi[1] - P.lo[1] : 1.0, L2 = P.dim > 2 ? P.hi[2] - P.lo[2] : 1.0;
    k_noalloc_lam2<<<1, 256, 0, s>>>(lam, P.n[0], P.n[1], P.n[2], L0, L1, L2);
    if (cudaGetLastError() != cudaSuccess) return SBEC_ERR_CUDA;
    int st = sbec::Ops<double>::init_tables(g, base + o_tw, s);
    if (st) return st;
    if (V) {
        g.V = V;
    } else {
        g.V = base + o_V;
        st = sbec::Ops<double>::harmonic_potential(g, base + o_V, P.lo, P.hi, s);
        if (st) return st;
    }
    st = sbec::Ops<double>::energy(g, w, X, s);
    if (st) return st;
    double host[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(&host[0], w.scal + SBEC_S_ENERGY, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&host[1], w.scal + SBEC_S_STATUS, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SBEC_ERR_CUDA;
    }
    *E = host[0];
    return (int)host[1];
}
