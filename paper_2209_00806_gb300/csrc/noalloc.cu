// Allocation-free correlation reduction.
//
// Some callers cannot allocate device memory: a host framework whose own
// pool owns the whole device and rejects allocations made behind its back,
// a plugin that may only allocate at start-up, or a latency-bound loop that
// cannot afford cudaMalloc/cudaFree, which may synchronise the device.
// tbpm_correlation_noalloc serves them: it computes the same quantities as
// the closing term of tbpm_propagate, per-state <psi0|phi> and <phi|phi>,
// summed deterministically in FP64 but in its own order (caller-order rows,
// grid-stride per block), so the two agree to rounding, not bit for bit.
// Its scratch (per-block partial sums and the finishing tickets) lives in a
// fixed, file-scope device array instead of buffers from cudaMalloc.
//
// The array is a static __device__ symbol, so every GPU that loads this
// library holds it (kScratchBytes, under 1 MB) until the process exits.  In
// host code the symbol's name is only a host-side stand-in: the device
// address is looked up with cudaGetSymbolAddress once per device, on the
// first call made on that device (with that device current), and cached
// per device ordinal for the life of the process.  Make that first call
// before any stream capture begins.  The cached address is the one of the
// device's primary context: after cudaDeviceReset, or under a non-primary
// context, it would be stale, so neither is supported.  All calls share
// the one array, so calls whose kernels overlap on the GPU (different
// streams, or different host threads on one device) race and must be
// serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kNaMaxStates = 16;     // states per call
constexpr int kNaBlocks = 2048;      // blocks per state (grid-stride over rows)
constexpr int kNaThreads = 256;

struct NoAllocScratch {
    double partial[kNaMaxStates][kNaBlocks][3];   // per-block (re, im, norm) sums
    unsigned int ticket[kNaMaxStates];             // finished blocks per state
};
constexpr size_t kScratchBytes = sizeof(NoAllocScratch);

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_na_mutex;
NoAllocScratch *g_na_addr[64] = {nullptr};   // device address per device ordinal

// Per-state sums over rows of the caller-order vectors psi0[s][n], phi[s][n]
// (complex128).  Block b of state s takes rows b*T + t, b*T + t + B*T, ...
// (fixed assignment), sums them in FP64, reduces the block in a fixed tree,
// and the last block of the state (ticket after a fence) adds the block sums
// in block order.  Deterministic, FP64 throughout; the order differs from
// the closing term's (which sums internally ordered rows in 1024-row
// chunks), so the results agree with it to rounding.
__global__ void __launch_bounds__(kNaThreads) k_corr_noalloc(NoAllocScratch *scr,
                                                           const double2 *psi0,
                                                           const double2 *phi, int64_t n,
                                                           double2 *corr_out, double *norm_out)
{
    __shared__ double red[kNaThreads / 32][3];
    __shared__ int last;
    const int s = blockIdx.y;
    const double2 *p0 = psi0 + (int64_t)s * n;
    const double2 *ph = phi + (int64_t)s * n;
    double dre = 0.0, dim = 0.0, nrm = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kNaThreads + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kNaThreads) {
        const double2 a = p0[r], o = ph[r];
        dre = fma(a.x, o.x, fma(a.y, o.y, dre));
        dim = fma(a.x, o.y, fma(-a.y, o.x, dim));
        nrm = fma(o.x, o.x, fma(o.y, o.y, nrm));
    }
    for (int off = 16; off > 0; off >>= 1) {
        dre += __shfl_xor_sync(0xffffffffu, dre, off);
        dim += __shfl_xor_sync(0xffffffffu, dim, off);
        nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
    }
    const int w = threadIdx.x / 32;
    if (threadIdx.x % 32 == 0) {
        red[w][0] = dre;
        red[w][1] = dim;
        red[w][2] = nrm;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) v += red[k][threadIdx.x];
        scr->partial[s][blockIdx.x][threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&scr->ticket[s], 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(&scr->partial[s][b][threadIdx.x]);
            if (threadIdx.x == 0) corr_out[s].x = v;
            if (threadIdx.x == 1) corr_out[s].y = v;
            if (threadIdx.x == 2) norm_out[s] = v;
        }
    }
}

int na_fail(int code, const std::string &m)
{
    set_thread_error(m);     // read back with tbpm_last_error(NULL)
    return code;
}

}  // namespace
}  // namespace tbpm

using namespace tbpm;

// The closing reduction's quantities for caller-held device vectors, with
// no device allocation.  Declared in include/tbpm.h.
extern "C" int tbpm_correlation_noalloc(const double *psi0, const double *phi, int64_t n_orb,
                                        int n_states, double *corr_out, double *norm_out,
                                        void *cuda_stream)
{
    if (!psi0 || !phi || !corr_out || !norm_out || n_orb < 1)
        return na_fail(TBPM_E_INVALID_ARG, "tbpm_correlation_noalloc: NULL pointer or n_orb < 1");
    if (n_states < 1 || n_states > kNaMaxStates)
        return na_fail(TBPM_E_INVALID_ARG,
                       "tbpm_correlation_noalloc: n_states must be 1.." +
                           std::to_string(kNaMaxStates) + " (the fixed scratch holds " +
                           std::to_string(kScratchBytes) + " bytes)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(TBPM_E_CUDA, std::string("tbpm_correlation_noalloc: no current device: ") +
                                        cudaGetErrorString(e));
    if (dev < 0 || dev >= 64)
        return na_fail(TBPM_E_UNSUPPORTED, "tbpm_correlation_noalloc: device ordinal " +
                                               std::to_string(dev) + " exceeds 63");
    NoAllocScratch *scr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            // one-time set-up on this device (the caller's current device)
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(TBPM_E_CUDA,
                               std::string("tbpm_correlation_noalloc: cudaGetSymbolAddress: ") +
                                   cudaGetErrorString(e));
            g_na_addr[dev] = static_cast<NoAllocScratch *>(p);
        }
        scr = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the tickets must start at zero; the partial sums are overwritten
    e = cudaMemsetAsync(scr->ticket, 0, sizeof(scr->ticket), st);
    if (e != cudaSuccess)
        return na_fail(TBPM_E_CUDA, std::string("tbpm_correlation_noalloc: ") + cudaGetErrorString(e));
    int64_t want = (n_orb + kNaThreads - 1) / kNaThreads;
    const int blocks = (int)(want < kNaBlocks ? want : kNaBlocks);
    k_corr_noalloc<<<dim3(blocks, n_states), kNaThreads, 0, st>>>(
        scr, reinterpret_cast<const double2 *>(psi0), reinterpret_cast<const double2 *>(phi),
        n_orb, reinterpret_cast<double2 *>(corr_out), norm_out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return na_fail(TBPM_E_CUDA, std::string("tbpm_correlation_noalloc: launch: ") +
                                        cudaGetErrorString(e));
    return TBPM_OK;
}
