// Persistent, TMA-staged form of the Chebyshev term kernel (a3).
//
// The plain term kernel spends most of its time waiting on a dependent
// chain per thread: slice offset -> column/value -> gathered vector, with
// short block lifetimes.  This form keeps one or two blocks per SM resident
// for the whole sweep and moves every row-contiguous stream of a tile
// (psi, z and x at the own rows, the tile's sliced-ELLPACK columns and
// values, the diagonal) from HBM into shared memory with bulk asynchronous
// copies (cp.async.bulk, completion counted on an mbarrier), STAGES tiles
// ahead of the computation.  Only the gathers x[col] stay on the critical
// path, and those mostly hit L2 because all blocks sweep the rows together.
//
// The arithmetic per row is exactly that of k_term (same operation order),
// so both forms give bit-identical states.  Every wait on an mbarrier is
// bounded; on expiry the block records TBPM_E_TIMEOUT's flag, waits (again
// bounded) for its own copies in flight, and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kStages = 3;
constexpr long long kWaitLimit = 1ll << 22;   // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the phase did not complete within kWaitLimit rounds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this block's shared memory, counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <typename V, int SPL> struct LaneT2;
template <> struct LaneT2<double, 1> { typedef double2 type; };
template <> struct LaneT2<float, 1> { typedef float2 type; };
template <> struct LaneT2<float, 2> { typedef float4 type; };

template <typename V, int SPL> struct Cx {
    V re[SPL], im[SPL];
};
__device__ __forceinline__ void unp(const double2 &v, Cx<double, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unp(const float2 &v, Cx<float, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unp(const float4 &v, Cx<float, 2> &o)
{
    o.re[0] = v.x; o.im[0] = v.y; o.re[1] = v.z; o.im[1] = v.w;
}
__device__ __forceinline__ double2 pk(const Cx<double, 1> &o) { return make_double2(o.re[0], o.im[0]); }
__device__ __forceinline__ float2 pk(const Cx<float, 1> &o) { return make_float2(o.re[0], o.im[0]); }
__device__ __forceinline__ float4 pk(const Cx<float, 2> &o)
{
    return make_float4(o.re[0], o.im[0], o.re[1], o.im[1]);
}

template <typename V> struct CoefT;
template <> struct CoefT<double> {
    __device__ static double g(const TermArgs &a) { return a.gamma; }
    __device__ static double hi(const TermArgs &a) { return a.c_hi; }
    __device__ static double lo(const TermArgs &a) { return a.c_lo; }
    __device__ static const double *scale(const TermArgs &a) { return a.scale; }
};
template <> struct CoefT<float> {
    __device__ static float g(const TermArgs &a) { return a.gamma_f; }
    __device__ static float hi(const TermArgs &a) { return a.c_hi_f; }
    __device__ static float lo(const TermArgs &a) { return a.c_lo_f; }
    __device__ static const float *scale(const TermArgs &a) { return a.scale_f; }
};

// Shared-memory layout of one stage (byte offsets, 128-byte aligned parts).
struct StageLayout {
    uint32_t psi, z, xo, col, val, diag, bytes;
};

__host__ __device__ inline uint32_t align128(uint32_t v) { return (v + 127u) & ~127u; }

__host__ __device__ inline StageLayout stage_layout(int tile_rows, int row_bytes, int max_width,
                                                    int val_bytes)
{
    StageLayout s;
    uint32_t o = 0;
    s.psi = o; o = align128(o + tile_rows * row_bytes);
    s.z = o; o = align128(o + tile_rows * row_bytes);
    s.xo = o; o = align128(o + tile_rows * row_bytes);
    s.col = o; o = align128(o + tile_rows * max_width * 4);
    s.val = o; o = align128(o + tile_rows * max_width * val_bytes);
    s.diag = o; o = align128(o + tile_rows * val_bytes);
    s.bytes = o;
    return s;
}

template <typename V, int L, int SPL>
__global__ void __launch_bounds__(1024) k_term_tma(TermArgs a, int tile_rows, int max_width,
                                                   int *err)
{
    typedef typename LaneT2<V, SPL>::type Lane;
    constexpr int B = L * SPL;
    constexpr int row_bytes = B * 2 * (int)sizeof(V);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    __shared__ int abort_flag;
    const StageLayout lay = stage_layout(tile_rows, row_bytes, max_width, (int)sizeof(V));
    unsigned char *stage0 = smem + 128;
    const int64_t n_tiles = a.n_rows / tile_rows;
    const int tid = threadIdx.x;
    const int lr = tid / L, l = tid % L;
    const bool has_z = a.z != nullptr;
    const bool has_x_own = !a.x_is_psi;   // x == psi: reuse the psi stage

    auto tile_of = [&](int64_t i) -> int64_t { return a.reverse ? n_tiles - 1 - i : i; };

    // one thread issues all copies of a tile into stage s
    auto issue = [&](int s, int64_t tile) {
        unsigned char *st = stage0 + (size_t)s * lay.bytes;
        const int64_t r0 = tile * tile_rows;
        const int64_t q0 = r0 / kSliceRows, q1 = (r0 + tile_rows) / kSliceRows;
        const int64_t e0 = a.H.slice_ptr[q0], e1 = a.H.slice_ptr[q1];
        const uint32_t vec = (uint32_t)(tile_rows * row_bytes);
        const uint32_t ne = (uint32_t)(e1 - e0);
        uint32_t total = vec + (has_z ? vec : 0) + (has_x_own ? vec : 0) + ne * 4u +
                         ne * (uint32_t)sizeof(V) + (uint32_t)(tile_rows * sizeof(V));
        mbar_expect_tx(&bars[s], total);
        bulk_g2s(st + lay.psi, reinterpret_cast<const unsigned char *>(a.psi) + r0 * row_bytes,
                 vec, &bars[s]);
        if (has_z)
            bulk_g2s(st + lay.z, reinterpret_cast<const unsigned char *>(a.z) + r0 * row_bytes, vec,
                     &bars[s]);
        if (has_x_own)
            bulk_g2s(st + lay.xo, reinterpret_cast<const unsigned char *>(a.x) + r0 * row_bytes,
                     vec, &bars[s]);
        if (ne) {
            bulk_g2s(st + lay.col, a.H.col + e0, ne * 4u, &bars[s]);
            bulk_g2s(st + lay.val, reinterpret_cast<const V *>(a.H.val) + e0,
                     ne * (uint32_t)sizeof(V), &bars[s]);
        }
        bulk_g2s(st + lay.diag, reinterpret_cast<const V *>(a.H.diag) + r0,
                 (uint32_t)(tile_rows * sizeof(V)), &bars[s]);
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < kStages; ++s) {
            const int64_t i = blockIdx.x + (int64_t)s * gridDim.x;
            if (i < n_tiles) issue(s, tile_of(i));
        }

    const V g = CoefT<V>::g(a), ch = CoefT<V>::hi(a), cl = CoefT<V>::lo(a);
    int k = 0;
    for (int64_t i = blockIdx.x; i < n_tiles; i += gridDim.x, ++k) {
        const int s = k % kStages;
        const uint32_t parity = (uint32_t)((k / kStages) & 1);
        if (tid == 0 && !mbar_wait_bounded(&bars[s], parity)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            if (tid == 0) {
                atomicOr(err, 4);
                // wait (bounded) for this block's copies still in flight
                for (int d = 0; d < kStages; ++d) {
                    const int64_t j = i + (int64_t)d * gridDim.x;
                    if (j < n_tiles)
                        mbar_wait_bounded(&bars[(k + d) % kStages],
                                          (uint32_t)(((k + d) / kStages) & 1));
                }
            }
            return;
        }
        mbar_try_wait(&bars[s], parity);   // completed: acquire for this thread
        const int64_t tile = tile_of(i);
        const unsigned char *st = stage0 + (size_t)s * lay.bytes;
        const int64_t r = tile * tile_rows + lr;
        const Lane *sp = reinterpret_cast<const Lane *>(st + lay.psi);
        const Lane *sz = reinterpret_cast<const Lane *>(st + lay.z);
        const Lane *sx = reinterpret_cast<const Lane *>(has_x_own ? st + lay.xo : st + lay.psi);
        const int32_t *scol = reinterpret_cast<const int32_t *>(st + lay.col);
        const V *sval = reinterpret_cast<const V *>(st + lay.val);
        const V *sdiag = reinterpret_cast<const V *>(st + lay.diag);

        Cx<V, SPL> p, zz, y;
        unp(sp[lr * L + l], p);
        if (has_z) {
            unp(sz[lr * L + l], zz);
        } else {
#pragma unroll
            for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
        }
        // slice of this row within the tile's entries
        const int64_t q = r / kSliceRows;
        const int64_t qb = tile * tile_rows / kSliceRows;
        const int64_t eb = __ldg(a.H.slice_ptr + qb);
        const int64_t es = __ldg(a.H.slice_ptr + q);
        const int w = (int)((__ldg(a.H.slice_ptr + q + 1) - es) / kSliceRows);
        const int32_t *colp = scol + (es - eb) + (lr % kSliceRows);
        const V *valp = sval + (es - eb) + (lr % kSliceRows);
        const V d = sdiag[lr];
        unp(sx[lr * L + l], y);
        const Lane *xg = reinterpret_cast<const Lane *>(a.x);
        const V *sc = CoefT<V>::scale(a);
        if (sc) sc += (int64_t)a.chunk_sample[r / kChunkRows] * B;
        Cx<V, SPL> o;
        bool summed = false;
        if constexpr (sizeof(V) == 8) {
            if (a.uniform) {
                // FP64 one-value form, as in the per-term kernels: the
                // neighbours summed in stored order, then
                // fma(gh, s, fma(gd, x_r, fma(c, psi, z)))
                summed = true;
                Cx<V, SPL> sm;
#pragma unroll
                for (int j = 0; j < SPL; ++j) { sm.re[j] = 0; sm.im[j] = 0; }
                auto group = [&](int kk, auto first) {
                    int32_t c[4];
                    bool ok[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        ok[u] = kk + u < w;
                        c[u] = ok[u] ? colp[(kk + u) * kSliceRows] : (int32_t)r;
                        ok[u] = ok[u] && c[u] != (int32_t)r;     // padding: the own row
                    }
                    Cx<V, SPL> xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) unp(__ldg(xg + (int64_t)c[u] * L + l), xv[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (decltype(first)::value && u == 0) {
#pragma unroll
                            for (int j = 0; j < SPL; ++j) {
                                sm.re[j] = ok[0] ? xv[0].re[j] : 0.0;
                                sm.im[j] = ok[0] ? xv[0].im[j] : 0.0;
                            }
                        } else if (ok[u]) {
#pragma unroll
                            for (int j = 0; j < SPL; ++j) {
                                sm.re[j] += xv[u].re[j];
                                sm.im[j] += xv[u].im[j];
                            }
                        }
                    }
                };
                if (w > 0) {
                    group(0, std::true_type{});
                    for (int kk = 4; kk < w; kk += 4) group(kk, std::false_type{});
                }
                if (sc) {
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        const V sv = sc[l * SPL + j];
                        p.re[j] *= sv;
                        p.im[j] *= sv;
                        if (a.x_is_psi) {
                            sm.re[j] *= sv;
                            sm.im[j] *= sv;
                            y.re[j] *= sv;
                            y.im[j] *= sv;
                        }
                    }
                }
                const V gd = a.zero_diag ? 0.0
                             : a.gdiag   ? xor_sign(__ldg(a.gdiag + r), a.gdiag_sign)
                                         : a.gamma * d;
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    V re = fma(ch, p.re[j], zz.re[j]);
                    V im = fma(ch, p.im[j], zz.im[j]);
                    if (!a.zero_diag) {
                        re = fma(gd, y.im[j], re);            // y holds x_r here
                        im = fma(-gd, y.re[j], im);
                    }
                    o.re[j] = fma(a.gh, sm.im[j], re);
                    o.im[j] = fma(-a.gh, sm.re[j], im);
                }
            }
        }
        if (!summed) {
#pragma unroll
            for (int j = 0; j < SPL; ++j) { y.re[j] *= d; y.im[j] *= d; }
            for (int kk = 0; kk < w; kk += 4) {
                int32_t c[4];
                V h[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = kk + u < w;
                    c[u] = ok ? colp[(kk + u) * kSliceRows] : (int32_t)r;
                    h[u] = ok ? valp[(kk + u) * kSliceRows] : (V)0;
                }
                Cx<V, SPL> xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) unp(__ldg(xg + (int64_t)c[u] * L + l), xv[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kk + u < w) {
#pragma unroll
                        for (int j = 0; j < SPL; ++j) {
                            y.re[j] = fma(h[u], xv[u].re[j], y.re[j]);
                            y.im[j] = fma(h[u], xv[u].im[j], y.im[j]);
                        }
                    }
                }
            }
            if (sc) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    const V sv = sc[l * SPL + j];
                    p.re[j] *= sv;
                    p.im[j] *= sv;
                    if (a.x_is_psi) { y.re[j] *= sv; y.im[j] *= sv; }
                }
            }
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                V re = fma(g, y.im[j], zz.re[j]);
                V im = fma(-g, y.re[j], zz.im[j]);
                if (sizeof(V) == 4) {
                    re = fma(cl, p.re[j], re);
                    im = fma(cl, p.im[j], im);
                }
                o.re[j] = fma(ch, p.re[j], re);
                o.im[j] = fma(ch, p.im[j], im);
            }
        }
        reinterpret_cast<Lane *>(a.out)[r * L + l] = pk(o);
        __syncthreads();          // stage s is free again
        if (tid == 0) {
            const int64_t nxt = i + (int64_t)kStages * gridDim.x;
            if (nxt < n_tiles) {
                // order this block's reads of the stage before the async refill
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(s, tile_of(nxt));
            }
        }
    }
}

template <typename V, int L, int SPL>
cudaError_t launch_tma_t(const TermArgs &a, int max_width, int *err, int num_sms,
                         cudaStream_t st)
{
    constexpr int B = L * SPL;
    constexpr int row_bytes = B * 2 * (int)sizeof(V);
    int tile_rows = 1024 / L;
    if (tile_rows > 256) tile_rows = 256;
    StageLayout lay = stage_layout(tile_rows, row_bytes, max_width, (int)sizeof(V));
    while (tile_rows > 32 && 128 + (size_t)kStages * lay.bytes > 200 * 1024) {
        tile_rows /= 2;
        lay = stage_layout(tile_rows, row_bytes, max_width, (int)sizeof(V));
    }
    const size_t smem = 128 + (size_t)kStages * lay.bytes;
    if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
    const int threads = tile_rows * L;
    cudaError_t e = cudaFuncSetAttribute(k_term_tma<V, L, SPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_term_tma<V, L, SPL>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t n_tiles = a.n_rows / tile_rows;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    k_term_tma<V, L, SPL><<<(unsigned)grid, threads, smem, st>>>(a, tile_rows, max_width, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_term_tma(const TermArgs &a, int fp32, int B, int max_width, int *err,
                            int num_sms, cudaStream_t st)
{
    if (max_width < 1) max_width = 1;
    if (!fp32) {
        switch (B) {
        case 1: return launch_tma_t<double, 1, 1>(a, max_width, err, num_sms, st);
        case 2: return launch_tma_t<double, 2, 1>(a, max_width, err, num_sms, st);
        case 4: return launch_tma_t<double, 4, 1>(a, max_width, err, num_sms, st);
        case 8: return launch_tma_t<double, 8, 1>(a, max_width, err, num_sms, st);
        }
    } else {
        switch (B) {
        case 1: return launch_tma_t<float, 1, 1>(a, max_width, err, num_sms, st);
        case 2: return launch_tma_t<float, 1, 2>(a, max_width, err, num_sms, st);
        case 4: return launch_tma_t<float, 2, 2>(a, max_width, err, num_sms, st);
        case 8: return launch_tma_t<float, 4, 2>(a, max_width, err, num_sms, st);
        case 16: return launch_tma_t<float, 8, 2>(a, max_width, err, num_sms, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tbpm
