// Wavefront-fused time step: all M-1 Clenshaw terms of one step in one
// persistent launch (a3 + a4).
//
// The per-term kernels stream four state vectors through HBM for every term
// (15 terms per step at z = pi/2).  Here the work of one step is cut into
// items (term j, row tile t).  Term j at tile t gathers the output of term
// j-1 at the tiles t-d .. t+d (d = the matrix bandwidth in tiles) and
// overwrites, in place, the output of term j-2 at tile t.  Items are handed
// out by one atomic counter in the order of the key k = t + j (d + 1): every
// item an item depends on -- (j-1, t') for |t' - t| <= d, which also covers
// the readers of the vector it overwrites -- has a smaller key, so it was
// handed out earlier to a block that is running (the grid is launched
// cooperatively, all blocks resident), and the scheme cannot deadlock.  The
// wavefront touches only a band of rows of each vector at a time, so the
// intermediate vectors are written and re-read in the 129 MB L2 instead of
// HBM; HBM sees psi, the matrix and the write-backs.
//
// Dependencies are per-item flags holding the step's epoch, published with
// a fence after the block's writes and polled with acquire loads; reads of
// vectors written during the launch bypass L1 (ld.global.cg).  Every poll is
// bounded: on expiry the block sets the TBPM_E_TIMEOUT flag and carries on,
// so a fault ends the launch with an error status instead of a hang.
// The arithmetic of each row is that of k_term, in the same order, so the
// fused step gives bit-identical states.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kFusedThreads = 512;
constexpr long long kPollLimit = 1ll << 22;

template <typename V, int SPL> struct LaneF;
template <> struct LaneF<double, 1> { typedef double2 type; };
template <> struct LaneF<float, 1> { typedef float2 type; };
template <> struct LaneF<float, 2> { typedef float4 type; };

template <typename V, int SPL> struct Cf {
    V re[SPL], im[SPL];
};
__device__ __forceinline__ void unpf(const double2 &v, Cf<double, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unpf(const float2 &v, Cf<float, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unpf(const float4 &v, Cf<float, 2> &o)
{
    o.re[0] = v.x; o.im[0] = v.y; o.re[1] = v.z; o.im[1] = v.w;
}
__device__ __forceinline__ double2 pkf(const Cf<double, 1> &o) { return make_double2(o.re[0], o.im[0]); }
__device__ __forceinline__ float2 pkf(const Cf<float, 1> &o) { return make_float2(o.re[0], o.im[0]); }
__device__ __forceinline__ float4 pkf(const Cf<float, 2> &o)
{
    return make_float4(o.re[0], o.im[0], o.re[1], o.im[1]);
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename V> struct FCoef;
template <> struct FCoef<double> {
    __device__ static double g(const FusedTerm &t) { return t.gamma; }
    __device__ static double hi(const FusedTerm &t) { return t.c_hi; }
    __device__ static double lo(const FusedTerm &t) { return t.c_lo; }
    __device__ static const double *scale(const FusedArgs &f) { return f.scale; }
};
template <> struct FCoef<float> {
    __device__ static float g(const FusedTerm &t) { return t.gamma_f; }
    __device__ static float hi(const FusedTerm &t) { return t.c_hi_f; }
    __device__ static float lo(const FusedTerm &t) { return t.c_lo_f; }
    __device__ static const float *scale(const FusedArgs &f) { return f.scale_f; }
};

// out = c psi + gamma (-i)(H~ x) + z for lane l of row r (same operation
// order as k_term).  x and z may have been written earlier in this launch by
// other blocks: read through L2 only.
template <typename V, int L, int SPL>
__device__ __forceinline__ Cf<V, SPL> fused_row(const FusedArgs &f, const FusedTerm &tm,
                                                const void *x, const void *z, int64_t r, int l,
                                                const V *sc)
{
    typedef typename LaneF<V, SPL>::type Lane;
    Cf<V, SPL> p, zz;
    unpf(__ldg(reinterpret_cast<const Lane *>(f.psi) + r * L + l), p);
    if (z) {
        unpf(__ldcg(reinterpret_cast<const Lane *>(z) + r * L + l), zz);
    } else {
#pragma unroll
        for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
    }
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    const int64_t base = __ldg(f.H.slice_ptr + q);
    const int w = (int)((__ldg(f.H.slice_ptr + q + 1) - base) / kSliceRows);
    const int32_t *colp = f.H.col + base + lr;
    const V *valp = reinterpret_cast<const V *>(f.H.val) + base + lr;
    const Lane *xl = reinterpret_cast<const Lane *>(x);
    const bool x_ro = tm.x < 0;          // x is psi: never written in the launch
    const V d = __ldg(reinterpret_cast<const V *>(f.H.diag) + r);
    Cf<V, SPL> y;
    unpf(x_ro ? __ldg(xl + r * L + l) : __ldcg(xl + r * L + l), y);
    if constexpr (sizeof(V) == 8) {
        if (f.uniform) {
            // FP64 one-value form, as in the per-term kernels: neighbours
            // summed in stored order (padding -- the own row -- skipped),
            // then fma(gh, s, fma(gd, x_r, fma(c, psi, z)))
            Cf<V, SPL> sm;
#pragma unroll
            for (int j = 0; j < SPL; ++j) { sm.re[j] = 0; sm.im[j] = 0; }
            auto group = [&](int k, auto first) {
                int32_t c[4];
                bool ok[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ok[u] = k + u < w;
                    c[u] = ok[u] ? __ldg(colp + (int64_t)(k + u) * kSliceRows) : (int32_t)r;
                    ok[u] = ok[u] && c[u] != (int32_t)r;
                }
                Cf<V, SPL> xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    unpf(x_ro ? __ldg(xl + (int64_t)c[u] * L + l) : __ldcg(xl + (int64_t)c[u] * L + l),
                         xv[u]);
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
                for (int k = 4; k < w; k += 4) group(k, std::false_type{});
            }
            if (sc) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    const V sv = sc[l * SPL + j];
                    p.re[j] *= sv;
                    p.im[j] *= sv;
                    if (x_ro) {
                        sm.re[j] *= sv;
                        sm.im[j] *= sv;
                        y.re[j] *= sv;
                        y.im[j] *= sv;
                    }
                }
            }
            const V gd = f.zero_diag     ? 0.0
                         : tm.gd_sel == 2 ? xor_sign(__ldg(f.diag2 + r), tm.gd_sign)
                         : tm.gd_sel == 1 ? xor_sign(d, tm.gd_sign)
                                          : tm.gamma * d;
            Cf<V, SPL> o;
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                V re = fma(tm.c_hi, p.re[j], zz.re[j]);
                V im = fma(tm.c_hi, p.im[j], zz.im[j]);
                if (!f.zero_diag) {
                    re = fma(gd, y.im[j], re);            // y holds x_r here
                    im = fma(-gd, y.re[j], im);
                }
                o.re[j] = fma(tm.gh, sm.im[j], re);
                o.im[j] = fma(-tm.gh, sm.re[j], im);
            }
            return o;
        }
    }
#pragma unroll
    for (int j = 0; j < SPL; ++j) { y.re[j] *= d; y.im[j] *= d; }
    for (int k = 0; k < w; k += 4) {
        int32_t c[4];
        V h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = k + u < w;
            c[u] = ok ? __ldg(colp + (int64_t)(k + u) * kSliceRows) : (int32_t)r;
            h[u] = ok ? __ldg(valp + (int64_t)(k + u) * kSliceRows) : (V)0;
        }
        Cf<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            unpf(x_ro ? __ldg(xl + (int64_t)c[u] * L + l) : __ldcg(xl + (int64_t)c[u] * L + l),
                 xv[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k + u < w) {
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
            const V s = sc[l * SPL + j];
            p.re[j] *= s;
            p.im[j] *= s;
            if (x_ro) { y.re[j] *= s; y.im[j] *= s; }
        }
    }
    const V g = FCoef<V>::g(tm), ch = FCoef<V>::hi(tm), cl = FCoef<V>::lo(tm);
    Cf<V, SPL> o;
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
    return o;
}

template <typename V, int L, int SPL>
__global__ void __launch_bounds__(kFusedThreads) k_step_fused(FusedArgs f)
{
    typedef typename LaneF<V, SPL>::type Lane;
    constexpr int B = L * SPL;
    constexpr int ROWS_PER_PASS = kFusedThreads / L;
    constexpr int NW = kFusedThreads / 32;
    __shared__ int64_t s_item, s_next;
    __shared__ double red[NW][B * 3];
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int l = tid % L;
    const int R = f.tile_rows;
    const int passes = R / ROWS_PER_PASS;
    const int epoch = *f.epoch_ptr + 1;
    const int per_chunk = R < kChunkRows ? kChunkRows / R : 1;

    if (tid == 0) s_next = atomicAdd(f.counter, 1ull);
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            s_item = s_next;
            if (s_next < f.n_items) s_next = atomicAdd(f.counter, 1ull);   // prefetch the next
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= f.n_items) break;
        const uint32_t packed = (uint32_t)f.items[item];
        const int j = (int)(packed >> 25);
        const int64_t t = (int64_t)(packed & ((1u << 25) - 1u));
        // wait for (j-1, t') with |t' - t| <= radius
        if (j > 0 && warp == 0) {
            const int *flags = f.done + (int64_t)(j - 1) * f.n_tiles;
            for (int64_t tt = t - f.radius + lane; tt <= t + f.radius; tt += 32) {
                if (tt < 0 || tt >= f.n_tiles) continue;
                long long it = 0;
                while (ld_acquire(flags + tt) < epoch) {
                    // give up after kPollLimit polls, or at once when another
                    // block already gave up (the launch then only drains)
                    if (++it > kPollLimit || (ld_acquire(f.err) & 4)) {
                        atomicOr(f.err, 4);
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __syncthreads();
        const FusedTerm tm = f.terms[j];
        void *out = f.bufs[tm.out];
        const void *x = tm.x < 0 ? f.psi : f.bufs[tm.x];
        const void *z = tm.z < 0 ? nullptr : f.bufs[tm.z];
        FF fre[SPL], fim[SPL], fnr[SPL];
        double dre[SPL], dim[SPL], dnr[SPL];
        auto zero = [&]() {
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                fre[q] = fim[q] = fnr[q] = FF{0.f, 0.f};
                dre[q] = dim[q] = dnr[q] = 0.0;
            }
        };
        auto shfl_ff = [&](FF &v, int off) {
            FF w;
            w.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
            w.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
            v = ff_add(v, w);
        };
        // block sum of the per-thread partials (FP32 form: exact products
        // and float-pair sums within the warp, FP64 from the warp sums up)
        // into `dst` (B*3 doubles)
        auto block_sum = [&](double *dst) {
#pragma unroll
            for (int off = L; off < 32; off <<= 1) {
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    if (sizeof(V) == 4) {
                        shfl_ff(fre[q], off);
                        shfl_ff(fim[q], off);
                        shfl_ff(fnr[q], off);
                    } else {
                        dre[q] += __shfl_xor_sync(0xffffffffu, dre[q], off);
                        dim[q] += __shfl_xor_sync(0xffffffffu, dim[q], off);
                        dnr[q] += __shfl_xor_sync(0xffffffffu, dnr[q], off);
                    }
                }
            }
            if (lane < L) {
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    const int b = lane * SPL + q;
                    red[warp][b * 3 + 0] = sizeof(V) == 4 ? ff_to_double(fre[q]) : dre[q];
                    red[warp][b * 3 + 1] = sizeof(V) == 4 ? ff_to_double(fim[q]) : dim[q];
                    red[warp][b * 3 + 2] = sizeof(V) == 4 ? ff_to_double(fnr[q]) : dnr[q];
                }
            }
            __syncthreads();
            if (tid < B * 3) {
                double s2 = 0.0;
                for (int w2 = 0; w2 < NW; ++w2) s2 += red[w2][tid];
                dst[tid] = s2;
            }
            __syncthreads();
        };
        zero();
        const int passes_per_chunk = kChunkRows / ROWS_PER_PASS;
        for (int pass = 0; pass < passes; ++pass) {
            const int64_t r = t * R + pass * ROWS_PER_PASS + tid / L;
            const V *sc = FCoef<V>::scale(f);
            if (sc) sc += (int64_t)f.chunk_sample[r / kChunkRows] * B;
            const Cf<V, SPL> o = fused_row<V, L, SPL>(f, tm, x, z, r, l, sc);
            reinterpret_cast<Lane *>(out)[r * L + l] = pkf(o);
            if (tm.final_term) {
                Cf<V, SPL> p0;
                unpf(__ldg(reinterpret_cast<const Lane *>(f.psi0) + r * L + l), p0);
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    if constexpr (sizeof(V) == 4) {
                        FF pre, pim, pnr;
                        ff_dot3(p0.re[q], p0.im[q], o.re[q], o.im[q], pre, pim, pnr);
                        fre[q] = ff_add(fre[q], pre);
                        fim[q] = ff_add(fim[q], pim);
                        fnr[q] = ff_add(fnr[q], pnr);
                    } else {
                        dre[q] += fma(p0.re[q], o.re[q], p0.im[q] * o.im[q]);
                        dim[q] += fma(p0.re[q], o.im[q], -(p0.im[q] * o.re[q]));
                        dnr[q] += fma(o.re[q], o.re[q], o.im[q] * o.im[q]);
                    }
                }
                // a tile of at least one chunk: the chunk's partial is complete here
                if (R >= kChunkRows && (pass + 1) % passes_per_chunk == 0) {
                    const int64_t chunk = (t * R + (int64_t)pass * ROWS_PER_PASS) / kChunkRows;
                    block_sum(f.partial + chunk * (B * 3));
                    zero();
                }
            }
        }
        if (tm.final_term && R < kChunkRows) {
            // tiles smaller than a chunk: per-tile partial, the chunk's last tile adds them
            const int64_t chunk = t / per_chunk;
            block_sum(f.tile_partial + t * (B * 3));
            if (tid == 0) {
                __threadfence();
                last = (atomicAdd(f.chunk_count + chunk, 1) == per_chunk - 1);
            }
            __syncthreads();
            if (last) {
                __threadfence();
                if (tid < B * 3) {
                    double s2 = 0.0;
                    for (int k = 0; k < per_chunk; ++k)
                        s2 += __ldcg(f.tile_partial + (chunk * per_chunk + k) * (B * 3) + tid);
                    f.partial[chunk * (B * 3) + tid] = s2;
                }
                if (tid == 0) f.chunk_count[chunk] = 0;
            }
        }
        __syncthreads();      // all writes of this item are issued
        if (tid == 0) {
            __threadfence();
            st_release(f.done + (int64_t)j * f.n_tiles + t, epoch);
        }
    }
}

template <typename V, int L, int SPL>
cudaError_t launch_fused_t(const FusedArgs &f, int num_sms, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused<V, L, SPL>,
                                                                  kFusedThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > f.n_items) grid = f.n_items;
    void *args[] = {const_cast<FusedArgs *>(&f)};
    return cudaLaunchCooperativeKernel((const void *)k_step_fused<V, L, SPL>, dim3((unsigned)grid),
                                       dim3(kFusedThreads), args, 0, st);
}

}  // namespace

int fused_tile_rows(int fp32, int B, int log4_mult)
{
    // 256 rows per item (times 4^log4_mult, at most the 1024-row reduction
    // chunk times 16) keeps the wavefront band small; rows per pass is 512 / L,
    // so the tile must be a multiple of that
    const int L = fp32 ? (B >= 2 ? B / 2 : 1) : B;
    const int rpp = kFusedThreads / L;
    int rows = rpp > 256 ? rpp : 256;
    for (int k = 0; k < log4_mult; ++k) rows *= 4;
    return rows;
}

// Blocks of the cooperative grid (all resident).
int fused_grid(int fp32, int B, int num_sms)
{
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define TBPM_OCC(V, L, SPL) \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused<V, L, SPL>, kFusedThreads, 0)
    if (!fp32) {
        switch (B) {
        case 1: TBPM_OCC(double, 1, 1); break;
        case 2: TBPM_OCC(double, 2, 1); break;
        case 4: TBPM_OCC(double, 4, 1); break;
        case 8: TBPM_OCC(double, 8, 1); break;
        }
    } else {
        switch (B) {
        case 1: TBPM_OCC(float, 1, 1); break;
        case 2: TBPM_OCC(float, 1, 2); break;
        case 4: TBPM_OCC(float, 2, 2); break;
        case 8: TBPM_OCC(float, 4, 2); break;
        case 16: TBPM_OCC(float, 8, 2); break;
        }
    }
#undef TBPM_OCC
    if (e != cudaSuccess || per_sm < 1) return 0;
    return per_sm * num_sms;
}

cudaError_t launch_step_fused(const FusedArgs &f, int fp32, int B, int num_sms, cudaStream_t st)
{
    if (!fp32) {
        switch (B) {
        case 1: return launch_fused_t<double, 1, 1>(f, num_sms, st);
        case 2: return launch_fused_t<double, 2, 1>(f, num_sms, st);
        case 4: return launch_fused_t<double, 4, 1>(f, num_sms, st);
        case 8: return launch_fused_t<double, 8, 1>(f, num_sms, st);
        }
    } else {
        switch (B) {
        case 1: return launch_fused_t<float, 1, 1>(f, num_sms, st);
        case 2: return launch_fused_t<float, 1, 2>(f, num_sms, st);
        case 4: return launch_fused_t<float, 2, 2>(f, num_sms, st);
        case 8: return launch_fused_t<float, 4, 2>(f, num_sms, st);
        case 16: return launch_fused_t<float, 8, 2>(f, num_sms, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tbpm
