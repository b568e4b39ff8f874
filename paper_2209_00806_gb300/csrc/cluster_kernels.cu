// Cluster-resident time stepping for small samples (TBPM_VARIANT_CLUSTER).
//
// A sample of up to 16 x 1024 rows -- the 64 x 64 graphene DOS workload has
// 8192 -- fits, with psi0, psi and the two Clenshaw buffers, in the shared
// memory of one thread-block cluster.  All time steps of the propagation then
// run in one launch: each block holds a contiguous range of rows (one row per
// thread), gathers x from the owning block's shared memory (distributed
// shared memory across the cluster), and a cluster barrier separates the
// Clenshaw terms (Sec. 2.2, Eq. psi_t).  The closing term's sums of
// <psi0|phi> and <phi|phi> are formed per block in a fixed tree after the
// block has arrived at the term's barrier (no later term needs them), and
// added over the blocks in rank order by block 0 two barriers later (FP64,
// deterministic).  Per row
// the arithmetic and its order are those of the plain term kernel, so the
// states equal the per-term launches' bit for bit; the launch cost of
// 15 kernels per step is gone.  FP64 states, one state, real values, at most
// kClusterMaxW entries per row, within the shared memory of a block.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "tbpm_internal.cuh"

namespace cg = cooperative_groups;

namespace tbpm {
namespace {

// Address of `p` (this block's shared memory) in the shared::cluster
// window of block `rank`, and a 16-byte load through that window.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, int rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ double2 ld_cluster(uint32_t addr)
{
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr));
    return v;
}

constexpr uint32_t kNoEntry = 0xffffffffu;

// MAXW: the widest row the launch allows (its gather addresses stay in
// registers: 4 for graphene-like lattices, kClusterMaxW otherwise).
template <int MAXW, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_cluster_steps(ClusterArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int K = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int R = a.rows_per_cta;
    const int t = threadIdx.x;
    const int64_t r = (int64_t)rank * R + t;
    extern __shared__ __align__(16) unsigned char sm[];
    double2 *vec = reinterpret_cast<double2 *>(sm);                  // [4][R]
    int32_t *ent = reinterpret_cast<int32_t *>(vec + 4 * R);         // [W][R] owner << 16 | local
    double *sval = reinterpret_cast<double *>(ent + a.max_w * R);    // [W][R] (general values)
    __shared__ double part[2][3];
    __shared__ double red[32][3];
    __shared__ FusedTerm tab[3 * kClusterMaxTerms];

    for (int i = t; i < 3 * a.J; i += blockDim.x)
        tab[i] = a.terms[(i / a.J) * kMaxTerms + i % a.J];
    // this row's entries, as (owning block, local row) pairs
    int w;
    int64_t base;
    if (a.fixed_width) {
        w = a.fixed_width;
        base = (r / kSliceRows) * (kSliceRows * (int64_t)w) + r % kSliceRows;
    } else {
        const int64_t q = r / kSliceRows;
        base = a.slice_ptr[q] + r % kSliceRows;
        w = (int)((a.slice_ptr[q + 1] - a.slice_ptr[q]) / kSliceRows);
    }
    for (int k = 0; k < w; ++k) {
        const int32_t c = a.col[base + (int64_t)k * kSliceRows];
        ent[k * R + t] = c == (int32_t)r && a.uniform ? -1 : ((c / R) << 16) | (c % R);
        if (!a.uniform) sval[k * R + t] = a.val[base + (int64_t)k * kSliceRows];
    }
    const double d = a.diag[r];
    const double d2 = d + d;                 // 2 d, exact: gamma d of the interior terms
    vec[t] = a.psi0[r];
    for (int b = 0; b < 3; ++b)
        vec[(1 + b) * R + t] = b == a.cur0 ? a.bufs[b][r] : make_double2(0.0, 0.0);
    cl.sync();
    // gathered entries' shared::cluster addresses in x buffer 0 (a buffer
    // is R rows further on), fixed for the launch; kNoEntry for padding
    // (one-value form)
    uint32_t gsrc[MAXW];
#pragma unroll
    for (int k = 0; k < MAXW; ++k) {
        gsrc[k] = kNoEntry;
        if (k < w) {
            const int32_t e = ent[k * R + t];
            if (e >= 0) gsrc[k] = cluster_addr(vec + (e & 0xffff), e >> 16);
        }
    }

    int cur = a.cur0;
    bool pending = false;                    // a cluster barrier arrived at, not yet waited on
    // a step whose block parts await block 0's sum, and the barrier waits
    // until they are all written: the closing term's own barrier completes
    // before the blocks write their parts, the next one after
    int sum_step = 0, sum_waits = 0;
    // block 0, warp 0: lane k loads block k's parts of step m, the lanes'
    // values are added in rank order; C_m, the norm and the drift checks
    auto cluster_sum = [&](int m) {
        double w0 = 0.0, w1 = 0.0, w2 = 0.0;
        if (t < K) {
            const double *pk = cl.map_shared_rank(&part[m & 1][0], t);
            w0 = pk[0];
            w1 = pk[1];
            w2 = pk[2];
        }
        double sm0 = 0.0, sm1 = 0.0, sm2 = 0.0;
        for (int k = 0; k < K; ++k) {
            sm0 += __shfl_sync(0xffffffffu, w0, k);
            sm1 += __shfl_sync(0xffffffffu, w1, k);
            sm2 += __shfl_sync(0xffffffffu, w2, k);
        }
        if (t == 0) {
            a.corr[m] = make_double2(sm0, sm1);
            a.norms[m] = sm2;
            const double ref = *a.norm_ref;
            const double drift = ref > 0.0 ? fabs(sm2 / ref - 1.0) : sm2;
            if (!(sm2 == sm2) || !(sm0 == sm0) || !(sm1 == sm1) || sm2 - sm2 != 0.0)
                atomicOr(a.err, 2);
            else if (drift > a.hard_bound)
                atomicOr(a.err, 1);
        }
    };
    for (int n = 1; n <= a.n_steps; ++n) {
        const FusedTerm *tt = tab + cur * a.J;
        for (int j = 0; j < a.J; ++j) {
            const FusedTerm tm = tt[j];
            const int xb = 1 + (tm.x < 0 ? cur : tm.x);
            // own-row operands (written only by this thread) before the wait
            const double2 p = vec[(1 + cur) * R + t];
            double2 zz = make_double2(0.0, 0.0);
            if (tm.z >= 0) zz = vec[(1 + tm.z) * R + t];
            const int xoff = xb * R;
            const uint32_t xoff_b = (uint32_t)xoff * (uint32_t)sizeof(double2);
            double2 o;
            // one-value form: its first product, fma(c, psi, z), needs nothing
            // of this term's x, so it runs before the barrier wait
            double re = 0.0, im = 0.0;
            if (a.uniform) {
                re = fma(tm.c_hi, p.x, zz.x);
                im = fma(tm.c_hi, p.y, zz.y);
            }
            if (pending) cl.barrier_wait();      // the gathered vector is complete
            pending = false;
            if (sum_waits > 0 && --sum_waits == 0 && rank == 0 && t < 32) cluster_sum(sum_step);
            if (a.uniform) {
                // the one-value form of the per-term kernels: neighbours summed
                // in stored order (padding only after a row's entries), then
                // fma(gh, s, fma(gd, x_r, fma(c, psi, z)))
                double2 sm = make_double2(0.0, 0.0);
                if (gsrc[0] != kNoEntry) sm = ld_cluster(gsrc[0] + xoff_b);
#pragma unroll
                for (int k = 1; k < MAXW; ++k) {
                    if (k < w && gsrc[k] != kNoEntry) {
                        const double2 x = ld_cluster(gsrc[k] + xoff_b);
                        sm.x += x.x;
                        sm.y += x.y;
                    }
                }
                if (!a.zero_diag) {
                    const double gd = tm.gd_sel == 2 ? xor_sign(d2, tm.gd_sign)
                                    : tm.gd_sel == 1 ? xor_sign(d, tm.gd_sign)
                                                     : tm.gamma * d;
                    const double2 xo = vec[xoff + t];
                    re = fma(gd, xo.y, re);
                    im = fma(-gd, xo.x, im);
                }
                o.x = fma(tm.gh, sm.y, re);
                o.y = fma(-tm.gh, sm.x, im);
            } else {
                // y = H~ x in the plain kernel's order: diagonal, then the entries
                // (a zero diagonal contributes only signed zeros: skipped, the
                // sums stay equal to the plain kernel's)
                double2 y = make_double2(0.0, 0.0);
                if (!a.zero_diag) {
                    y = vec[xoff + t];
                    y.x *= d;
                    y.y *= d;
                }
#pragma unroll
                for (int k = 0; k < MAXW; ++k) {
                    if (k < w) {
                        const double h = sval[k * R + t];
                        const double2 x = ld_cluster(gsrc[k] + xoff_b);
                        y.x = fma(h, x.x, y.x);
                        y.y = fma(h, x.y, y.y);
                    }
                }
                re = fma(tm.gamma, y.y, zz.x);
                im = fma(-tm.gamma, y.x, zz.y);
                o.x = fma(tm.c_hi, p.x, re);
                o.y = fma(tm.c_hi, p.y, im);
            }
            vec[(1 + tm.out) * R + t] = o;
            cl.barrier_arrive();                 // release this term's writes
            pending = true;
            if (tm.final_term) {
                // the step's sums, off the critical path: nothing of the next
                // terms needs them, so they are formed while the other blocks
                // reach the barrier; block 0 adds the blocks' parts two
                // barriers on (part is double-buffered by step parity)
                const double2 p0 = vec[t];
                double v0 = fma(p0.x, o.x, p0.y * o.y);
                double v1 = fma(p0.x, o.y, -(p0.y * o.x));
                double v2 = fma(o.x, o.x, o.y * o.y);
                for (int off = 16; off > 0; off >>= 1) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, off);
                }
                if (t % 32 == 0) {
                    red[t / 32][0] = v0;
                    red[t / 32][1] = v1;
                    red[t / 32][2] = v2;
                }
                __syncthreads();
                if (t < 32) {               // warp q's sums in order, loaded at once
                    const int nq = (R + 31) / 32;
                    double w0 = 0.0, w1 = 0.0, w2 = 0.0;
                    if (t < nq) {
                        w0 = red[t][0];
                        w1 = red[t][1];
                        w2 = red[t][2];
                    }
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                    for (int q = 0; q < nq; ++q) {
                        s0 += __shfl_sync(0xffffffffu, w0, q);
                        s1 += __shfl_sync(0xffffffffu, w1, q);
                        s2 += __shfl_sync(0xffffffffu, w2, q);
                    }
                    if (t == 0) {
                        part[n & 1][0] = s0;
                        part[n & 1][1] = s1;
                        part[n & 1][2] = s2;
                    }
                }
                sum_step = n;
                sum_waits = 2;
            }
        }
        cur = a.next_cur[cur];
    }
    // the last step's parts: its closing barrier, one more, then block 0 adds them
    if (pending) {
        cl.barrier_wait();
        if (sum_waits > 0) --sum_waits;
    }
    pending = false;
    if (sum_waits > 0) {
        cl.sync();
        if (rank == 0 && t < 32) cluster_sum(sum_step);
    }
    a.bufs[cur][r] = vec[(1 + cur) * R + t];
    cl.sync();                                           // no block leaves while others read it
}

}  // namespace

int cluster_blocks_for(int64_t n_rows, int max_w, int uniform)
{
    if (n_rows <= 0 || n_rows > 16 * 1024 || max_w > kClusterMaxW) return 0;
    // 16 blocks (non-portable size) where the device runs such a cluster:
    // GB300's FP64 rate per SM makes more SMs pay; else 8
    static int best16 = -1;
    if (best16 < 0) {
        best16 = 0;
        if (cudaFuncSetAttribute(k_cluster_steps<kClusterMaxW, 1024>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = 16;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(512);
            cfg.dynamicSmemBytes = 64 * 1024;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            int n = 0;
            cudaFuncSetAttribute(k_cluster_steps<kClusterMaxW, 1024>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            if (cudaOccupancyMaxActiveClusters(&n, k_cluster_steps<kClusterMaxW, 1024>, &cfg) ==
                    cudaSuccess &&
                n >= 1)
                best16 = 1;
        }
        cudaGetLastError();
    }
    auto fits = [&](int K) {
        if (n_rows % K || n_rows / K > 1024) return false;
        const int64_t R = n_rows / K;
        const int64_t smem = 4 * R * 16 + (int64_t)std::max(1, max_w) * R * (uniform ? 4 : 12);
        return smem <= 200 * 1024;
    };
    if (best16 && fits(16)) return 16;
    return fits(8) ? 8 : 0;
}

template <int MAXW, int MAXT>
cudaError_t launch_cluster_t(const ClusterArgs &a, int K, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(k_cluster_steps<MAXW, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (K > 8) {
        e = cudaFuncSetAttribute(k_cluster_steps<MAXW, MAXT>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = K;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(a.rows_per_cta);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cluster_steps<MAXW, MAXT>, a);
}

cudaError_t launch_cluster_steps(const ClusterArgs &a, int K, cudaStream_t st)
{
    const int R = a.rows_per_cta;
    const size_t smem = (size_t)4 * R * sizeof(double2) + (size_t)a.max_w * R * sizeof(int32_t) +
                        (a.uniform ? 0 : (size_t)a.max_w * R * sizeof(double));
    // up to 512 rows per block: 128 registers a thread, else 64
    if (R <= 512)
        return a.max_w <= 4 ? launch_cluster_t<4, 512>(a, K, smem, st)
                            : launch_cluster_t<kClusterMaxW, 512>(a, K, smem, st);
    return a.max_w <= 4 ? launch_cluster_t<4, 1024>(a, K, smem, st)
                        : launch_cluster_t<kClusterMaxW, 1024>(a, K, smem, st);
}

}  // namespace tbpm
