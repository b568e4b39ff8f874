// a8: adjoint of the Chebyshev propagation (FP64).
//
// For a real loss L of the correlations C_n = <psi0|phi_n> the caller gives
// gbar_n = dL/dRe C_n + i dL/dIm C_n per sample and state.  The adjoint of
// the trajectory obeys Lambda_N = gbar_N psi0 and
// Lambda_n = gbar_n psi0 + P^dagger Lambda_{n+1}, with P the one-step
// propagator of the Chebyshev sum (Sec. 2.2).  H~ is Hermitian, so
// P^dagger = sum_m a_m T^_m(H~)^dagger is the same series with +i in place
// of -i: the backward pass reuses the Clenshaw schedule of the forward one
// with gamma -> -gamma.  Its intermediate vectors are exactly the adjoints
// mu_m of the forward polynomials T^_m, so the kernel that forms mu_m from
// the gathered mu_{m+1} also accumulates, for every stored entry (r, c),
//   G_rc += g_{m+1} Im(conj(mu_{m+1, c}) T^_{m, r}),
// the contribution of the transposed element to dL/dH~ (g = 2, or 1 for the
// closing term).  A bond's gradient is the sum of its two stored entries;
// the diagonal entry gives dL/deps.  Entries of a row are owned by one
// thread, so the accumulation needs no atomics and is deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

__device__ __forceinline__ double2 ldg2(const void *p, int64_t i)
{
    return __ldg(reinterpret_cast<const double2 *>(p) + i);
}

// Sum over the L lanes that serve one row (xor offsets below L).
template <int L>
__device__ __forceinline__ double row_sum(double v)
{
#pragma unroll
    for (int off = 1; off < L; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int L>
__global__ void __launch_bounds__(1024) k_adj_term(AdjArgs a)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = t / L;
    const int l = (int)(t % L);
    // the grid covers exactly n_rows * L threads (n_rows is a multiple of
    // kChunkRows), so every warp is complete and shuffles below are safe
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    const int64_t base = __ldg(a.H.slice_ptr + q);
    const int w = (int)((__ldg(a.H.slice_ptr + q + 1) - base) / kSliceRows);  // warp-uniform
    const int32_t *colp = a.H.col + base + lr;
    const double *valp = reinterpret_cast<const double *>(a.H.val) + base + lr;
    const double2 T = ldg2(a.T_own, r * L + l);

    const double d = __ldg(reinterpret_cast<const double *>(a.H.diag) + r);
    const double2 xr = ldg2(a.x, r * L + l);
    double yr = d * xr.x, yi = d * xr.y;
    {
        const double gd = row_sum<L>(xr.x * T.y - xr.y * T.x);
        if (l == 0) a.Gdiag[r] += a.gfac * gd;
    }
    for (int k = 0; k < w; k += 4) {
        int32_t c[4];
        double h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = k + u < w;
            c[u] = ok ? __ldg(colp + (int64_t)(k + u) * kSliceRows) : (int32_t)r;
            h[u] = ok ? __ldg(valp + (int64_t)(k + u) * kSliceRows) : 0.0;
        }
        double2 xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ldg2(a.x, (int64_t)c[u] * L + l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            yr = fma(h[u], xv[u].x, yr);
            yi = fma(h[u], xv[u].y, yi);
            const double gi = row_sum<L>(xv[u].x * T.y - xv[u].y * T.x);
            if (l == 0 && k + u < w) a.G[base + (int64_t)(k + u) * kSliceRows + lr] += a.gfac * gi;
        }
    }
    const double2 p = ldg2(a.psi, r * L + l);
    double2 zz = make_double2(0.0, 0.0);
    if (a.z) zz = reinterpret_cast<const double2 *>(a.z)[r * L + l];
    double ore = fma(a.gamma, yi, zz.x);
    double oim = fma(-a.gamma, yr, zz.y);
    ore = fma(a.c, p.x, ore);
    oim = fma(a.c, p.y, oim);
    if (a.gbar) {   // + gbar_n psi0 (the adjoint source of step n)
        const int s = a.chunk_sample[r / kChunkRows];
        const double2 g = a.gbar[((int64_t)s * a.n_states + a.state0 + l) * (a.n_steps + 1) + a.step];
        const double2 p0 = ldg2(a.psi0, r * L + l);
        ore += g.x * p0.x - g.y * p0.y;
        oim += g.x * p0.y + g.y * p0.x;
    }
    reinterpret_cast<double2 *>(a.out)[r * L + l] = make_double2(ore, oim);
}

// out = gbar_N psi0 (the adjoint of the last state).
__global__ void k_source_init(int64_t n_rows, int B, const int32_t *chunk_sample,
                              const double2 *gbar, int n_states, int state0, int n_steps,
                              int step, const double2 *psi0, double2 *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rows * B) return;
    const int64_t r = i / B;
    const int b = (int)(i % B);
    const int s = chunk_sample[r / kChunkRows];
    const double2 g = gbar[((int64_t)s * n_states + state0 + b) * (n_steps + 1) + step];
    const double2 p = psi0[i];
    out[i] = make_double2(g.x * p.x - g.y * p.y, g.x * p.y + g.y * p.x);
}

__device__ __forceinline__ double find_entry(const int64_t *slice_ptr, const int32_t *col,
                                             const double *G, int32_t r, int32_t c)
{
    const int64_t q = r / kSliceRows;
    const int lr = r % kSliceRows;
    const int64_t base = slice_ptr[q];
    const int w = (int)((slice_ptr[q + 1] - base) / kSliceRows);
    for (int k = 0; k < w; ++k) {
        const int64_t e = base + (int64_t)k * kSliceRows + lr;
        if (col[e] == c) return G[e];
    }
    return __longlong_as_double(0x7ff8000000000000LL);   // not stored: NaN flags it
}

__global__ void k_bond_grad(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                            const int32_t *col, const double *G, double inv_s, double *grad)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_hop) return;
    const int32_t ri = bond_rows[2 * b], rj = bond_rows[2 * b + 1];
    grad[b] = (find_entry(slice_ptr, col, G, ri, rj) + find_entry(slice_ptr, col, G, rj, ri)) *
              inv_s;
}

__global__ void k_onsite_grad(int64_t n_orb, const int32_t *user_to_row, const double *Gd,
                              double inv_s, double *grad)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u < n_orb) grad[u] = Gd[user_to_row[u]] * inv_s;
}

}  // namespace

cudaError_t launch_adj_term(const AdjArgs &a, int B, int threads, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((a.n_rows * B + threads - 1) / threads);
    switch (B) {
    case 1: k_adj_term<1><<<blocks, threads, 0, st>>>(a); break;
    case 2: k_adj_term<2><<<blocks, threads, 0, st>>>(a); break;
    case 4: k_adj_term<4><<<blocks, threads, 0, st>>>(a); break;
    case 8: k_adj_term<8><<<blocks, threads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_source_init(int64_t n_rows, int B, const int32_t *chunk_sample,
                               const double2 *gbar, int n_states, int state0, int n_steps,
                               int step, const void *psi0, void *out, cudaStream_t st)
{
    const int64_t n = n_rows * B;
    k_source_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        n_rows, B, chunk_sample, gbar, n_states, state0, n_steps, step,
        reinterpret_cast<const double2 *>(psi0), reinterpret_cast<double2 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_param_grads(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                               const int32_t *col, const double *G, const double *Gd,
                               int64_t n_orb, const int32_t *user_to_row, double inv_s,
                               double *grad_hop, double *grad_onsite, cudaStream_t st)
{
    if (n_hop > 0)
        k_bond_grad<<<(unsigned)((n_hop + 255) / 256), 256, 0, st>>>(n_hop, bond_rows, slice_ptr,
                                                                     col, G, inv_s, grad_hop);
    k_onsite_grad<<<(unsigned)((n_orb + 255) / 256), 256, 0, st>>>(n_orb, user_to_row, Gd, inv_s,
                                                                   grad_onsite);
    return cudaGetLastError();
}

}  // namespace tbpm
