// AC-conductivity path (Sec. 2.7 with the Fermi-Dirac operator of Sec. 2.2).
//
// Preparation (once per random state, FP64, four lanes per row):
//   lanes 0, 1 <- psi;  lanes 2, 3 <- J_x psi, J_y psi with
//   (J_a v)_r = -i s sum_c H~_rc d^a_rc v_c   (the hopping current with e / hbar
//   factored out, units eV nm; d_rc = r_c - r_r is the bond vector of the
//   stored entry, so periodic bonds carry their own image); then the Fermi
//   operator by Clenshaw's
//   recurrence on lanes 1 .. 3, b_k = c_k v + 2 H~ b_{k+1} - b_{k+2},
//   f v = c_0 v / 2 + H~ b_1 - b_2.
// Observer (after every time step, in the group's precision): per row and
// lane quad, g_a = sum_c H~_rc d^a_rc psi_2,c and the four products
// conj(g_a) psi_1b,r, reduced deterministically per sample.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// h x for a stored value h: a full complex product for complex values, two
// products for real ones (half the FP64 work of the preparation).
template <bool CX> __device__ __forceinline__ double2 hmul(double2 h, double2 x)
{
    if (CX) return cmul(h, x);
    return make_double2(h.x * x.x, h.x * x.y);
}

// One stored value as complex double.
template <typename VT, bool CX> struct HVal;
template <> struct HVal<double, false> {
    __device__ static double2 get(const void *v, int64_t e)
    {
        return make_double2(__ldg(reinterpret_cast<const double *>(v) + e), 0.0);
    }
};
template <> struct HVal<float, false> {
    __device__ static double2 get(const void *v, int64_t e)
    {
        return make_double2((double)__ldg(reinterpret_cast<const float *>(v) + e), 0.0);
    }
};
template <> struct HVal<double, true> {
    __device__ static double2 get(const void *v, int64_t e)
    {
        return __ldg(reinterpret_cast<const double2 *>(v) + e);
    }
};
template <> struct HVal<float, true> {
    __device__ static double2 get(const void *v, int64_t e)
    {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(v) + e);
        return make_double2((double)f.x, (double)f.y);
    }
};

template <typename VT> __device__ __forceinline__ double diag_of(const void *d, int64_t r)
{
    return (double)__ldg(reinterpret_cast<const VT *>(d) + r);
}

// State element (row r, lane l) of a [row][B] buffer as complex double.
template <typename V> struct StateLd;
template <> struct StateLd<double> {
    __device__ static double2 get(const void *p, int64_t i)
    {
        return __ldg(reinterpret_cast<const double2 *>(p) + i);
    }
};
template <> struct StateLd<float> {
    __device__ static double2 get(const void *p, int64_t i)
    {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(p) + i);
        return make_double2((double)f.x, (double)f.y);
    }
};

// ---- preparation ------------------------------------------------------------

__global__ void k_ac_load(const double2 *psi_user, int p, int64_t n_orb,
                          const int32_t *user_to_row, double2 *v4)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_orb) return;
    const int64_t r = user_to_row[i];
    const double2 v = psi_user[(int64_t)p * n_orb + i];
    v4[r * 4 + 0] = v;
    v4[r * 4 + 1] = v;
}

template <typename VT, bool CX>
__global__ void k_current4(SellView H, int64_t n_rows, const double *dxe, const double *dye,
                           double s, double2 *v4)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t q = r / kSliceRows, lr = r % kSliceRows;
    const int64_t base = H.slice_ptr[q];
    const int w = (int)((H.slice_ptr[q + 1] - base) / kSliceRows);
    double2 gx = make_double2(0.0, 0.0), gy = make_double2(0.0, 0.0);
    for (int k = 0; k < w; ++k) {
        const int64_t e = base + (int64_t)k * kSliceRows + lr;
        const int32_t c = __ldg(H.col + e);
        const double2 hv = hmul<CX>(HVal<VT, CX>::get(H.val, e), v4[(int64_t)c * 4]);
        const double dx = __ldg(dxe + e), dy = __ldg(dye + e);
        gx.x = fma(dx, hv.x, gx.x);
        gx.y = fma(dx, hv.y, gx.y);
        gy.x = fma(dy, hv.x, gy.x);
        gy.y = fma(dy, hv.y, gy.y);
    }
    // -i s g = s (g.y, -g.x)
    v4[r * 4 + 2] = make_double2(s * gx.y, -s * gx.x);
    v4[r * 4 + 3] = make_double2(s * gy.y, -s * gy.x);
}

// out = c v + gamma (H~ x) + zeta z, one thread per (row, lane) for lanes
// 1 .. 3 (lane 0 holds psi itself, which needs no Fermi operator); x ==
// nullptr drops the product, z == nullptr the last term; out may alias z.
template <typename VT, bool CX>
__global__ void k_cheb_real4(SellView H, int64_t n_rows, double c, double gamma, double zeta,
                             const double2 *v, const double2 *x, const double2 *z, double2 *out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_rows * 3) return;
    const int64_t r = t / 3;
    const int l = 1 + (int)(t % 3);
    double2 y = make_double2(0.0, 0.0);
    if (x) {
        const double d = diag_of<VT>(H.diag, r);
        const double2 xo = x[r * 4 + l];
        y.x = d * xo.x;
        y.y = d * xo.y;
        const int64_t q = r / kSliceRows, lr = r % kSliceRows;
        const int64_t base = H.slice_ptr[q];
        const int w = (int)((H.slice_ptr[q + 1] - base) / kSliceRows);
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + (int64_t)k * kSliceRows + lr;
            const int32_t cc = __ldg(H.col + e);
            const double2 hv = hmul<CX>(HVal<VT, CX>::get(H.val, e), x[(int64_t)cc * 4 + l]);
            y.x += hv.x;
            y.y += hv.y;
        }
    }
    const double2 vv = v[r * 4 + l];
    double2 o;
    o.x = fma(c, vv.x, gamma * y.x);
    o.y = fma(c, vv.y, gamma * y.y);
    if (z) {
        const double2 zz = z[r * 4 + l];
        o.x = fma(zeta, zz.x, o.x);
        o.y = fma(zeta, zz.y, o.y);
    }
    out[r * 4 + l] = o;
}

__global__ void k_ac_store(const double2 *v4, const double2 *f4, int p, int64_t n_orb,
                           const int32_t *user_to_row, double2 *out_user)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_orb) return;
    const int64_t r = user_to_row[i];
    double2 *o = out_user + (int64_t)(4 * p) * n_orb + i;
    o[0] = v4[r * 4 + 0];                       // psi
    o[n_orb] = f4[r * 4 + 1];                   // f psi
    const double2 jx = v4[r * 4 + 2], fx = f4[r * 4 + 2];
    const double2 jy = v4[r * 4 + 3], fy = f4[r * 4 + 3];
    o[2 * n_orb] = make_double2(jx.x - fx.x, jx.y - fx.y);   // (1 - f) J_x psi
    o[3 * n_orb] = make_double2(jy.x - fy.x, jy.y - fy.y);   // (1 - f) J_y psi
}

// Bond vectors onto the stored entries: bond b = (i, j) with d_b = r_j - r_i
// gives d_b to entry (row i, col j) and -d_b to entry (row j, col i).  A pair
// listed twice has two entries with the same column; each bond claims the
// first unclaimed one (claim[] starts at zero).
__device__ void put_bond_vector(const int64_t *slice_ptr, const int32_t *col, int32_t r,
                                int32_t c, double dx, double dy, int *claim, double *dxe,
                                double *dye, int *err)
{
    const int64_t q = r / kSliceRows, lr = r % kSliceRows;
    const int64_t base = slice_ptr[q];
    const int w = (int)((slice_ptr[q + 1] - base) / kSliceRows);
    for (int k = 0; k < w; ++k) {
        const int64_t e = base + (int64_t)k * kSliceRows + lr;
        if (col[e] == c && atomicCAS(claim + e, 0, 1) == 0) {
            dxe[e] = dx;
            dye[e] = dy;
            return;
        }
    }
    atomicOr(err, 1);               // no entry left: the bond list changed
}

__global__ void k_bond_vectors(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                               const int32_t *col, const double *dx, const double *dy, int *claim,
                               double *dxe, double *dye, int *err)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_hop) return;
    const int32_t ri = bond_rows[2 * b], rj = bond_rows[2 * b + 1];
    const double x = dx[b], y = dy[b];
    if (!(x - x == 0.0) || !(y - y == 0.0)) { atomicOr(err, 2); return; }
    put_bond_vector(slice_ptr, col, ri, rj, x, y, claim, dxe, dye, err);
    put_bond_vector(slice_ptr, col, rj, ri, -x, -y, claim, dxe, dye, err);
}

// ---- observer ------------------------------------------------------------------

// Complex value in the observer's arithmetic type A (the group's precision).
template <typename A> struct C2 { A x, y; };

template <typename A, bool CX> __device__ __forceinline__ C2<A> obs_h(const void *v, int64_t e)
{
    C2<A> h;
    if (CX) {
        if (sizeof(A) == 4) {
            const float2 f = __ldg(reinterpret_cast<const float2 *>(v) + e);
            h.x = (A)f.x; h.y = (A)f.y;
        } else {
            const double2 d = __ldg(reinterpret_cast<const double2 *>(v) + e);
            h.x = (A)d.x; h.y = (A)d.y;
        }
    } else {
        h.x = __ldg(reinterpret_cast<const A *>(v) + e);
        h.y = (A)0;
    }
    return h;
}
template <typename A> __device__ __forceinline__ C2<A> obs_state(const void *p, int64_t i)
{
    C2<A> c;
    if (sizeof(A) == 4) {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(p) + i);
        c.x = (A)f.x; c.y = (A)f.y;
    } else {
        const double2 d = __ldg(reinterpret_cast<const double2 *>(p) + i);
        c.x = (A)d.x; c.y = (A)d.y;
    }
    return c;
}

// Arithmetic in the group's precision A: in the FP32 form the per-row sums,
// the products and the block's sum over its 128 rows are FP32 (their
// rounding is that of the FP32 states), with one conversion to FP64 per value
// and block -- GB300 issues FP64 instructions, conversions included, at a
// small fraction of the FP32 rate; the FP64 form is FP64 throughout.  Block
// partials and everything above them are FP64.
template <typename A, bool CX>
__global__ void __launch_bounds__(kAcRows) k_ac_observe(AcArgs a)
{
    const int64_t r = blockIdx.x * (int64_t)kAcRows + threadIdx.x;   // n_rows % 1024 == 0
    const int quad = blockIdx.y;
    const int B = a.B;
    const int l2 = 4 * quad + 1;
    const int64_t q = r / kSliceRows, lr = r % kSliceRows;
    const int64_t base = a.H.slice_ptr[q];
    const int w = (int)((a.H.slice_ptr[q + 1] - base) / kSliceRows);
    const A *dxp = reinterpret_cast<const A *>(sizeof(A) == 4 ? (const void *)a.dx32 : (const void *)a.dx);
    const A *dyp = reinterpret_cast<const A *>(sizeof(A) == 4 ? (const void *)a.dy32 : (const void *)a.dy);
    C2<A> gx = {(A)0, (A)0}, gy = {(A)0, (A)0};
    for (int k = 0; k < w; ++k) {
        const int64_t e = base + (int64_t)k * kSliceRows + lr;
        const int32_t c = __ldg(a.H.col + e);
        const C2<A> h = obs_h<A, CX>(a.H.val, e);
        const C2<A> x = obs_state<A>(a.psi, (int64_t)c * B + l2);
        C2<A> hv;
        hv.x = h.x * x.x;
        hv.y = h.x * x.y;
        if (CX) {
            hv.x = fma(-h.y, x.y, hv.x);
            hv.y = fma(h.y, x.x, hv.y);
        }
        const A dx = __ldg(dxp + e), dy = __ldg(dyp + e);
        gx.x = fma(dx, hv.x, gx.x);
        gx.y = fma(dx, hv.y, gx.y);
        gy.x = fma(dy, hv.x, gy.x);
        gy.y = fma(dy, hv.y, gy.y);
    }
    C2<A> u1x = obs_state<A>(a.psi, r * B + l2 + 1);
    C2<A> u1y = obs_state<A>(a.psi, r * B + l2 + 2);
    if (a.scale) {      // FP32 norm carry of the three lanes
        const int smp = a.chunk_sample[r / kChunkRows];
        const float *sf = a.scale_f + (int64_t)smp * B;
        const A s2 = (A)sf[l2], sx = (A)sf[l2 + 1], sy = (A)sf[l2 + 2];
        gx.x *= s2; gx.y *= s2; gy.x *= s2; gy.y *= s2;
        u1x.x *= sx; u1x.y *= sx; u1y.x *= sy; u1y.y *= sy;
    }
    // conj(g_a) u_b for ab = xx, xy, yx, yy
    const C2<A> ga[2] = {gx, gy}, ub[2] = {u1x, u1y};
    if constexpr (sizeof(A) == 4) {
        // FP32 form: exact float-pair products, the block's rows summed as
        // float pairs in fixed parts (FP64-grade), one conversion per value
        __shared__ FF redf[kAcRows][8];
        __shared__ FF redp[kAcRows];
#pragma unroll
        for (int ia = 0; ia < 2; ++ia)
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                FF re, im, nr;
                ff_dot3(ga[ia].x, ga[ia].y, ub[ib].x, ub[ib].y, re, im, nr);
                redf[threadIdx.x][(2 * ia + ib) * 2 + 0] = re;
                redf[threadIdx.x][(2 * ia + ib) * 2 + 1] = im;
            }
        __syncthreads();
        constexpr int P = kAcRows / 8;                  // parts per value
        {
            const int v = threadIdx.x % 8, part = threadIdx.x / 8;
            FF acc = redf[part][v];
            for (int row = part + P; row < kAcRows; row += P) acc = ff_add(acc, redf[row][v]);
            redp[threadIdx.x] = acc;
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            FF acc = redp[threadIdx.x];
            for (int part = 1; part < P; ++part) acc = ff_add(acc, redp[part * 8 + threadIdx.x]);
            a.block_partial[((int64_t)blockIdx.x * (B / 4) + quad) * 8 + threadIdx.x] =
                ff_to_double(acc);
        }
        return;
    }
    A v[8];
#pragma unroll
    for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) {
            v[(2 * ia + ib) * 2 + 0] = fma(ga[ia].x, ub[ib].x, ga[ia].y * ub[ib].y);
            v[(2 * ia + ib) * 2 + 1] = fma(ga[ia].x, ub[ib].y, -(ga[ia].y * ub[ib].x));
        }
    // block sum: warp butterflies, then the four warps in order
    __shared__ A red[kAcRows / 32][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        A x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[j] = x;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) red[warp][j] = v[j];
    __syncthreads();
    if (threadIdx.x < 8) {
        A acc = (A)0;
#pragma unroll
        for (int wp = 0; wp < kAcRows / 32; ++wp) acc += red[wp][threadIdx.x];
        a.block_partial[((int64_t)blockIdx.x * (B / 4) + quad) * 8 + threadIdx.x] = (double)acc;
    }
}

// FP32 copy of the per-entry bond vectors (for the FP32 observer).
__global__ void k_vec_to_f32(int64_t n, const double *src, float *dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

// One CTA of 512 threads per (sample, quad): thread (j, k) sums value k of
// blocks j, j + 64, ... of the sample; then 8 threads add the 64 partials in
// order.  Writes i s (sum) at the step index of the sample.
constexpr int kAcSplit = 64;

__global__ void __launch_bounds__(kAcSplit * 8) k_ac_reduce(AcReduceArgs a)
{
    const int smp = blockIdx.x, quad = blockIdx.y;
    const int k = threadIdx.x & 7, j = threadIdx.x >> 3;
    const int per_chunk = kChunkRows / kAcRows;
    const int64_t b0 = a.sample_chunk_off[smp] * per_chunk;
    const int64_t b1 = a.sample_chunk_off[smp + 1] * per_chunk;
    const int nq = a.B / 4;
    double acc = 0.0;
    for (int64_t b = b0 + j; b < b1; b += kAcSplit) acc += a.block_partial[(b * nq + quad) * 8 + k];
    __shared__ double part[kAcSplit][8];
    part[j][k] = acc;
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int jj = 0; jj < kAcSplit; ++jj) t += part[jj][threadIdx.x];
        part[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int ab = threadIdx.x;
        const double re = part[0][2 * ab], im = part[0][2 * ab + 1];
        const int step = a.step[smp] - 1;
        const int p = a.group_state0 / 4 + quad;
        const int64_t idx = (((int64_t)smp * (a.n_states / 4) + p) * 4 + ab) * (a.n_steps + 1) + step;
        a.corr_ac[idx] = make_double2(-a.s * im, a.s * re);   // i s (re + i im)
    }
}

}  // namespace

cudaError_t launch_ac_load(const double2 *psi_user, int p, int64_t n_orb,
                           const int32_t *user_to_row, double2 *v4, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_orb + 255) / 256);
    k_ac_load<<<blocks, 256, 0, st>>>(psi_user, p, n_orb, user_to_row, v4);
    return cudaGetLastError();
}

cudaError_t launch_current4(SellView H, int fp32_vals, int cplx, int64_t n_rows,
                            const double *dxe, const double *dye, double s, double2 *v4,
                            cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_rows + 127) / 128);
    if (fp32_vals) {
        if (cplx) k_current4<float, true><<<blocks, 128, 0, st>>>(H, n_rows, dxe, dye, s, v4);
        else k_current4<float, false><<<blocks, 128, 0, st>>>(H, n_rows, dxe, dye, s, v4);
    } else {
        if (cplx) k_current4<double, true><<<blocks, 128, 0, st>>>(H, n_rows, dxe, dye, s, v4);
        else k_current4<double, false><<<blocks, 128, 0, st>>>(H, n_rows, dxe, dye, s, v4);
    }
    return cudaGetLastError();
}

cudaError_t launch_cheb_real4(SellView H, int fp32_vals, int cplx, int64_t n_rows, double c,
                              double gamma, double zeta, const double2 *v, const double2 *x,
                              const double2 *z, double2 *out, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_rows * 3 + 255) / 256);
    if (fp32_vals) {
        if (cplx) k_cheb_real4<float, true><<<blocks, 256, 0, st>>>(H, n_rows, c, gamma, zeta, v, x, z, out);
        else k_cheb_real4<float, false><<<blocks, 256, 0, st>>>(H, n_rows, c, gamma, zeta, v, x, z, out);
    } else {
        if (cplx) k_cheb_real4<double, true><<<blocks, 256, 0, st>>>(H, n_rows, c, gamma, zeta, v, x, z, out);
        else k_cheb_real4<double, false><<<blocks, 256, 0, st>>>(H, n_rows, c, gamma, zeta, v, x, z, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_ac_store(const double2 *v4, const double2 *f4, int p, int64_t n_orb,
                            const int32_t *user_to_row, double2 *out_user, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_orb + 255) / 256);
    k_ac_store<<<blocks, 256, 0, st>>>(v4, f4, p, n_orb, user_to_row, out_user);
    return cudaGetLastError();
}

cudaError_t launch_bond_vectors(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                                const int32_t *col, const double *dx, const double *dy,
                                int *claim, double *dxe, double *dye, int *err, cudaStream_t st)
{
    if (n_hop == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_hop + 255) / 256);
    k_bond_vectors<<<blocks, 256, 0, st>>>(n_hop, bond_rows, slice_ptr, col, dx, dy, claim, dxe,
                                           dye, err);
    return cudaGetLastError();
}

cudaError_t launch_ac_observe(const AcArgs &a, int fp32, int cplx, cudaStream_t st)
{
    const dim3 grid((unsigned)(a.n_rows / kAcRows), (unsigned)(a.B / 4));
    if (fp32) {
        if (cplx) k_ac_observe<float, true><<<grid, kAcRows, 0, st>>>(a);
        else k_ac_observe<float, false><<<grid, kAcRows, 0, st>>>(a);
    } else {
        if (cplx) k_ac_observe<double, true><<<grid, kAcRows, 0, st>>>(a);
        else k_ac_observe<double, false><<<grid, kAcRows, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_vec_to_f32(int64_t n, const double *src, float *dst, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_vec_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_ac_reduce(const AcReduceArgs &a, cudaStream_t st)
{
    k_ac_reduce<<<dim3((unsigned)a.n_samples, (unsigned)(a.B / 4)), kAcSplit * 8, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tbpm
