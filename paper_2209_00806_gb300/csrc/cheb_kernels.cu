// a3-a5: the fused Chebyshev term kernels and the correlation reduction.
//
// One time step evaluates psi(t + tau) = sum_{m<M} a_m T^_m(H~) psi(t)
// (Sec. 2.2, Eq. psi_t: a_0 = J_0(z), a_m = 2 J_m(z), modified polynomials
// T^_{m+1} = -2i H~ T^_m + T^_{m-1}).  The paper sums forward; this library
// evaluates the same sum by Clenshaw's backward recurrence,
//   b_m = a_m psi + (-2i H~) b_{m+1} + b_{m+2},   b_M = b_{M+1} = 0,
//   psi(t + tau) = a_0 psi + (-i H~) b_1 + b_2,
// which needs one sparse product per term like the forward sum but moves
// four vectors per term instead of five (no accumulator read-modify-write).
// Every term is one kernel:
//   out = c psi + gamma (-i) (H~ x) + z
// with x gathered through the sparse rows, psi, z and out at the thread's
// own row.  The closing term (gamma = 1) also reduces <psi0|out> and
// <out|out> in FP64 per state.
//
// Vectors hold B states per orbital, interleaved: element (row r, state b)
// is complex number r * B + b.  A row is served by L lanes; each lane moves
// 16 bytes (one complex128, or two complex64) so a warp reads 512
// contiguous bytes of the own-row vectors, and every gathered row is one or
// more full 32-byte sectors.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

// A lane moves 16 bytes (one complex128, or two complex64) in the default
// layout, or 32 bytes (two of those) in the wide-lane variant.
struct W32F { float4 a, b; };
struct W32D { double2 a, b; };

template <typename V, int SPL> struct LaneT;
template <> struct LaneT<double, 1> { typedef double2 type; };
template <> struct LaneT<double, 2> { typedef W32D type; };
template <> struct LaneT<float, 1> { typedef float2 type; };
template <> struct LaneT<float, 2> { typedef float4 type; };
template <> struct LaneT<float, 4> { typedef W32F type; };

template <typename V, int SPL> struct Cv {
    V re[SPL], im[SPL];
};

__device__ __forceinline__ void unpack(const double2 &v, Cv<double, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unpack(const float2 &v, Cv<float, 1> &o) { o.re[0] = v.x; o.im[0] = v.y; }
__device__ __forceinline__ void unpack(const float4 &v, Cv<float, 2> &o)
{
    o.re[0] = v.x; o.im[0] = v.y; o.re[1] = v.z; o.im[1] = v.w;
}
__device__ __forceinline__ void unpack(const W32D &v, Cv<double, 2> &o)
{
    o.re[0] = v.a.x; o.im[0] = v.a.y; o.re[1] = v.b.x; o.im[1] = v.b.y;
}
__device__ __forceinline__ void unpack(const W32F &v, Cv<float, 4> &o)
{
    o.re[0] = v.a.x; o.im[0] = v.a.y; o.re[1] = v.a.z; o.im[1] = v.a.w;
    o.re[2] = v.b.x; o.im[2] = v.b.y; o.re[3] = v.b.z; o.im[3] = v.b.w;
}
__device__ __forceinline__ double2 pack(const Cv<double, 1> &o) { return make_double2(o.re[0], o.im[0]); }
__device__ __forceinline__ float2 pack(const Cv<float, 1> &o) { return make_float2(o.re[0], o.im[0]); }
__device__ __forceinline__ float4 pack(const Cv<float, 2> &o)
{
    return make_float4(o.re[0], o.im[0], o.re[1], o.im[1]);
}
__device__ __forceinline__ W32D pack(const Cv<double, 2> &o)
{
    W32D v;
    v.a = make_double2(o.re[0], o.im[0]);
    v.b = make_double2(o.re[1], o.im[1]);
    return v;
}
__device__ __forceinline__ W32F pack(const Cv<float, 4> &o)
{
    W32F v;
    v.a = make_float4(o.re[0], o.im[0], o.re[1], o.im[1]);
    v.b = make_float4(o.re[2], o.im[2], o.re[3], o.im[3]);
    return v;
}

// 16-byte lanes load as one vector access, 32-byte lanes as two.
template <typename T> __device__ __forceinline__ T lane_ldg(const T *p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ T lane_ldcs(const T *p) { return __ldcs(p); }
template <typename T> __device__ __forceinline__ T lane_ld(const T *p) { return *p; }
template <typename T> __device__ __forceinline__ void lane_st(T *p, const T &v) { *p = v; }
template <> __device__ __forceinline__ W32F lane_ldg(const W32F *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    W32F v; v.a = __ldg(q); v.b = __ldg(q + 1); return v;
}
template <> __device__ __forceinline__ W32D lane_ldg(const W32D *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    W32D v; v.a = __ldg(q); v.b = __ldg(q + 1); return v;
}
template <> __device__ __forceinline__ W32F lane_ldcs(const W32F *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    W32F v; v.a = __ldcs(q); v.b = __ldcs(q + 1); return v;
}
template <> __device__ __forceinline__ W32D lane_ldcs(const W32D *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    W32D v; v.a = __ldcs(q); v.b = __ldcs(q + 1); return v;
}
template <> __device__ __forceinline__ W32F lane_ld(const W32F *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    W32F v; v.a = q[0]; v.b = q[1]; return v;
}
template <> __device__ __forceinline__ W32D lane_ld(const W32D *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    W32D v; v.a = q[0]; v.b = q[1]; return v;
}
template <> __device__ __forceinline__ void lane_st(W32F *p, const W32F &v)
{
    float4 *q = reinterpret_cast<float4 *>(p);
    q[0] = v.a; q[1] = v.b;
}
template <> __device__ __forceinline__ void lane_st(W32D *p, const W32D &v)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = v.a; q[1] = v.b;
}

// Load the lane data of row `r` through the read-only path.
template <typename V, int L, int SPL>
__device__ __forceinline__ Cv<V, SPL> ld_ro(const void *base, int64_t r, int l)
{
    typedef typename LaneT<V, SPL>::type Lane;
    Cv<V, SPL> o;
    unpack(lane_ldg(reinterpret_cast<const Lane *>(base) + r * L + l), o);
    return o;
}
template <typename V, int L, int SPL>
__device__ __forceinline__ Cv<V, SPL> ld(const void *base, int64_t r, int l)
{
    typedef typename LaneT<V, SPL>::type Lane;
    Cv<V, SPL> o;
    unpack(lane_ld(reinterpret_cast<const Lane *>(base) + r * L + l), o);
    return o;
}
// Own-row stream read with an evict-first hint (kept out of the way of the
// gathered vector in L2).
template <typename V, int L, int SPL>
__device__ __forceinline__ Cv<V, SPL> ld_cs(const void *base, int64_t r, int l)
{
    typedef typename LaneT<V, SPL>::type Lane;
    Cv<V, SPL> o;
    unpack(lane_ldcs(reinterpret_cast<const Lane *>(base) + r * L + l), o);
    return o;
}
template <typename V, int L, int SPL>
__device__ __forceinline__ void st(void *base, int64_t r, int l, const Cv<V, SPL> &v)
{
    typedef typename LaneT<V, SPL>::type Lane;
    lane_st(reinterpret_cast<Lane *>(base) + r * L + l, pack(v));
}

// out = c psi + gamma (-i) (H~ x) + z for lane l of row r.  The own-row
// streams (psi, z) are issued first so that they are in flight while the
// dependent slice -> column -> gather chain resolves; padded slots of the
// slice cost a load of the own row (always in bounds) but no arithmetic.
// Coefficients in the kernel's own precision, read from the launch
// arguments without any FP64 -> FP32 conversion on the device (GB300 runs
// conversions involving FP64 at the FP64 rate).
template <typename V> struct Coef;
template <> struct Coef<double> {
    __device__ static double g(const TermArgs &a) { return a.gamma; }
    __device__ static double hi(const TermArgs &a) { return a.c_hi; }
    __device__ static double lo(const TermArgs &a) { return a.c_lo; }
    __device__ static const double *scale(const TermArgs &a) { return a.scale; }
    __device__ static double hu(const TermArgs &a) { return a.h_uniform; }
};
template <> struct Coef<float> {
    __device__ static float g(const TermArgs &a) { return a.gamma_f; }
    __device__ static float hi(const TermArgs &a) { return a.c_hi_f; }
    __device__ static float lo(const TermArgs &a) { return a.c_lo_f; }
    __device__ static const float *scale(const TermArgs &a) { return a.scale_f; }
    __device__ static float hu(const TermArgs &a) { return a.h_uniform_f; }
};

template <typename V> struct Val2;
template <> struct Val2<double> { typedef double2 type; };
template <> struct Val2<float> { typedef float2 type; };

// FP64 one-value form (every off-diagonal entry equal to h): a row's
// neighbours are added first, s = x_k1 + x_k2 + ... in stored order, and
// gamma enters through gd = gamma d_r and gh = gamma h:
//   out = z + (-i)(gd x_r + gh s) + c psi,
// evaluated per component as fma(gh, s, fma(gd, x_r, fma(c, psi, z))) with
// the signs of (-i): the own-row product first, the neighbours last.  That is 2(E-1) adds and 6 FMAs per state and row for E
// entries (4 FMAs without a diagonal), against 6 + 2E operations when the
// product is formed entry by entry; GB300 runs the FP64 form at its FP64
// instruction rate, so the count sets its time.  (The FP32 form, bound by
// memory, keeps the entry-by-entry order of the general form.)  gd is read
// when the host formed it exactly (|gamma| = 1 or 2), else multiplied.
__device__ __forceinline__ double gdiag_at(const TermArgs &a, int64_t r)
{
    if (a.gdiag) return xor_sign(__ldg(a.gdiag + r), a.gdiag_sign);
    return a.gamma * __ldg(reinterpret_cast<const double *>(a.H.diag) + r);
}

// the combine above for SPL states; xo is unused when zero_diag
template <int SPL>
__device__ __forceinline__ Cv<double, SPL> combine_sum(const TermArgs &a, double gd,
                                                       const Cv<double, SPL> &xo,
                                                       const Cv<double, SPL> &s,
                                                       const Cv<double, SPL> &p,
                                                       const Cv<double, SPL> &zz)
{
    const double gh = a.gh, ch = a.c_hi;
    Cv<double, SPL> o;
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        double re = fma(ch, p.re[j], zz.re[j]);
        double im = fma(ch, p.im[j], zz.im[j]);
        if (!a.zero_diag) {
            re = fma(gd, xo.im[j], re);
            im = fma(-gd, xo.re[j], im);
        }
        o.re[j] = fma(gh, s.im[j], re);
        o.im[j] = fma(-gh, s.re[j], im);
    }
    return o;
}

template <int L, int SPL, int RS>
__device__ __forceinline__ Cv<double, SPL> term_row_sum(const TermArgs &a, int64_t r, int l,
                                                        const double *sc, int part)
{
    typedef double V;
    Cv<V, SPL> p, zz;
    if (a.variant & kVariantStreamHints) {
        p = ld_cs<V, L, SPL>(a.psi, r, l);
        if (a.z) zz = ld_cs<V, L, SPL>(a.z, r, l);
    } else {
        p = ld_ro<V, L, SPL>(a.psi, r, l);
        if (a.z) zz = ld<V, L, SPL>(a.z, r, l);
    }
    if (!a.z) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
    }
    Cv<V, SPL> xo;
    V gd = 0;
    if (!a.zero_diag) {
        xo = ld_ro<V, L, SPL>(a.x, r, l);
        gd = gdiag_at(a, r);
    }
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    int64_t base;
    int w;
    if (a.fixed_width) {
        w = a.fixed_width;
        base = q * (kSliceRows * (int64_t)w);
    } else {
        base = __ldg(a.H.slice_ptr + q);
        w = (int)((__ldg(a.H.slice_ptr + q + 1) - base) / kSliceRows);
    }
    const int32_t *colp = a.H.col + base + lr;
    Cv<V, SPL> s;
#pragma unroll
    for (int j = 0; j < SPL; ++j) { s.re[j] = 0; s.im[j] = 0; }
    // entries part, part + RS, ...: a row's entries precede its padding
    // (column = own row), so the part's first slot starts the sum or the
    // part has none
    auto group = [&](int k, auto first) {
        int32_t c[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ku = k + u * RS;
            ok[u] = ku < w;
            c[u] = ok[u] ? __ldg(colp + (int64_t)ku * kSliceRows) : (int32_t)r;
            ok[u] = ok[u] && c[u] != (int32_t)r;
        }
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_ro<V, L, SPL>(a.x, c[u], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (decltype(first)::value && u == 0) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    s.re[j] = ok[0] ? xv[0].re[j] : 0.0;
                    s.im[j] = ok[0] ? xv[0].im[j] : 0.0;
                }
            } else if (ok[u]) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    s.re[j] += xv[u].re[j];
                    s.im[j] += xv[u].im[j];
                }
            }
        }
    };
    if (part < w) {
        group(part, std::true_type{});
        for (int k = part + 4 * RS; k < w; k += 4 * RS) group(k, std::false_type{});
    }
    if (RS > 1) {
#pragma unroll
        for (int o = 1; o < RS; o <<= 1)
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                s.re[j] += __shfl_xor_sync(0xffffffffu, s.re[j], o);
                s.im[j] += __shfl_xor_sync(0xffffffffu, s.im[j], o);
            }
    }
    if (sc) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const V sv = sc[l * SPL + j];
            p.re[j] *= sv;
            p.im[j] *= sv;
            if (a.x_is_psi) {
                s.re[j] *= sv;
                s.im[j] *= sv;
                xo.re[j] *= sv;
                xo.im[j] *= sv;
            }
        }
    }
    return combine_sum<SPL>(a, gd, xo, s, p, zz);
}

// CX: complex matrix values (re, im) per stored entry (Peierls phases);
// otherwise real values.  RS > 1 splits each row's entries over RS adjacent
// threads (part = 0 .. RS-1 takes entries part, part + RS, ...; shuffles add
// the parts): long rows get RS times the gathers in flight.
template <typename V, int L, int SPL, bool CX, int RS = 1>
__device__ __forceinline__ Cv<V, SPL> term_row(const TermArgs &a, int64_t r, int l,
                                               const V *sc, int part = 0)
{
    if constexpr (sizeof(V) == 8 && !CX) {
        if (a.uniform) return term_row_sum<L, SPL, RS>(a, r, l, sc, part);
    }
    Cv<V, SPL> p, zz;
    if (a.variant & kVariantStreamHints) {
        p = ld_cs<V, L, SPL>(a.psi, r, l);
        if (a.z) zz = ld_cs<V, L, SPL>(a.z, r, l);
    } else {
        p = ld_ro<V, L, SPL>(a.psi, r, l);
        if (a.z) zz = ld<V, L, SPL>(a.z, r, l);
    }
    if (!a.z) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
    }
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    int64_t base;
    int w;
    if (a.fixed_width) {        // no slice-pointer load: one dependent round trip less
        w = a.fixed_width;
        base = q * (kSliceRows * (int64_t)w);
    } else {
        base = __ldg(a.H.slice_ptr + q);
        w = (int)((__ldg(a.H.slice_ptr + q + 1) - base) / kSliceRows);
    }
    const int32_t *colp = a.H.col + base + lr;
    const V *valp = reinterpret_cast<const V *>(a.H.val) + base + lr;

    // y = H~ x: diagonal first, then the row's entries in stored order,
    // four at a time so that the gathers are in flight together.
    const V d = part == 0 ? __ldg(reinterpret_cast<const V *>(a.H.diag) + r) : (V)0;
    Cv<V, SPL> y = ld_ro<V, L, SPL>(a.x, r, l);
#pragma unroll
    for (int j = 0; j < SPL; ++j) { y.re[j] *= d; y.im[j] *= d; }
    typedef typename Val2<V>::type V2;
    const V2 *valp2 = reinterpret_cast<const V2 *>(a.H.val) + base + lr;
    for (int k = part; k < w; k += 4 * RS) {
        int32_t c[4];
        V h[4], hm[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ku = k + u * RS;
            ok[u] = ku < w;
            c[u] = ok[u] ? __ldg(colp + (int64_t)ku * kSliceRows) : (int32_t)r;
            hm[u] = (V)0;
            if (CX) {
                V2 v2;
                v2.x = (V)0;
                v2.y = (V)0;
                if (ok[u]) v2 = __ldg(valp2 + (int64_t)ku * kSliceRows);
                h[u] = v2.x;
                hm[u] = v2.y;
            } else if (a.uniform) {
                // one value for all entries; padded slots (col == own row) add nothing
                ok[u] = ok[u] && c[u] != (int32_t)r;
                h[u] = Coef<V>::hu(a);
            } else {
                h[u] = ok[u] ? __ldg(valp + (int64_t)ku * kSliceRows) : (V)0;
            }
        }
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_ro<V, L, SPL>(a.x, c[u], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    y.re[j] = fma(h[u], xv[u].re[j], y.re[j]);
                    y.im[j] = fma(h[u], xv[u].im[j], y.im[j]);
                    if (CX) {       // (h + i hm)(x_re + i x_im)
                        y.re[j] = fma(-hm[u], xv[u].im[j], y.re[j]);
                        y.im[j] = fma(hm[u], xv[u].re[j], y.im[j]);
                    }
                }
            }
        }
    }
    if (RS > 1) {           // add the parts of the row (adjacent lanes of a warp)
#pragma unroll
        for (int o = 1; o < RS; o <<= 1)
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                y.re[j] += __shfl_xor_sync(0xffffffffu, y.re[j], o);
                y.im[j] += __shfl_xor_sync(0xffffffffu, y.im[j], o);
            }
    }
    if (sc) {               // FP32 norm carry: psi -> psi * scale (per state)
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const V s = sc[l * SPL + j];
            p.re[j] *= s;
            p.im[j] *= s;
            if (a.x_is_psi) { y.re[j] *= s; y.im[j] *= s; }
        }
    }
    const V g = Coef<V>::g(a), ch = Coef<V>::hi(a), cl = Coef<V>::lo(a);
    Cv<V, SPL> o;
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        // (-i)(y_re + i y_im) = y_im - i y_re
        V re = fma(g, y.im[j], zz.re[j]);
        V im = fma(-g, y.re[j], zz.im[j]);
        if (sizeof(V) == 4) {           // coefficient carried as hi + lo in FP32
            re = fma(cl, p.re[j], re);
            im = fma(cl, p.im[j], im);
        }
        o.re[j] = fma(ch, p.re[j], re);
        o.im[j] = fma(ch, p.im[j], im);
    }
    return o;
}

// Block index in traversal order: with kVariantZigZag the term kernels walk
// the rows from the end on odd launches, so they start on the rows the
// previous launch wrote last (still in L2).
__device__ __forceinline__ int64_t block_in_order(const TermArgs &a)
{
    return a.reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x;
}

// FP32: at most 40 registers for 16-byte lanes and 64 for the wide lanes
// (16 blocks of 64 threads per SM, without spills; the 85-register bound
// before was 5 % slower per term) -- the kernel is latency-bound, so
// residency matters; FP64: 64 registers for 16-byte lanes, 85 for the wide
// lanes (the one-value form's summed path and the general path share the
// kernel: uncapped, the pair took 94 registers and halved the resident
// warps).
// Thread t works on row t / (L RS), lane (t / RS) % L, part t % RS.  Rows are
// a multiple of 1024, so a warp never straddles the last row (the part
// shuffles see full warps).
template <typename V, int L, int SPL, bool CX, int RS>
__global__ void __launch_bounds__(256, sizeof(V) == 4 ? (SPL <= 2 ? 6 : 4) : (SPL == 1 ? 4 : 3)) k_term(TermArgs a)
{
    const int64_t t = block_in_order(a) * blockDim.x + threadIdx.x;
    const int64_t r = t / (L * RS);
    const int l = (int)((t / RS) % L);
    const int part = (int)(t % RS);
    if (r >= a.n_rows) return;
    const V *sc = Coef<V>::scale(a);
    if (sc) sc += (int64_t)a.chunk_sample[r / kChunkRows] * (L * SPL);
    Cv<V, SPL> o = term_row<V, L, SPL, CX, RS>(a, r, l, sc, part);
    if (part == 0) st<V, L, SPL>(a.out, r, l, o);
}

// Register-pipelined term (TBPM_VARIANT_PREFETCH; real values): a
// persistent grid whose threads walk rows with a stride (in zig-zag order
// when asked).  A row's first four column indices, their values and its
// diagonal are loaded one row ahead, so the row's own-row loads and its
// gathers leave together instead of the gathers waiting on the column
// loads.  Per row the arithmetic and its order are term_row's (plain
// kernel; in FP64 with one value, term_row_sum's): the states are
// bit-identical to it.
template <typename V>
struct RowAhead {
    int64_t base;
    int w;
    int32_t c[4];
    V h[4];
    V d;
};

template <typename V, int L, int SPL>
__device__ __forceinline__ void row_ahead(const TermArgs &a, int64_t r, RowAhead<V> &n)
{
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    if (a.fixed_width) {
        n.w = a.fixed_width;
        n.base = q * (kSliceRows * (int64_t)n.w);
    } else {
        n.base = __ldg(a.H.slice_ptr + q);
        n.w = (int)((__ldg(a.H.slice_ptr + q + 1) - n.base) / kSliceRows);
    }
    const int32_t *colp = a.H.col + n.base + lr;
    const V *valp = reinterpret_cast<const V *>(a.H.val) + n.base + lr;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool ok = u < n.w;
        n.c[u] = ok ? __ldg(colp + (int64_t)u * kSliceRows) : (int32_t)r;
        n.h[u] = a.uniform ? Coef<V>::hu(a) : (ok ? __ldg(valp + (int64_t)u * kSliceRows) : (V)0);
    }
    n.d = __ldg(reinterpret_cast<const V *>(a.H.diag) + r);
    if constexpr (sizeof(V) == 8) {              // FP64 one-value form: gamma d
        if (a.uniform) n.d = a.zero_diag ? 0.0 : gdiag_at(a, r);
    }
}

template <typename V, int L, int SPL>
__global__ void __launch_bounds__(256, sizeof(V) == 4 ? (SPL <= 2 ? 4 : 3) : 2) k_term_pf(TermArgs a)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t rows_per_pass = (int64_t)gridDim.x * blockDim.x / L;
    const int l = (int)(t % L);
    int64_t i = t / L;                                   // position in traversal order
    auto row_of = [&](int64_t k) { return a.reverse ? a.n_rows - 1 - k : k; };
    RowAhead<V> cur;
    if (i < a.n_rows) row_ahead<V, L, SPL>(a, row_of(i), cur);
    for (; i < a.n_rows; i += rows_per_pass) {
        const int64_t r = row_of(i);
        Cv<V, SPL> p, zz;
        if (a.variant & kVariantStreamHints) {
            p = ld_cs<V, L, SPL>(a.psi, r, l);
            if (a.z) zz = ld_cs<V, L, SPL>(a.z, r, l);
        } else {
            p = ld_ro<V, L, SPL>(a.psi, r, l);
            if (a.z) zz = ld<V, L, SPL>(a.z, r, l);
        }
        if (!a.z) {
#pragma unroll
            for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
        }
        Cv<V, SPL> y = ld_ro<V, L, SPL>(a.x, r, l);
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_ro<V, L, SPL>(a.x, cur.c[u], l);
        // the next row's indices, values and diagonal, in flight meanwhile
        RowAhead<V> nxt;
        const int64_t i2 = i + rows_per_pass;
        if (i2 < a.n_rows) row_ahead<V, L, SPL>(a, row_of(i2), nxt);
        if constexpr (sizeof(V) == 8) {
            if (a.uniform) {
                // FP64 one-value form (term_row_sum): neighbours summed in
                // stored order, the first valid entry starting the sum
                Cv<V, SPL> sm;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = u < cur.w && cur.c[u] != (int32_t)r;
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        if (u == 0) {
                            sm.re[j] = ok ? xv[0].re[j] : 0.0;
                            sm.im[j] = ok ? xv[0].im[j] : 0.0;
                        } else if (ok) {
                            sm.re[j] += xv[u].re[j];
                            sm.im[j] += xv[u].im[j];
                        }
                    }
                }
                const int64_t lr0 = r % kSliceRows;
                for (int k = 4; k < cur.w; k += 4) {
                    int32_t c[4];
                    bool okk[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        okk[u] = k + u < cur.w;
                        c[u] = okk[u] ? __ldg(a.H.col + cur.base + lr0 + (int64_t)(k + u) * kSliceRows)
                                      : (int32_t)r;
                        okk[u] = okk[u] && c[u] != (int32_t)r;
                    }
                    Cv<V, SPL> xw[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xw[u] = ld_ro<V, L, SPL>(a.x, c[u], l);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (okk[u]) {
#pragma unroll
                            for (int j = 0; j < SPL; ++j) {
                                sm.re[j] += xw[u].re[j];
                                sm.im[j] += xw[u].im[j];
                            }
                        }
                    }
                }
                const V *sc = Coef<V>::scale(a);
                if (sc) {
                    sc += (int64_t)a.chunk_sample[r / kChunkRows] * (L * SPL);
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
                st<V, L, SPL>(a.out, r, l, combine_sum<SPL>(a, cur.d, y, sm, p, zz));
                cur = nxt;
                continue;
            }
        }
#pragma unroll
        for (int j = 0; j < SPL; ++j) { y.re[j] *= cur.d; y.im[j] *= cur.d; }
        // the first four entries (as term_row's first round), then the rest
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ok[u] = u < cur.w;
            if (a.uniform) ok[u] = ok[u] && cur.c[u] != (int32_t)r;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    y.re[j] = fma(cur.h[u], xv[u].re[j], y.re[j]);
                    y.im[j] = fma(cur.h[u], xv[u].im[j], y.im[j]);
                }
            }
        }
        const int64_t lr = r % kSliceRows;
        for (int k = 4; k < cur.w; k += 4) {
            int32_t c[4];
            V h[4];
            bool okk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ku = k + u;
                okk[u] = ku < cur.w;
                c[u] = okk[u] ? __ldg(a.H.col + cur.base + lr + (int64_t)ku * kSliceRows)
                              : (int32_t)r;
                if (a.uniform) {
                    okk[u] = okk[u] && c[u] != (int32_t)r;
                    h[u] = Coef<V>::hu(a);
                } else {
                    h[u] = okk[u] ? __ldg(reinterpret_cast<const V *>(a.H.val) + cur.base + lr +
                                          (int64_t)ku * kSliceRows)
                                  : (V)0;
                }
            }
            Cv<V, SPL> xw[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xw[u] = ld_ro<V, L, SPL>(a.x, c[u], l);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (okk[u]) {
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        y.re[j] = fma(h[u], xw[u].re[j], y.re[j]);
                        y.im[j] = fma(h[u], xw[u].im[j], y.im[j]);
                    }
                }
            }
        }
        const V *sc = Coef<V>::scale(a);
        if (sc) {
            sc += (int64_t)a.chunk_sample[r / kChunkRows] * (L * SPL);
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const V s = sc[l * SPL + j];
                p.re[j] *= s;
                p.im[j] *= s;
                if (a.x_is_psi) { y.re[j] *= s; y.im[j] *= s; }
            }
        }
        const V g = Coef<V>::g(a), ch = Coef<V>::hi(a), cl = Coef<V>::lo(a);
        Cv<V, SPL> o;
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
        st<V, L, SPL>(a.out, r, l, o);
        cur = nxt;
    }
}

// Closing term, one row per thread like k_term, with the sums of
// <psi0|out> and <out|out> per state into one partial per block, then the
// last block of each kChunkRows chunk (atomic ticket after a fence) adds the
// chunk's block partials in block order.  Every sum has a fixed order, so the
// result does not depend on which block finishes last.
//
// GB300 runs FP64 at a small fraction of the FP32 rate, so the FP32 form's
// reduction stays on the FP32 pipe without giving up FP64-grade sums: each
// row's products are exact float pairs (TwoProduct), the block's rows are
// added as pairs (TwoSum, Fast2Sum; about 48 significant bits), and one
// pair -> FP64 conversion per value and block hands over to FP64 from the
// block partials up.  In the FP64 form every product and sum is FP64, with
// rows summed in a shared-memory tree (one add per value) instead of a
// butterfly (one add per value and level on every lane).
constexpr int kFinalThreads = 128;

// Block reduction of the closing term: block `bid` covers ROWS rows, thread
// (lrow, l) holds the lane values o of its row and psi0's p0.  Writes the
// block partial; the chunk's last block adds the chunk's partials in order.
template <typename V, int L, int SPL, int ROWS>
__device__ __forceinline__ void final_reduce(const TermArgs &a, int64_t bid, int lrow, int l,
                                             const Cv<V, SPL> &o, const Cv<V, SPL> &p0)
{
    constexpr int B = L * SPL;
    constexpr int NT = ROWS * L;                     // threads of the block
    constexpr int NV = B * 3;                        // (re, im, norm) per state
    constexpr int P = NT / NV;                       // FP32: parts per value
    __shared__ double red[sizeof(V) == 8 ? ROWS * NV : 1];
    __shared__ FF redf[sizeof(V) == 4 ? ROWS * NV : 1];
    __shared__ FF redp[sizeof(V) == 4 ? P * NV : 1];
    __shared__ double grp[8][NV];
    __shared__ int last;
    if constexpr (sizeof(V) == 4) {
        // FP32: exact per-row products as float pairs, [row][value] in shared
        // memory; value v's rows are summed in P fixed parts (rows part,
        // part + P, ...), then the parts in order
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            FF re, im, nr;
            ff_dot3((float)p0.re[j], (float)p0.im[j], (float)o.re[j], (float)o.im[j], re, im, nr);
            const int v = (l * SPL + j) * 3;
            redf[lrow * NV + v + 0] = re;
            redf[lrow * NV + v + 1] = im;
            redf[lrow * NV + v + 2] = nr;
        }
        __syncthreads();
        if (threadIdx.x < P * NV) {
            const int v = threadIdx.x % NV, part = threadIdx.x / NV;
            FF acc = redf[part * NV + v];
            for (int row = part + P; row < ROWS; row += P) acc = ff_add(acc, redf[row * NV + v]);
            redp[threadIdx.x] = acc;
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            FF acc = redp[threadIdx.x];
            for (int part = 1; part < P; ++part) acc = ff_add(acc, redp[part * NV + threadIdx.x]);
            grp[0][threadIdx.x] = ff_to_double(acc);
        }
    } else {
        // FP64: shared-memory tree, 8 groups of rows then the groups
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const int v = (l * SPL + j) * 3;
            red[lrow * NV + v + 0] = fma(p0.re[j], o.re[j], p0.im[j] * o.im[j]);
            red[lrow * NV + v + 1] = fma(p0.re[j], o.im[j], -(p0.im[j] * o.re[j]));
            red[lrow * NV + v + 2] = fma(o.re[j], o.re[j], o.im[j] * o.im[j]);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < 8 * NV; idx += NT) {
            const int gidx = idx / NV, v = idx % NV;
            double s = 0.0;
            for (int row = gidx; row < ROWS; row += 8) s += red[row * NV + v];
            grp[gidx][v] = s;
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            double s = 0.0;
            for (int g2 = 0; g2 < 8; ++g2) s += grp[g2][threadIdx.x];
            grp[0][threadIdx.x] = s;
        }
    }
    __syncthreads();
    constexpr int per_chunk = kChunkRows / ROWS;     // blocks per chunk
    const int64_t chunk = bid / per_chunk;
    if (threadIdx.x == 0) {
        // one writer, one fence, one ticket per block
        for (int v = 0; v < NV; ++v) a.block_partial[bid * NV + v] = grp[0][v];
        __threadfence();
        const int ticket = atomicAdd(a.chunk_count + chunk, 1);
        last = (ticket == per_chunk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < NV) {
            double s = 0.0;
            const int64_t b0 = chunk * per_chunk;
            for (int k = 0; k < per_chunk; ++k)
                s += __ldcg(a.block_partial + (b0 + k) * NV + threadIdx.x);
            a.partial[chunk * NV + threadIdx.x] = s;
        }
        if (threadIdx.x == 0) a.chunk_count[chunk] = 0;     // ready for the next launch
    }
}

template <typename V, int L, int SPL, bool COMPUTE, bool CX>
__global__ void __launch_bounds__(kFinalThreads) k_final(TermArgs a)
{
    constexpr int B = L * SPL;
    const int64_t bid = block_in_order(a);
    const int64_t t = bid * kFinalThreads + threadIdx.x;
    const int64_t r = t / L;
    const int l = (int)(t % L);
    const V *sc = Coef<V>::scale(a);
    if (sc) sc += (int64_t)a.chunk_sample[r / kChunkRows] * B;
    Cv<V, SPL> o;
    if (COMPUTE) {
        o = term_row<V, L, SPL, CX>(a, r, l, sc);
        st<V, L, SPL>(a.out, r, l, o);
    } else {
        o = ld<V, L, SPL>(a.out, r, l);
    }
    const Cv<V, SPL> p0 = ld_ro<V, L, SPL>(a.psi0, r, l);
    final_reduce<V, L, SPL, kFinalThreads / L>(a, bid, threadIdx.x / L, l, o, p0);
}

// Reduction-only closing pass, FP32 (after a term kernel that wrote `out`,
// and the C_0 pass): RPT rows per thread (rows lrow, lrow + ROWS, ... of the
// block's ROWS * RPT), each row's <psi0|phi> and <phi|phi> terms exact float
// pairs added in registers, then the block's threads through a [row][value]
// table in fixed parts as in final_reduce, one FP64 partial per block and
// the chunk tickets.  The block-table phases then serve RPT times the rows.
template <int L, int SPL, int RPT>
__global__ void __launch_bounds__(kFinalThreads) k_final_sums(TermArgs a)
{
    constexpr int B = L * SPL;
    constexpr int ROWS = kFinalThreads / L;          // thread-rows of a block
    constexpr int NV = B * 3;
    constexpr int P = kFinalThreads / NV;            // parts per value
    __shared__ FF redf[ROWS * NV];
    __shared__ FF redp[P * NV];
    __shared__ double tot[NV];
    __shared__ int last;
    const int64_t bid = block_in_order(a);
    const int lrow = threadIdx.x / L, l = threadIdx.x % L;
    const int64_t r0 = bid * (int64_t)(ROWS * RPT) + lrow;
    FF acc[SPL][3];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int64_t r = r0 + (int64_t)k * ROWS;
        const Cv<float, SPL> o = ld<float, L, SPL>(a.out, r, l);
        const Cv<float, SPL> p0 = ld_ro<float, L, SPL>(a.psi0, r, l);
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            FF re, im, nr;
            ff_dot3(p0.re[j], p0.im[j], o.re[j], o.im[j], re, im, nr);
            if (k == 0) {
                acc[j][0] = re;
                acc[j][1] = im;
                acc[j][2] = nr;
            } else {
                acc[j][0] = ff_add(acc[j][0], re);
                acc[j][1] = ff_add(acc[j][1], im);
                acc[j][2] = ff_add(acc[j][2], nr);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        const int v = (l * SPL + j) * 3;
        redf[lrow * NV + v + 0] = acc[j][0];
        redf[lrow * NV + v + 1] = acc[j][1];
        redf[lrow * NV + v + 2] = acc[j][2];
    }
    __syncthreads();
    if (threadIdx.x < P * NV) {
        const int v = threadIdx.x % NV, part = threadIdx.x / NV;
        FF s = redf[part * NV + v];
        for (int row = part + P; row < ROWS; row += P) s = ff_add(s, redf[row * NV + v]);
        redp[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        FF s = redp[threadIdx.x];
        for (int part = 1; part < P; ++part) s = ff_add(s, redp[part * NV + threadIdx.x]);
        tot[threadIdx.x] = ff_to_double(s);
    }
    __syncthreads();
    constexpr int per_chunk = kChunkRows / (ROWS * RPT);   // blocks per chunk
    const int64_t chunk = bid / per_chunk;
    if (threadIdx.x == 0) {
        for (int v = 0; v < NV; ++v) a.block_partial[bid * NV + v] = tot[v];
        __threadfence();
        const int ticket = atomicAdd(a.chunk_count + chunk, 1);
        last = (ticket == per_chunk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < NV) {
            double sum = 0.0;
            const int64_t b0 = chunk * per_chunk;
            for (int k = 0; k < per_chunk; ++k)
                sum += __ldcg(a.block_partial + (b0 + k) * NV + threadIdx.x);
            a.partial[chunk * NV + threadIdx.x] = sum;
        }
        if (threadIdx.x == 0) a.chunk_count[chunk] = 0;     // ready for the next launch
    }
}

// ---- staged-gather term (TBPM_VARIANT_HALO) --------------------------------
// A block of kHaloRows rows first copies its halo -- the x lanes of its own
// rows, then of every other row its entries reference -- into shared memory
// with 16-byte asynchronous copies, then gathers from that copy by the 16-bit
// positions lcol: long rows (the twisted bilayer's ~68 entries) then read
// their neighbours' states from shared memory instead of L1/L2 lines.  The
// 16-byte chunks of a row are XOR-permuted by the row's position so that
// rows sharing a 128-byte bank line spread their chunks over all banks.
// Real values and 32-byte lanes (two chunks per lane); the arithmetic and
// its order are term_row's, so the states are bit-identical to it.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Chunk permutation of halo row h for C chunks per row (C = 2, 4, 8).
template <int C> __device__ __forceinline__ int halo_swz(int h)
{
    return (h >> (C == 2 ? 2 : C == 4 ? 1 : 0)) & (C - 1);
}

template <typename V, int L, int SPL>
__device__ __forceinline__ Cv<V, SPL> ld_halo(const unsigned char *xs, int h, int l)
{
    constexpr int C = 2 * L;
    typedef typename LaneT<V, SPL>::type Lane;
    const int sw = halo_swz<C>(h);
    Lane v;
    typedef typename std::conditional<sizeof(V) == 4, float4, double2>::type Half;
    Half *hv = reinterpret_cast<Half *>(&v);
    hv[0] = *reinterpret_cast<const Half *>(xs + (h * C + ((2 * l) ^ sw)) * 16);
    hv[1] = *reinterpret_cast<const Half *>(xs + (h * C + ((2 * l + 1) ^ sw)) * 16);
    Cv<V, SPL> o;
    unpack(v, o);
    return o;
}

// The FP64 one-value form (term_row_sum) with the neighbours gathered from
// the block's shared copy by their packed 16-bit positions.
template <int L, int SPL>
__device__ __forceinline__ Cv<double, SPL> halo_row_sum(const TermArgs &a, const unsigned char *xs,
                                                        int lr, int l, int w, const uint16_t *lcp,
                                                        const double *sc, double gd,
                                                        Cv<double, SPL> p, const Cv<double, SPL> &zz)
{
    typedef double V;
    Cv<V, SPL> xo, s;
    if (!a.zero_diag) xo = ld_halo<V, L, SPL>(xs, lr, l);
#pragma unroll
    for (int j = 0; j < SPL; ++j) { s.re[j] = 0; s.im[j] = 0; }
    auto group = [&](int k, auto first) {
        int hp[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ku = k + u;
            ok[u] = ku < w;
            hp[u] = ok[u] ? (int)__ldg(lcp + (ku >> 2) * (4 * kSliceRows) + (ku & 3)) : lr;
            ok[u] = ok[u] && hp[u] != lr;            // padded slots point at the own row
        }
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_halo<V, L, SPL>(xs, hp[u], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (decltype(first)::value && u == 0) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    s.re[j] = ok[0] ? xv[0].re[j] : 0.0;
                    s.im[j] = ok[0] ? xv[0].im[j] : 0.0;
                }
            } else if (ok[u]) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    s.re[j] += xv[u].re[j];
                    s.im[j] += xv[u].im[j];
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
            if (a.x_is_psi) {
                s.re[j] *= sv;
                s.im[j] *= sv;
                xo.re[j] *= sv;
                xo.im[j] *= sv;
            }
        }
    }
    return combine_sum<SPL>(a, gd, xo, s, p, zz);
}

// 64 registers a thread (1024 resident threads per SM, no spills).
template <typename V, int L, int SPL, bool FINAL>
__global__ void __launch_bounds__(kHaloRows * L, 8 / L) k_term_halo(TermArgs a)
{
    extern __shared__ __align__(16) unsigned char xs[];
    constexpr int C = 2 * L;                     // 16-byte chunks per row of x
    constexpr int NT = kHaloRows * L;
    const int64_t hb = block_in_order(a);
    const int tid = threadIdx.x;
    const int lr = tid / L, l = tid % L;
    const int64_t r = hb * kHaloRows + lr;
    // own-row streams first: in flight while the halo arrives
    Cv<V, SPL> p = ld_ro<V, L, SPL>(a.psi, r, l), zz;
    if (a.z) {
        zz = ld<V, L, SPL>(a.z, r, l);
    } else {
#pragma unroll
        for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
    }
    const V *sc = Coef<V>::scale(a);
    if (sc) sc += (int64_t)a.chunk_sample[r / kChunkRows] * (L * SPL);
    const int64_t h0 = a.halo_ptr[hb];
    const int H = (int)(a.halo_ptr[hb + 1] - h0);
    const unsigned char *xg = reinterpret_cast<const unsigned char *>(a.x);
    for (int idx = tid; idx < H * C; idx += NT) {
        const int h = idx / C, c = idx % C;
        const int64_t g = __ldg(a.halo_rows + h0 + h);
        cp_async16(xs + (h * C + (c ^ halo_swz<C>(h))) * 16, xg + (g * C + c) * 16);
    }
    const int64_t q = r / kSliceRows;
    int64_t base;
    int w;
    if (a.fixed_width) {
        w = a.fixed_width;
        base = q * (kSliceRows * (int64_t)w);
    } else {
        base = __ldg(a.H.slice_ptr + q);
        w = (int)((__ldg(a.H.slice_ptr + q + 1) - base) / kSliceRows);
    }
    const uint16_t *lcp = a.lcol + a.pslice[q] + (r % kSliceRows) * 4;     // packed
    const V *valp = reinterpret_cast<const V *>(a.H.val) + base + (r % kSliceRows);
    const V d = __ldg(reinterpret_cast<const V *>(a.H.diag) + r);
    V gd = 0;
    if constexpr (sizeof(V) == 8) {
        if (a.uniform && !a.zero_diag) gd = gdiag_at(a, r);
    }
    cp_async_wait_all();
    __syncthreads();

    Cv<V, SPL> o;
    if constexpr (sizeof(V) == 8) {
        if (a.uniform) {                 // FP64 one-value form: neighbours summed first
            o = halo_row_sum<L, SPL>(a, xs, lr, l, w, lcp, sc, gd, p, zz);
            st<V, L, SPL>(a.out, r, l, o);
            if constexpr (FINAL) {
                const Cv<V, SPL> p0 = ld_ro<V, L, SPL>(a.psi0, r, l);
                final_reduce<V, L, SPL, kHaloRows>(a, hb, lr, l, o, p0);
            }
            return;
        }
    }
    Cv<V, SPL> y = ld_halo<V, L, SPL>(xs, lr, l);
#pragma unroll
    for (int j = 0; j < SPL; ++j) { y.re[j] *= d; y.im[j] *= d; }
    for (int k = 0; k < w; k += 4) {
        int hp[4];
        V h[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ku = k + u;
            ok[u] = ku < w;
            hp[u] = ok[u] ? (int)__ldg(lcp + (ku >> 2) * (4 * kSliceRows) + (ku & 3)) : lr;
            if (a.uniform) {
                ok[u] = ok[u] && hp[u] != lr;        // padded slots point at the own row
                h[u] = Coef<V>::hu(a);
            } else {
                h[u] = ok[u] ? __ldg(valp + (int64_t)ku * kSliceRows) : (V)0;
            }
        }
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_halo<V, L, SPL>(xs, hp[u], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (ok[u]) {
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
            if (a.x_is_psi) { y.re[j] *= s; y.im[j] *= s; }
        }
    }
    const V g = Coef<V>::g(a), ch = Coef<V>::hi(a), cl = Coef<V>::lo(a);
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
    st<V, L, SPL>(a.out, r, l, o);
    if constexpr (FINAL) {
        const Cv<V, SPL> p0 = ld_ro<V, L, SPL>(a.psi0, r, l);
        final_reduce<V, L, SPL, kHaloRows>(a, hb, lr, l, o, p0);
    }
}

template <typename V, int L, int SPL, bool FINAL>
cudaError_t launch_halo_t(const TermArgs &a, cudaStream_t st)
{
    static int configured = -1;              // dynamic shared bytes already allowed
    const int smem = a.halo_max * (2 * L) * 16;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_term_halo<V, L, SPL, FINAL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    const unsigned blocks = (unsigned)(a.n_rows / kHaloRows);
    k_term_halo<V, L, SPL, FINAL><<<blocks, kHaloRows * L, smem, st>>>(a);
    return cudaGetLastError();
}

// ---- pipelined staged-gather term (TBPM_VARIANT_HALO | TBPM_VARIANT_PIPE) ----
// A persistent grid (one block per SM) walks the 128-row halo blocks; while
// it computes block i from one shared-memory stage, the 16-byte asynchronous
// copies of block i+1 fill the other stage: the x lanes of its halo rows,
// and its 16-bit positions and values, each one contiguous range (the
// block's four slices).  No global load then sits between an entry and its
// gather.  Lanes are 16 bytes (two FP32 or one FP64 state), C lanes per row
// of x; same arithmetic and order as term_row, so the states are
// bit-identical to the plain kernel.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Lane l of halo row h in a stage: rows of C 16-byte chunks, chunk l of
// each row read by the row's thread l (a quarter-warp reads two whole rows,
// so no chunk permutation changes its bank conflicts); xl = stage + 16 l.
template <typename V, int C>
__device__ __forceinline__ Cv<V, 16 / (2 * sizeof(V))> ld_halo16(const unsigned char *xl, int h)
{
    constexpr int SPL = 16 / (2 * sizeof(V));
    typedef typename LaneT<V, SPL>::type Lane;
    const Lane v = *reinterpret_cast<const Lane *>(xl + h * (C * 16));
    Cv<V, SPL> o;
    unpack(v, o);
    return o;
}

struct PipeShape {
    int halo_bytes;     // halo_max x C x 16
    int lcol_bytes;     // ent_max x 2, rounded up to 16
    int val_bytes;      // ent_max x value bytes (0 in the one-value form)
    int stage_bytes;
    int n_hb;           // halo blocks
};

// The FP64 one-value form (term_row_sum) for the pipelined kernel: one
// FP64 state per 16-byte lane, four packed positions a round, the next
// round's read before this round's gathers; sc: this lane's state scale.
template <int C>
__device__ __forceinline__ Cv<double, 1> pipe_row_sum(const TermArgs &a, const unsigned char *xl,
                                                      int lr, int w, const uint16_t *lcs, double gd,
                                                      Cv<double, 1> p, const Cv<double, 1> &zz,
                                                      const double *sc)
{
    typedef double V;
    Cv<V, 1> xo, s;
    if (!a.zero_diag) xo = ld_halo16<V, C>(xl, lr);
    s.re[0] = 0;
    s.im[0] = 0;
    uint2 pk = make_uint2(0u, 0u);
    if (w > 0) pk = *reinterpret_cast<const uint2 *>(lcs);
    auto group = [&](int k, auto first) {
        const int hp[4] = {(int)(pk.x & 0xffff), (int)(pk.x >> 16), (int)(pk.y & 0xffff),
                           (int)(pk.y >> 16)};
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ok[u] = k + u < w && hp[u] != lr;   // padding: the own row
        Cv<V, 1> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_halo16<V, C>(xl, hp[u]);
        if (k + 4 < w) pk = *reinterpret_cast<const uint2 *>(lcs + ((k + 4) >> 2) * (4 * kSliceRows));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (decltype(first)::value && u == 0) {
                s.re[0] = ok[0] ? xv[0].re[0] : 0.0;
                s.im[0] = ok[0] ? xv[0].im[0] : 0.0;
            } else if (ok[u]) {
                s.re[0] += xv[u].re[0];
                s.im[0] += xv[u].im[0];
            }
        }
    };
    if (w > 0) {
        group(0, std::true_type{});
        for (int k = 4; k < w; k += 4) group(k, std::false_type{});
    }
    if (sc) {
        const V sv = *sc;
        p.re[0] *= sv;
        p.im[0] *= sv;
        if (a.x_is_psi) {
            s.re[0] *= sv;
            s.im[0] *= sv;
            xo.re[0] *= sv;
            xo.im[0] *= sv;
        }
    }
    return combine_sum<1>(a, gd, xo, s, p, zz);
}

// One row of a staged block: the term for lane l of row r (local row lr)
// from a shared-memory stage holding the block's halo rows (16-byte lanes,
// C per row), its packed 16-bit positions and, unless one value serves all,
// its packed values; w, off: the row's entry count and packed offset.  Four
// entries a round, their positions in one 8-byte and their values in one
// 16-byte (FP32) shared load, the next round's read before this round's
// gathers; same arithmetic and order as term_row.
template <typename V, int C>
__device__ __forceinline__ Cv<V, 16 / (2 * sizeof(V))> staged_row(
    const TermArgs &a, const unsigned char *stg, const PipeShape &ps, int64_t r, int lr, int l,
    int w, int off, Cv<V, 16 / (2 * sizeof(V))> p, const Cv<V, 16 / (2 * sizeof(V))> &zz, V d,
    V gd)
{
    constexpr int SPL = 16 / (2 * sizeof(V));
    const unsigned char *xl = stg + l * 16;
    const uint16_t *lcs = reinterpret_cast<const uint16_t *>(stg + ps.halo_bytes) + off;
    const V *vs = reinterpret_cast<const V *>(stg + ps.halo_bytes + ps.lcol_bytes) + off;
    if constexpr (sizeof(V) == 8) {
        if (a.uniform)                       // FP64 one-value form: neighbours summed first
            return pipe_row_sum<C>(a, xl, lr, w, lcs, gd, p, zz,
                                   Coef<V>::scale(a) ? Coef<V>::scale(a) +
                                       (int64_t)a.chunk_sample[r / kChunkRows] * (C * SPL) + l * SPL
                                                     : nullptr);
    }
    Cv<V, SPL> y = ld_halo16<V, C>(xl, lr);
#pragma unroll
    for (int j = 0; j < SPL; ++j) { y.re[j] *= d; y.im[j] *= d; }
    uint2 pk = make_uint2(0u, 0u);
    V hv[4] = {0, 0, 0, 0};
    auto load4 = [&](int k) {
        const int g4 = (k >> 2) * (4 * kSliceRows);
        pk = *reinterpret_cast<const uint2 *>(lcs + g4);
        if (!a.uniform) {
            if constexpr (sizeof(V) == 4) {
                const float4 v4 = *reinterpret_cast<const float4 *>(vs + g4);
                hv[0] = v4.x; hv[1] = v4.y; hv[2] = v4.z; hv[3] = v4.w;
            } else {
                const double2 v0 = *reinterpret_cast<const double2 *>(vs + g4);
                const double2 v1 = *reinterpret_cast<const double2 *>(vs + g4 + 2);
                hv[0] = v0.x; hv[1] = v0.y; hv[2] = v1.x; hv[3] = v1.y;
            }
        }
    };
    if (w > 0) load4(0);
    for (int k = 0; k < w; k += 4) {
        const int hp[4] = {(int)(pk.x & 0xffff), (int)(pk.x >> 16), (int)(pk.y & 0xffff),
                           (int)(pk.y >> 16)};
        V h[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ok[u] = k + u < w;
            h[u] = hv[u];
            if (a.uniform) {
                ok[u] = ok[u] && hp[u] != lr;        // padded slots point at the own row
                h[u] = Coef<V>::hu(a);
            }
        }
        Cv<V, SPL> xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = ld_halo16<V, C>(xl, hp[u]);
        if (k + 4 < w) load4(k + 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < SPL; ++j) {
                    y.re[j] = fma(h[u], xv[u].re[j], y.re[j]);
                    y.im[j] = fma(h[u], xv[u].im[j], y.im[j]);
                }
            }
        }
    }
    const V *sc = Coef<V>::scale(a);
    if (sc) {
        sc += (int64_t)a.chunk_sample[r / kChunkRows] * (C * SPL);
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const V s = sc[l * SPL + j];
            p.re[j] *= s;
            p.im[j] *= s;
            if (a.x_is_psi) { y.re[j] *= s; y.im[j] *= s; }
        }
    }
    const V g = Coef<V>::g(a), ch = Coef<V>::hi(a), cl = Coef<V>::lo(a);
    Cv<V, SPL> o;
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

// Where block j's lists start and how long they are.
struct PipeMeta {
    int64_t h0;         // first halo row of the block's list
    int64_t e0;         // first packed entry of the block's four slices
    int H;              // halo rows
    int E;              // packed entries (a multiple of 128)
};

constexpr int kPipeIdx = (kHaloRows + kHaloMaxExt + kHaloRows - 1) / kHaloRows;  // halo rows per thread

// Per thread: four entries of its row a round, their positions in one
// 8-byte and their values in one 16-byte (FP32) shared-memory load, the
// next four's loads issued before this four's gathers.  The global loads
// that address the copies are software-pipelined across the CTA's blocks:
// the list bounds of block i+3 and the halo row numbers of block i+2 are
// loaded while block i computes, so issuing block i+1's copies waits on no
// global load (with one resident block per SM every warp would otherwise
// wait on that chain together).
template <typename V, int C>
__global__ void __launch_bounds__(kHaloRows * C) k_term_halo_pipe(TermArgs a, PipeShape ps)
{
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int SPL = 16 / (2 * sizeof(V));
    constexpr int NT = kHaloRows * C;
    constexpr int SPB = kHaloRows / kSliceRows;      // slices per halo block
    const int tid = threadIdx.x;
    const int l = tid % C, lr = tid / C;
    const unsigned char *xg = reinterpret_cast<const unsigned char *>(a.x);
    const int64_t G = gridDim.x;
    auto block_at = [&](int64_t i) -> int64_t {        // i-th block of this CTA, or -1
        const int64_t k = blockIdx.x + i * G;
        if (k >= ps.n_hb) return -1;
        return a.reverse ? ps.n_hb - 1 - k : k;
    };
    auto meta_of = [&](int64_t hb) {
        PipeMeta m = {0, 0, 0, 0};
        if (hb >= 0) {
            m.h0 = __ldg(a.halo_ptr + hb);
            m.H = (int)(__ldg(a.halo_ptr + hb + 1) - m.h0);
            m.e0 = __ldg(a.pslice + hb * SPB);
            m.E = (int)(__ldg(a.pslice + (hb + 1) * SPB) - m.e0);
        }
        return m;
    };
    // halo rows lr, lr + 128, ... of a block: the x rows this thread copies
    auto rows_of = [&](const PipeMeta &m, int32_t (&g)[kPipeIdx]) {
#pragma unroll
        for (int k = 0; k < kPipeIdx; ++k) {       // predicated, not a loop exit: the
            const int h = lr + k * kHaloRows;      // loads stay ahead of their use
            g[k] = h < m.H ? __ldg(a.halo_rows + m.h0 + h) : 0;
        }
    };
    // this thread's row of block hb: its entry count and packed offset
    auto row_of = [&](int64_t hb, const PipeMeta &m, int &w, int &off) {
        w = 0;
        off = 0;
        if (hb < 0) return;
        const int64_t q = (hb * kHaloRows + lr) / kSliceRows;
        w = a.fixed_width ? a.fixed_width
                          : (int)((__ldg(a.H.slice_ptr + q + 1) - __ldg(a.H.slice_ptr + q)) / kSliceRows);
        off = (int)(__ldg(a.pslice + q) - m.e0) + (lr % kSliceRows) * 4;
    };
    auto issue = [&](const PipeMeta &m, const int32_t (&g)[kPipeIdx], int s) {
        unsigned char *stg = sm + (int64_t)s * ps.stage_bytes;
#pragma unroll
        for (int k = 0; k < kPipeIdx; ++k) {
            const int h = lr + k * kHaloRows;
            if (h < m.H) cp_async16(stg + (h * C + l) * 16, xg + ((int64_t)g[k] * C + l) * 16);
        }
        unsigned char *lc = stg + ps.halo_bytes;
        for (int idx = tid; idx < m.E / 8; idx += NT)
            cp_async16(lc + idx * 16, a.lcol + m.e0 + idx * 8);
        if (!a.uniform) {
            constexpr int per = 16 / sizeof(V);
            unsigned char *vs = lc + ps.lcol_bytes;
            for (int idx = tid; idx < m.E / per; idx += NT)
                cp_async16(vs + idx * 16, reinterpret_cast<const V *>(a.vpack) + m.e0 + idx * per);
        }
        cp_async_commit();
    };

    // prologue: block 0's copies, then the bounds and rows one and two ahead
    int64_t hb = block_at(0);
    int32_t g1[kPipeIdx];
    PipeMeta m1, m2;
    int w, off;
    {
        const PipeMeta m0 = meta_of(hb);
        m1 = meta_of(block_at(1));
        m2 = meta_of(block_at(2));
        int32_t g0[kPipeIdx];
        rows_of(m0, g0);
        rows_of(m1, g1);
        row_of(hb, m0, w, off);
        if (hb >= 0) issue(m0, g0, 0);
    }
    for (int64_t i = 0; hb >= 0; ++i) {
        const int64_t nxt = block_at(i + 1);
        if (nxt >= 0) issue(m1, g1, (int)((i + 1) & 1));
        else cp_async_commit();                          // an empty group keeps the count
        const PipeMeta m3 = meta_of(block_at(i + 3));
        int w1, off1;
        row_of(nxt, m1, w1, off1);
        // own-row streams of block i, in flight while its stage lands
        const int64_t r = hb * kHaloRows + lr;
        Cv<V, SPL> p = ld_ro<V, C, SPL>(a.psi, r, l), zz;
        if (a.z) {
            zz = ld<V, C, SPL>(a.z, r, l);
        } else {
#pragma unroll
            for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
        }
        const V d = __ldg(reinterpret_cast<const V *>(a.H.diag) + r);
        V gd = 0;
        if constexpr (sizeof(V) == 8) {
            if (a.uniform && !a.zero_diag) gd = gdiag_at(a, r);
        }
        cp_async_wait_group<1>();
        __syncthreads();
        rows_of(m2, g1);                                 // block i+2's rows, used next round
        const unsigned char *stg = sm + (int64_t)(i & 1) * ps.stage_bytes;
        const Cv<V, SPL> o = staged_row<V, C>(a, stg, ps, r, lr, l, w, off, p, zz, d, gd);
        st<V, C, SPL>(a.out, r, l, o);
        __syncthreads();                                 // stage i & 1 may be refilled now
        hb = nxt;
        m1 = m2;
        m2 = m3;
        w = w1;
        off = off1;
    }
    cp_async_wait_group<0>();
}

// ---- one-stage staged-gather term (TBPM_VARIANT_HALO | TBPM_VARIANT_STAGED) ----
// One block per 128-row halo block: its halo rows, packed positions and
// values copied into one shared-memory stage, then its rows computed from it
// (staged_row, the pipelined kernel's arithmetic).  Without the pipelined
// kernel's prefetch carried across blocks it fits 64 registers, so two
// blocks share an SM where the stage allows (~113 KB each): one block's
// copies, and the dependent loads that address them, overlap the other's
// gathers, with twice the warps in flight.
template <typename V, int C>
__global__ void __launch_bounds__(kHaloRows * C, 2) k_term_staged(TermArgs a, PipeShape ps)
{
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int SPL = 16 / (2 * sizeof(V));
    constexpr int NT = kHaloRows * C;
    constexpr int SPB = kHaloRows / kSliceRows;
    const int tid = threadIdx.x;
    const int l = tid % C, lr = tid / C;
    const int64_t hb = block_in_order(a);
    const int64_t h0 = __ldg(a.halo_ptr + hb);
    const int H = (int)(__ldg(a.halo_ptr + hb + 1) - h0);
    const int64_t e0 = __ldg(a.pslice + hb * SPB);
    const int E = (int)(__ldg(a.pslice + (hb + 1) * SPB) - e0);
    const unsigned char *xg = reinterpret_cast<const unsigned char *>(a.x);
    {
        int32_t g[kPipeIdx];                         // halo rows lr, lr + 128, ...
#pragma unroll
        for (int k = 0; k < kPipeIdx; ++k) {
            const int h = lr + k * kHaloRows;
            g[k] = h < H ? __ldg(a.halo_rows + h0 + h) : 0;
        }
#pragma unroll
        for (int k = 0; k < kPipeIdx; ++k) {
            const int h = lr + k * kHaloRows;
            if (h < H) cp_async16(sm + (h * C + l) * 16, xg + ((int64_t)g[k] * C + l) * 16);
        }
    }
    unsigned char *lc = sm + ps.halo_bytes;
    for (int idx = tid; idx < E / 8; idx += NT) cp_async16(lc + idx * 16, a.lcol + e0 + idx * 8);
    if (!a.uniform) {
        constexpr int per = 16 / sizeof(V);
        unsigned char *vs = lc + ps.lcol_bytes;
        for (int idx = tid; idx < E / per; idx += NT)
            cp_async16(vs + idx * 16, reinterpret_cast<const V *>(a.vpack) + e0 + idx * per);
    }
    cp_async_commit();
    // own-row streams and the row's entry count, in flight while the stage lands
    const int64_t r = hb * kHaloRows + lr;
    Cv<V, SPL> p = ld_ro<V, C, SPL>(a.psi, r, l), zz;
    if (a.z) {
        zz = ld<V, C, SPL>(a.z, r, l);
    } else {
#pragma unroll
        for (int j = 0; j < SPL; ++j) { zz.re[j] = 0; zz.im[j] = 0; }
    }
    const V d = __ldg(reinterpret_cast<const V *>(a.H.diag) + r);
    V gd = 0;
    if constexpr (sizeof(V) == 8) {
        if (a.uniform && !a.zero_diag) gd = gdiag_at(a, r);
    }
    const int64_t q = r / kSliceRows;
    const int w = a.fixed_width ? a.fixed_width
                                : (int)((__ldg(a.H.slice_ptr + q + 1) - __ldg(a.H.slice_ptr + q)) /
                                        kSliceRows);
    const int off = (int)(__ldg(a.pslice + q) - e0) + (lr % kSliceRows) * 4;
    cp_async_wait_group<0>();
    __syncthreads();
    const Cv<V, SPL> o = staged_row<V, C>(a, sm, ps, r, lr, l, w, off, p, zz, d, gd);
    st<V, C, SPL>(a.out, r, l, o);
}

int g_staged_configured[2][2] = {};   // dynamic shared bytes allowed, [fp32][C/4]

template <typename V, int C>
cudaError_t launch_staged_t(const TermArgs &a, cudaStream_t st)
{
    PipeShape ps;
    ps.halo_bytes = a.halo_max * C * 16;
    ps.lcol_bytes = (a.halo_ent_max * 2 + 15) / 16 * 16;
    ps.val_bytes = a.uniform ? 0 : a.halo_ent_max * (int)sizeof(V);
    ps.stage_bytes = ps.halo_bytes + ps.lcol_bytes + ps.val_bytes;
    ps.n_hb = (int)(a.n_rows / kHaloRows);
    const int smem = ps.stage_bytes;
    int &conf = g_staged_configured[sizeof(V) == 4][C / 4];
    if (smem > conf) {
        cudaError_t e = cudaFuncSetAttribute(k_term_staged<V, C>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        conf = smem;
    }
    k_term_staged<V, C><<<(unsigned)ps.n_hb, kHaloRows * C, smem, st>>>(a, ps);
    return cudaGetLastError();
}

cudaError_t dispatch_staged(const TermArgs &a, int fp32, int B, cudaStream_t st)
{
    if (fp32) return B == 4 ? launch_staged_t<float, 2>(a, st) : launch_staged_t<float, 4>(a, st);
    return B == 2 ? launch_staged_t<double, 2>(a, st) : launch_staged_t<double, 4>(a, st);
}

int g_pipe_configured[2][2] = {};   // dynamic shared bytes allowed, [fp32][C/4]

template <typename V, int C>
cudaError_t launch_pipe_t(const TermArgs &a, int num_sms, cudaStream_t st)
{
    PipeShape ps;
    ps.halo_bytes = a.halo_max * C * 16;
    ps.lcol_bytes = (a.halo_ent_max * 2 + 15) / 16 * 16;
    ps.val_bytes = a.uniform ? 0 : a.halo_ent_max * (int)sizeof(V);
    ps.stage_bytes = ps.halo_bytes + ps.lcol_bytes + ps.val_bytes;
    ps.n_hb = (int)(a.n_rows / kHaloRows);
    const int smem = 2 * ps.stage_bytes;
    int &conf = g_pipe_configured[sizeof(V) == 4][C / 4];
    if (smem > conf) {
        cudaError_t e = cudaFuncSetAttribute(k_term_halo_pipe<V, C>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        conf = smem;
    }
    // as many resident blocks per SM as shared memory and registers allow
    // (one for the twisted bilayer's ~200 KB stages, several for lattices
    // with short rows), the persistent grid a multiple of the SM count
    static int occ_cache[2][2] = {};
    static int occ_smem[2][2] = {};
    int &occ = occ_cache[sizeof(V) == 4][C / 4];
    if (occ_smem[sizeof(V) == 4][C / 4] != smem) {
        int nb = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_term_halo_pipe<V, C>,
                                                          kHaloRows * C, smem) != cudaSuccess)
            nb = 1;
        occ = std::max(1, nb);
        occ_smem[sizeof(V) == 4][C / 4] = smem;
    }
    const int grid = (int)std::min<int64_t>((int64_t)num_sms * occ, ps.n_hb);
    k_term_halo_pipe<V, C><<<grid, kHaloRows * C, smem, st>>>(a, ps);
    return cudaGetLastError();
}

cudaError_t dispatch_pipe(const TermArgs &a, int fp32, int B, cudaStream_t st)
{
    if (fp32) return B == 4 ? launch_pipe_t<float, 2>(a, a.num_sms, st)
                            : launch_pipe_t<float, 4>(a, a.num_sms, st);
    return B == 2 ? launch_pipe_t<double, 2>(a, a.num_sms, st)
                  : launch_pipe_t<double, 4>(a, a.num_sms, st);
}

// Interior terms: FP32 groups of 4, 8, 16 states, FP64 of 2, 4, 8; the
// closing term up to 8 (FP32) / 4 (FP64) states, whose reduction scratch
// for 128 rows stays within the static shared-memory limit.
template <bool FINAL>
cudaError_t dispatch_halo(const TermArgs &a, int fp32, int B, cudaStream_t st)
{
    if (!fp32) {
        switch (B) {
        case 2: return launch_halo_t<double, 1, 2, FINAL>(a, st);
        case 4: return launch_halo_t<double, 2, 2, FINAL>(a, st);
        case 8: if constexpr (!FINAL) return launch_halo_t<double, 4, 2, FINAL>(a, st); break;
        }
    } else {
        switch (B) {
        case 4: return launch_halo_t<float, 1, 4, FINAL>(a, st);
        case 8: return launch_halo_t<float, 2, 4, FINAL>(a, st);
        case 16: if constexpr (!FINAL) return launch_halo_t<float, 4, 4, FINAL>(a, st); break;
        }
    }
    return cudaErrorInvalidValue;
}

// Sum of the chunk partials of each sample, spread over kReduceSplit blocks
// per sample (GB300's FP64 adder throughput per SM is small, so one block
// per sample would take tens of microseconds): block (s, j) sums chunks
// j, j + kReduceSplit, ... of sample s in order; the last of the sample's
// blocks (ticket after a fence) adds the kReduceSplit sums in order and
// writes the correlation entry, the squared norm, the drift checks and (FP32)
// the scale of the next step's starting state.
constexpr int kReduceSplit = 64;

__global__ void __launch_bounds__(64) k_reduce(ReduceArgs a)
{
    __shared__ int last;
    const int s = blockIdx.x, j = blockIdx.y;
    const int B3 = a.B * 3;
    const int t = threadIdx.x;
    const int64_t c0 = a.sample_chunk_off[s], c1 = a.sample_chunk_off[s + 1];
    double *mine = a.partial2 + ((int64_t)s * kReduceSplit + j) * B3;
    if (t < B3) {
        double acc = 0.0;
#pragma unroll 4
        for (int64_t c = c0 + j; c < c1; c += kReduceSplit) acc += a.partial[c * B3 + t];
        mine[t] = acc;
        __threadfence();
    }
    __syncthreads();
    if (t == 0) last = (atomicAdd(a.sample_ticket + s, 1u) == kReduceSplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double v[48];
    if (t < B3) {
        double acc = 0.0;
        const double *base = a.partial2 + (int64_t)s * kReduceSplit * B3;
        for (int k = 0; k < kReduceSplit; ++k) acc += __ldcg(base + (int64_t)k * B3 + t);
        v[t] = acc;
    }
    __syncthreads();
    const int step = a.step[s];
    if (t < a.B) {
        const double re = v[t * 3], im = v[t * 3 + 1], nn = v[t * 3 + 2];
        const int state = a.group_state0 + t;
        const int64_t idx = ((int64_t)s * a.n_states + state) * (a.n_steps + 1) + step;
        a.corr[idx] = make_double2(re, im);
        a.norms[idx] = nn;
        // drift relative to the squared norm at t = 0 (1 for normalised states;
        // the AC-conductivity states are not normalised)
        const int64_t ridx = (int64_t)s * a.n_states + state;
        if (a.set_ref) a.norm_ref[ridx] = nn;
        const double ref = a.set_ref ? nn : a.norm_ref[ridx];
        const double drift = ref > 0.0 ? fabs(nn / ref - 1.0) : nn;
        if (!(nn == nn) || !(re == re) || !(im == im) || nn - nn != 0.0) {
            atomicOr(a.error_flags, 2);
        } else if (drift > a.hard_bound) {
            atomicOr(a.error_flags, 1);
        }
        if (a.scale) {
            double sc = 1.0;
            if (drift > a.renorm_bound && nn > 0.0 && ref > 0.0 && nn - nn == 0.0) {
                sc = sqrt(ref / nn);
                atomicAdd(a.renorm_count, 1ull);
            }
            a.scale[(int64_t)s * a.B + t] = sc;
            if (a.scale_f) a.scale_f[(int64_t)s * a.B + t] = (float)sc;
        }
    }
    __syncthreads();
    if (t == 0) {
        a.step[s] = step + 1;
        a.sample_ticket[s] = 0;          // ready for the next launch
    }
}

template <typename V, int SPL> struct StoreC;
template <> struct StoreC<double, 1> {
    __device__ static void put(void *psi, int64_t idx, double re, double im)
    {
        reinterpret_cast<double2 *>(psi)[idx] = make_double2(re, im);
    }
    __device__ static double2 get(const void *psi, int64_t idx)
    {
        return reinterpret_cast<const double2 *>(psi)[idx];
    }
};
template <> struct StoreC<float, 1> {
    __device__ static void put(void *psi, int64_t idx, double re, double im)
    {
        reinterpret_cast<float2 *>(psi)[idx] = make_float2((float)re, (float)im);
    }
    __device__ static double2 get(const void *psi, int64_t idx)
    {
        float2 v = reinterpret_cast<const float2 *>(psi)[idx];
        return make_double2(v.x, v.y);
    }
};

// psi0_u = exp(i theta_u) / sqrt(N_k) in caller order (complex128).
__global__ void k_phase_user(const double *theta, int64_t n_orb, int n_states,
                             const double *inv_sqrt_n, const int32_t *orb_sample,
                             double2 *psi_user)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    const double a = inv_sqrt_n[orb_sample[u]];
    for (int p = 0; p < n_states; ++p) {
        double sn, cs;
        sincos(theta[(int64_t)p * n_orb + u], &sn, &cs);
        psi_user[(int64_t)p * n_orb + u] = make_double2(a * cs, a * sn);
    }
}

template <typename V>
__global__ void k_set_states(const double2 *src, int64_t n_orb, const int32_t *user_to_row,
                             int g0, int B, void *psi)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    const int64_t r = user_to_row[u];
    for (int b = 0; b < B; ++b) {
        double2 v = src[(int64_t)(g0 + b) * n_orb + u];
        StoreC<V, 1>::put(psi, r * B + b, v.x, v.y);
    }
}

template <typename V>
__global__ void k_get_states(const void *psi, int64_t n_orb, const int32_t *user_to_row,
                             int g0, int B, double2 *dst)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    const int64_t r = user_to_row[u];
    for (int b = 0; b < B; ++b)
        dst[(int64_t)(g0 + b) * n_orb + u] = StoreC<V, 1>::get(psi, r * B + b);
}

// State average of the correlation (Sec. 2.4: the mean over the random
// states in Eq. dos_tbpm): avg[k][n] = (sum_p corr[k][p][n]) / S, the states
// added in order.
__global__ void k_corr_mean(const double2 *corr, int n_samples, int S, int n1, double2 *avg)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_samples * n1) return;
    const int64_t k = i / n1, n = i % n1;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < S; ++p) {
        const double2 v = corr[(k * S + p) * n1 + n];
        re += v.x;
        im += v.y;
    }
    avg[i] = make_double2(re / S, im / S);
}

// Its adjoint: each state's C_n gets dL/dC-bar_n / S.
__global__ void k_corr_mean_adjoint(const double2 *gavg, int n_samples, int S, int n1,
                                    double2 *g)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_samples * S * n1) return;
    const int64_t n = i % n1, k = i / ((int64_t)S * n1);
    const double2 v = gavg[k * n1 + n];
    g[i] = make_double2(v.x / S, v.y / S);
}

template <typename V, int L, int SPL, bool CX, int RS = 1>
cudaError_t launch_term_t(const TermArgs &a, int threads, cudaStream_t st)
{
    const int64_t n_threads = a.n_rows * L * RS;
    const unsigned blocks = (unsigned)((n_threads + threads - 1) / threads);
    k_term<V, L, SPL, CX, RS><<<blocks, threads, 0, st>>>(a);
    return cudaGetLastError();
}

// The register-pipelined kernel: a persistent grid of the SMs times the
// blocks that fit on one, at most one thread per lane-row.
template <typename V, int L, int SPL>
cudaError_t launch_term_pf_t(const TermArgs &a, int threads, cudaStream_t st)
{
    static int occ[4] = {0, 0, 0, 0};            // resident blocks per SM by threads 64 .. 512
    const int ti = threads <= 64 ? 0 : threads <= 128 ? 1 : threads <= 256 ? 2 : 3;
    if (!occ[ti]) {
        int nb = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_term_pf<V, L, SPL>, threads, 0) !=
            cudaSuccess)
            nb = 1;
        occ[ti] = std::max(1, nb);
    }
    const int64_t n_threads = a.n_rows * L;
    const int64_t want = (n_threads + threads - 1) / threads;
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, a.num_sms) * occ[ti], want));
    k_term_pf<V, L, SPL><<<blocks, threads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch_pf(const TermArgs &a, int fp32, int B, int threads, cudaStream_t st)
{
    if (!fp32) {
        if (a.variant & kVariantWide) {
            switch (B) {
            case 2: return launch_term_pf_t<double, 1, 2>(a, threads, st);
            case 4: return launch_term_pf_t<double, 2, 2>(a, threads, st);
            case 8: return launch_term_pf_t<double, 4, 2>(a, threads, st);
            }
        }
        switch (B) {
        case 1: return launch_term_pf_t<double, 1, 1>(a, threads, st);
        case 2: return launch_term_pf_t<double, 2, 1>(a, threads, st);
        case 4: return launch_term_pf_t<double, 4, 1>(a, threads, st);
        case 8: return launch_term_pf_t<double, 8, 1>(a, threads, st);
        }
        return cudaErrorInvalidValue;
    }
    if (a.variant & kVariantWide) {
        switch (B) {
        case 4: return launch_term_pf_t<float, 1, 4>(a, threads, st);
        case 8: return launch_term_pf_t<float, 2, 4>(a, threads, st);
        case 16: return launch_term_pf_t<float, 4, 4>(a, threads, st);
        }
    }
    switch (B) {
    case 1: return launch_term_pf_t<float, 1, 1>(a, threads, st);
    case 2: return launch_term_pf_t<float, 1, 2>(a, threads, st);
    case 4: return launch_term_pf_t<float, 2, 2>(a, threads, st);
    case 8: return launch_term_pf_t<float, 4, 2>(a, threads, st);
    case 16: return launch_term_pf_t<float, 8, 2>(a, threads, st);
    }
    return cudaErrorInvalidValue;
}

// Row-split launch (real values, interior terms): RS from the variant bits.
template <typename V, int L, int SPL>
cudaError_t launch_term_split(const TermArgs &a, int threads, cudaStream_t st)
{
    if (a.variant & kVariantSplit4) return launch_term_t<V, L, SPL, false, 4>(a, threads, st);
    return launch_term_t<V, L, SPL, false, 2>(a, threads, st);
}

template <typename V, int L, int SPL, bool CX>
cudaError_t launch_final_t(const TermArgs &a, int threads, bool compute, cudaStream_t st)
{
    (void)threads;   // the closing term has its own block size
    if constexpr (sizeof(V) == 4 && !CX) {
        if (!compute) {           // FP32 reduction-only pass: four rows a thread
            constexpr int RPT = 4;
            const unsigned rblocks = (unsigned)(a.n_rows * L / (kFinalThreads * RPT));
            k_final_sums<L, SPL, RPT><<<rblocks, kFinalThreads, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    const unsigned blocks = (unsigned)(a.n_rows * L / kFinalThreads);
    if (compute)
        k_final<V, L, SPL, true, CX><<<blocks, kFinalThreads, 0, st>>>(a);
    else
        k_final<V, L, SPL, false, CX><<<blocks, kFinalThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <bool FINAL, bool CX>
cudaError_t dispatch_cx(const TermArgs &a, int fp32, int B, int threads, bool compute,
                        cudaStream_t st)
{
    if (!FINAL && !CX && (a.variant & (kVariantSplit2 | kVariantSplit4))) {
        if (a.variant & kVariantWide) {
            if (!fp32) {
                switch (B) {
                case 2: return launch_term_split<double, 1, 2>(a, threads, st);
                case 4: return launch_term_split<double, 2, 2>(a, threads, st);
                case 8: return launch_term_split<double, 4, 2>(a, threads, st);
                }
            } else {
                switch (B) {
                case 4: return launch_term_split<float, 1, 4>(a, threads, st);
                case 8: return launch_term_split<float, 2, 4>(a, threads, st);
                case 16: return launch_term_split<float, 4, 4>(a, threads, st);
                }
            }
        }
        if (!fp32) {
            switch (B) {
            case 1: return launch_term_split<double, 1, 1>(a, threads, st);
            case 2: return launch_term_split<double, 2, 1>(a, threads, st);
            case 4: return launch_term_split<double, 4, 1>(a, threads, st);
            case 8: return launch_term_split<double, 8, 1>(a, threads, st);
            }
        } else {
            switch (B) {
            case 1: return launch_term_split<float, 1, 1>(a, threads, st);
            case 2: return launch_term_split<float, 1, 2>(a, threads, st);
            case 4: return launch_term_split<float, 2, 2>(a, threads, st);
            case 8: return launch_term_split<float, 4, 2>(a, threads, st);
            case 16: return launch_term_split<float, 8, 2>(a, threads, st);
            }
        }
    }
#define TBPM_CASE(V, L, SPL)                                                  \
    return FINAL ? launch_final_t<V, L, SPL, CX>(a, threads, compute, st)    \
                 : launch_term_t<V, L, SPL, CX>(a, threads, st)
    if constexpr (!CX) if (a.variant & kVariantWide) {
        // one thread per row and 32-byte lanes: fewer lanes share the index loads
        if (!fp32) {
            switch (B) {
            case 2: TBPM_CASE(double, 1, 2);
            case 4: TBPM_CASE(double, 2, 2);
            case 8: TBPM_CASE(double, 4, 2);
            }
        } else {
            switch (B) {
            case 4: TBPM_CASE(float, 1, 4);
            case 8: TBPM_CASE(float, 2, 4);
            case 16: TBPM_CASE(float, 4, 4);
            }
        }
    }
    if (!fp32) {
        switch (B) {
        case 1: TBPM_CASE(double, 1, 1);
        case 2: TBPM_CASE(double, 2, 1);
        case 4: TBPM_CASE(double, 4, 1);
        case 8: TBPM_CASE(double, 8, 1);
        }
    } else {
        switch (B) {
        case 1: TBPM_CASE(float, 1, 1);
        case 2: TBPM_CASE(float, 1, 2);
        case 4: TBPM_CASE(float, 2, 2);
        case 8: TBPM_CASE(float, 4, 2);
        case 16: TBPM_CASE(float, 8, 2);
        }
    }
#undef TBPM_CASE
    return cudaErrorInvalidValue;
}

template <bool FINAL>
cudaError_t dispatch(const TermArgs &a, int fp32, int B, int threads, bool compute,
                     cudaStream_t st)
{
    return a.cplx ? dispatch_cx<FINAL, true>(a, fp32, B, threads, compute, st)
                  : dispatch_cx<FINAL, false>(a, fp32, B, threads, compute, st);
}

}  // namespace

int pipe_smem_bytes(int fp32, int B, int halo_max, int ent_max, int uniform)
{
    const int C = B * (fp32 ? 8 : 16) / 16;
    return 2 * (halo_max * C * 16 + (ent_max * 2 + 15) / 16 * 16 +
                (uniform ? 0 : ent_max * (fp32 ? 4 : 8)));
}

bool pipe_launchable(int fp32, int B, int halo_max, int ent_max, int uniform)
{
    const bool shape = fp32 ? (B == 4 || B == 8) : (B == 2 || B == 4);
    return shape && pipe_smem_bytes(fp32, B, halo_max, ent_max, uniform) <= kPipeSmemMax;
}

bool staged_launchable(int fp32, int B, int halo_max, int ent_max, int uniform)
{
    const bool shape = fp32 ? (B == 4 || B == 8) : (B == 2 || B == 4);
    return shape && pipe_smem_bytes(fp32, B, halo_max, ent_max, uniform) / 2 <= kPipeSmemMax;
}

bool halo_launchable(int fp32, int B, bool final_term, int halo_max)
{
    // the shared copy (halo rows x B states) must leave room for the
    // reduction scratch and a second resident block
    if ((int64_t)halo_max * B * (fp32 ? 8 : 16) > kHaloSmemMax) return false;
    if (final_term) return fp32 ? (B == 4 || B == 8) : (B == 2 || B == 4);
    return fp32 ? (B == 4 || B == 8 || B == 16) : (B == 2 || B == 4 || B == 8);
}

cudaError_t launch_term(const TermArgs &a, int fp32, int B, int threads, cudaStream_t st)
{
    // the register-pipelined kernel: real values, unsplit rows
    if ((a.variant & kVariantPrefetch) && !a.cplx && !(a.variant & kVariantHalo) &&
        !(a.variant & (kVariantSplit2 | kVariantSplit4)))
        return dispatch_pf(a, fp32, B, threads, st);
    // the one-stage staged kernel, like the pipelined one, keeps rows unsplit
    if ((a.variant & kVariantHalo) && (a.variant & kVariantStaged) && a.lcol && !a.cplx &&
        (a.vpack || a.uniform) && !(a.variant & (kVariantSplit2 | kVariantSplit4)) &&
        staged_launchable(fp32, B, a.halo_max, a.halo_ent_max, a.uniform))
        return dispatch_staged(a, fp32, B, st);
    // the pipelined kernel does not split rows: with a row split requested,
    // the plain split kernel below keeps the requested summation order
    if ((a.variant & kVariantHalo) && (a.variant & kVariantPipe) && a.lcol && !a.cplx &&
        (a.vpack || a.uniform) && !(a.variant & (kVariantSplit2 | kVariantSplit4)) &&
        pipe_launchable(fp32, B, a.halo_max, a.halo_ent_max, a.uniform))
        return dispatch_pipe(a, fp32, B, st);
    // the one-stage staged-gather kernel does not split rows: with a row
    // split requested, the plain split kernel keeps the requested order
    if ((a.variant & kVariantHalo) && a.lcol && !a.cplx &&
        !(a.variant & (kVariantSplit2 | kVariantSplit4)) &&
        halo_launchable(fp32, B, false, a.halo_max))
        return dispatch_halo<false>(a, fp32, B, st);
    return dispatch<false>(a, fp32, B, threads, true, st);
}

cudaError_t launch_final(const TermArgs &a, int fp32, int B, int threads, cudaStream_t st,
                         int *n_launch)
{
    if (n_launch) *n_launch = 1;
    // the register-pipelined term writes `out`, then the closing reduction
    // reads it (states as the plain closing term's, sums in its order)
    if ((a.variant & kVariantPrefetch) && !a.cplx && !(a.variant & kVariantHalo) && a.H.col) {
        cudaError_t e = dispatch_pf(a, fp32, B, threads, st);
        if (e != cudaSuccess) return e;
        TermArgs r = a;
        r.H.col = nullptr;
        if (n_launch) *n_launch = 2;      // the term, then the reduction pass
        return dispatch<true>(r, fp32, B, threads, false, st);
    }
    if ((a.variant & kVariantHalo) && (a.variant & kVariantStaged) && a.lcol && !a.cplx &&
        (a.vpack || a.uniform) && a.H.col &&
        staged_launchable(fp32, B, a.halo_max, a.halo_ent_max, a.uniform)) {
        cudaError_t e = dispatch_staged(a, fp32, B, st);   // then the closing reduction
        if (e != cudaSuccess) return e;
        TermArgs r = a;
        r.H.col = nullptr;
        if (n_launch) *n_launch = 2;      // the term, then the reduction pass
        return dispatch<true>(r, fp32, B, threads, false, st);
    }
    if ((a.variant & kVariantHalo) && (a.variant & kVariantPipe) && a.lcol && !a.cplx &&
        (a.vpack || a.uniform) && a.H.col &&
        pipe_launchable(fp32, B, a.halo_max, a.halo_ent_max, a.uniform)) {
        // the pipelined term writes `out`, then the closing reduction reads it;
        // unsplit rows, as the plain closing term (the states then match the
        // per-term kernels' bit for bit with or without the row split)
        cudaError_t e = dispatch_pipe(a, fp32, B, st);
        if (e != cudaSuccess) return e;
        TermArgs r = a;
        r.H.col = nullptr;
        if (n_launch) *n_launch = 2;      // the term, then the reduction pass
        return dispatch<true>(r, fp32, B, threads, false, st);
    }
    if ((a.variant & kVariantHalo) && a.lcol && !a.cplx && a.H.col &&
        halo_launchable(fp32, B, true, a.halo_max))
        return dispatch_halo<true>(a, fp32, B, st);
    return dispatch<true>(a, fp32, B, threads, a.H.col != nullptr, st);
}

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st)
{
    k_reduce<<<dim3(a.n_samples, kReduceSplit), 64, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t kernel_binary_version(int *version)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_corr_mean);
    if (e == cudaSuccess) *version = fa.binaryVersion;
    return e;
}

cudaError_t launch_corr_mean(const double2 *corr, int n_samples, int S, int n1, double2 *avg,
                             cudaStream_t st)
{
    const int64_t n = (int64_t)n_samples * n1;
    k_corr_mean<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(corr, n_samples, S, n1, avg);
    return cudaGetLastError();
}

cudaError_t launch_corr_mean_adjoint(const double2 *gavg, int n_samples, int S, int n1,
                                     double2 *g, cudaStream_t st)
{
    const int64_t n = (int64_t)n_samples * S * n1;
    k_corr_mean_adjoint<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gavg, n_samples, S, n1, g);
    return cudaGetLastError();
}

cudaError_t launch_phase_user(const double *theta, int64_t n_orb, int n_states,
                              const double *inv_sqrt_n, const int32_t *orb_sample,
                              double2 *psi_user, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_orb + 255) / 256);
    k_phase_user<<<blocks, 256, 0, st>>>(theta, n_orb, n_states, inv_sqrt_n, orb_sample,
                                         psi_user);
    return cudaGetLastError();
}

cudaError_t launch_set_states(const double2 *psi_user, int64_t n_orb, int n_states,
                              const int32_t *user_to_row, int g0, int B, int fp32, void *psi,
                              cudaStream_t st)
{
    (void)n_states;
    const unsigned blocks = (unsigned)((n_orb + 255) / 256);
    if (fp32)
        k_set_states<float><<<blocks, 256, 0, st>>>(psi_user, n_orb, user_to_row, g0, B, psi);
    else
        k_set_states<double><<<blocks, 256, 0, st>>>(psi_user, n_orb, user_to_row, g0, B, psi);
    return cudaGetLastError();
}

cudaError_t launch_get_states(const void *psi, int64_t n_orb, int n_states,
                              const int32_t *user_to_row, int g0, int B, int fp32,
                              double2 *out_user, cudaStream_t st)
{
    (void)n_states;
    const unsigned blocks = (unsigned)((n_orb + 255) / 256);
    if (fp32)
        k_get_states<float><<<blocks, 256, 0, st>>>(psi, n_orb, user_to_row, g0, B, out_user);
    else
        k_get_states<double><<<blocks, 256, 0, st>>>(psi, n_orb, user_to_row, g0, B, out_user);
    return cudaGetLastError();
}

}  // namespace tbpm
