// a1: bond list -> sliced-ELLPACK H~ = H / s on the GPU.
//
// The Hamiltonian of Sec. 2.1 (Eq. ham_mat_finite, hopping convention of
// Sec. 4.1) has H_ij = t and H_ji = conj(t) = t (real hoppings) for a bond
// (i, j, t) and H_ii = eps_i.  The off-diagonal part is stored as sliced
// ELLPACK with 32-row slices: slice q holds width_q entries per row, entry k
// of local row r at slice_ptr[q] + 32 k + r.  Rows shorter than the slice
// width are padded with (col = own row, value 0), so every load stays in
// bounds and needs no predicate beyond the slice width.  The diagonal is a
// separate dense array.  Each sample occupies a block of rows padded to a
// multiple of kChunkRows; padding rows are empty.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

#define CK(call)                                                              \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            msg = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return e_ == cudaErrorMemoryAllocation ? TBPM_E_OOM : TBPM_E_CUDA; \
        }                                                                     \
    } while (0)

__device__ __forceinline__ int find_sample(const int64_t *off, int n_samples, int64_t u)
{
    int lo = 0, hi = n_samples - 1;
    while (lo < hi) {                       // last k with off[k] <= u
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_map_orbitals(int64_t n_orb, int n_samples, const int64_t *sample_off,
                               const int64_t *row_off, const int32_t *perm,
                               int32_t *user_to_row, int32_t *orb_sample)
{
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    int s = find_sample(sample_off, n_samples, u);
    int64_t local = perm ? (int64_t)perm[u] : u - sample_off[s];
    user_to_row[u] = (int32_t)(row_off[s] + local);
    orb_sample[u] = s;
}

// error bits: 1 index out of range, 2 self bond, 4 bond across samples,
// 8 non-finite value
__global__ void k_count(int64_t n_hop, int64_t n_orb, const int64_t *hi, const int64_t *hj,
                        const double *hv, int vw, const int32_t *user_to_row,
                        const int32_t *orb_sample, int32_t *deg, int *err)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_hop) return;
    int64_t i = hi[b], j = hj[b];
    if (i < 0 || j < 0 || i >= n_orb || j >= n_orb) { atomicOr(err, 1); return; }
    if (i == j) { atomicOr(err, 2); return; }
    if (orb_sample[i] != orb_sample[j]) { atomicOr(err, 4); return; }
    for (int q = 0; q < vw; ++q) {
        double v = hv[b * vw + q];
        if (!(v == v) || v - v != 0.0) { atomicOr(err, 8); return; }
    }
    atomicAdd(&deg[user_to_row[i]], 1);
    atomicAdd(&deg[user_to_row[j]], 1);
}

// slice_ptr[q] = 32 q w for the fixed-width layout.
__global__ void k_fixed_slices(int64_t n_slices, int w, int64_t *slice_ptr)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q <= n_slices) slice_ptr[q] = q * kSliceRows * (int64_t)w;
}

__global__ void k_slice_width(int64_t n_slices, const int32_t *deg, int64_t *entries,
                              int *max_width)
{
    int64_t q = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (q >= n_slices) return;
    int d = deg[q * kSliceRows + lane];
    for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (lane == 0) {
        entries[q] = (int64_t)d * kSliceRows;
        atomicMax(max_width, d);
    }
}

// ---- exclusive scan of int64 (three phases, recursive over block sums) ----
constexpr int kScanBlock = 1024;

__global__ void k_scan_block(const int64_t *in, int64_t *out, int64_t n, int64_t *block_sums)
{
    __shared__ int64_t warp_tot[32];
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t before = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    if (i < n) out[i] = before;
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = before + v;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *block_off)
{
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}

// out[0 .. n] = exclusive scan of in[0 .. n-1]; out[n] = total.
int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st,
                   std::string &msg)
{
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int64_t *sums = nullptr, *sums_scan = nullptr;
    CK(cudaMalloc(&sums, (nb + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&sums_scan, (nb + 1) * sizeof(int64_t)));
    k_scan_block<<<(unsigned)nb, kScanBlock, 0, st>>>(in, out, n, sums);
    CK(cudaGetLastError());
    int rc = TBPM_OK;
    if (nb > 1) {
        rc = scan_exclusive(sums, sums_scan, nb, st, msg);
        if (rc == TBPM_OK) {
            k_scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(out, n, sums_scan);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(out + n, sums_scan + nb, sizeof(int64_t),
                               cudaMemcpyDeviceToDevice, st));
        }
    } else {
        CK(cudaMemcpyAsync(out + n, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    cudaFree(sums);
    cudaFree(sums_scan);
    return rc;
}

// Values are VW numbers of type T (double, or float when only the FP32 copy
// is kept) per entry: 1 (real hoppings) or 2 (complex, re/im).
template <int VW, typename T>
__global__ void k_pad_fill(int64_t n_rows, const int64_t *slice_ptr, int32_t *col,
                           T *val)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t q = r / kSliceRows;
    int lr = (int)(r % kSliceRows);
    int64_t base = slice_ptr[q];
    int w = (int)((slice_ptr[q + 1] - base) / kSliceRows);
    for (int k = 0; k < w; ++k) {
        col[base + (int64_t)k * kSliceRows + lr] = (int32_t)r;
        for (int q = 0; q < VW; ++q) val[(base + (int64_t)k * kSliceRows + lr) * VW + q] = (T)0;
    }
}

template <int VW, typename T>
__global__ void k_fill(int64_t n_hop, const int64_t *hi, const int64_t *hj, const double *hv,
                       double inv_s, const int32_t *user_to_row, const int64_t *slice_ptr,
                       int32_t *fill, int32_t *col, T *val)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_hop) return;
    int32_t ri = user_to_row[hi[b]], rj = user_to_row[hj[b]];
    int pi = atomicAdd(&fill[ri], 1);
    int64_t ei = slice_ptr[ri / kSliceRows] + (int64_t)pi * kSliceRows + ri % kSliceRows;
    col[ei] = rj;
    int pj = atomicAdd(&fill[rj], 1);
    int64_t ej = slice_ptr[rj / kSliceRows] + (int64_t)pj * kSliceRows + rj % kSliceRows;
    col[ej] = ri;
    // H_ij = t, H_ji = conj(t), scaled in FP64 and rounded once to T
    val[ei * VW] = (T)(hv[b * VW] * inv_s);
    val[ej * VW] = (T)(hv[b * VW] * inv_s);
    if (VW == 2) {
        val[ei * VW + 1] = (T)(hv[b * VW + 1] * inv_s);
        val[ej * VW + 1] = (T)(-(hv[b * VW + 1] * inv_s));
    }
}

__global__ void k_diag(int64_t n_orb, const double *onsite, double inv_s,
                       const int32_t *user_to_row, double *diag)
{
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    diag[user_to_row[u]] = onsite ? onsite[u] * inv_s : 0.0;
}

// Per row: insertion sort of the filled entries by (col, value) so the
// product's summation order is independent of the fill order; then the
// Gershgorin row bound |d_r| + sum |H~_rc|, max-reduced as the bit pattern of
// a non-negative double (which orders like an unsigned integer).
template <int VW, typename T>
__global__ void k_sort_rows(int64_t n_rows, const int64_t *slice_ptr, const int32_t *deg,
                            const double *diag, int32_t *col, T *val,
                            unsigned long long *gersh_bits, unsigned long long *band)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    int64_t base = slice_ptr[r / kSliceRows] + r % kSliceRows;
    int d = deg[r];
    auto E = [&](int k) { return base + (int64_t)k * kSliceRows; };
    for (int a = 1; a < d; ++a) {
        int32_t c = col[E(a)];
        T v0 = val[E(a) * VW], v1 = VW == 2 ? val[E(a) * VW + 1] : (T)0;
        int b = a - 1;
        while (b >= 0) {
            int32_t cb = col[E(b)];
            T w0 = val[E(b) * VW], w1 = VW == 2 ? val[E(b) * VW + 1] : (T)0;
            if (cb < c || (cb == c && (w0 < v0 || (w0 == v0 && w1 <= v1)))) break;
            col[E(b + 1)] = cb;
            val[E(b + 1) * VW] = w0;
            if (VW == 2) val[E(b + 1) * VW + 1] = w1;
            --b;
        }
        col[E(b + 1)] = c;
        val[E(b + 1) * VW] = v0;
        if (VW == 2) val[E(b + 1) * VW + 1] = v1;
    }
    double g = fabs(diag[r]);
    long long bw = 0;
    for (int a = 0; a < d; ++a) {
        g += VW == 2 ? hypot((double)val[E(a) * VW], (double)val[E(a) * VW + 1])
                     : fabs((double)val[E(a) * VW]);
        const long long dist = (long long)col[base + (int64_t)a * kSliceRows] - (long long)r;
        bw = max(bw, dist < 0 ? -dist : dist);
    }
    atomicMax(gersh_bits, (unsigned long long)__double_as_longlong(g));
    if (bw > 0) atomicMax(band, (unsigned long long)bw);
}

__global__ void k_bond_rows(int64_t n_hop, const int64_t *hi, const int64_t *hj,
                            const int32_t *user_to_row, int32_t *rows)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n_hop) return;
    rows[2 * b] = user_to_row[hi[b]];
    rows[2 * b + 1] = user_to_row[hj[b]];
}

// Clears *zero unless every onsite energy is zero.
// (one atomic per block: a disordered diagonal would otherwise send every
// thread's atomic to the same word)
__global__ void k_zero_onsite(int64_t n, const double *onsite, int *zero)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (__syncthreads_or(i < n && onsite[i] != 0.0) && threadIdx.x == 0) atomicAnd(zero, 0);
}

// Clears *same unless every hopping equals the first one (after scaling).
__global__ void k_uniform(int64_t n_hop, const double *hv, double inv_s, int *same)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool diff = b < n_hop && hv[b] * inv_s != hv[0] * inv_s;
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicAnd(same, 0);
}

__global__ void k_to_f32(int64_t n, const double *src, float *dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- halo lists of the staged-gather term kernel --------------------------
// For each block of kHaloRows consecutive rows: the block's own rows (halo
// positions 0 .. kHaloRows-1, in order), then the distinct other rows its
// stored entries reference, ascending; and per stored entry the 16-bit
// position of its column in that list.  Distinct columns are found with an
// open-addressing set in shared memory (bounded probes) and sorted by a
// bitonic sort, so the lists do not depend on thread timing.
//
// The positions (and, for the pipelined kernel, a copy of the values) are
// stored "packed": within a slice, the entries of a row come in groups of
// four adjacent numbers, entry k of local row lr at
//   pslice[q] + (k / 4) * 128 + lr * 4 + k % 4,
// with each slice's width rounded up to a multiple of four (the extra slots
// point at the own row with value 0).  A thread then reads four positions
// in one 8-byte load and four FP32 values in one 16-byte load.
constexpr int kHaloHash = 4096;          // set slots per block (load <= 1/2)
constexpr int kHaloThreads = 256;

__device__ __forceinline__ unsigned halo_slot(int32_t c)
{
    return ((unsigned)c * 2654435761u) >> (32 - 12);      // 12 bits: kHaloHash slots
}

// Collect the distinct external columns of block hb into ext[0 .. *n_ext),
// sorted when `sort` (the count pass needs only their number).  Sets
// *overflow when more than kHaloMaxExt are met.
__device__ void halo_collect(int64_t hb, const int64_t *slice_ptr, const int32_t *col,
                             int32_t *keys, int32_t *ext, int *n_ext, int *overflow, bool sort)
{
    const int tid = threadIdx.x;
    for (int k = tid; k < kHaloHash; k += kHaloThreads) keys[k] = -1;
    if (tid == 0) { *n_ext = 0; *overflow = 0; }
    __syncthreads();
    const int64_t r0 = hb * kHaloRows;
    const int64_t q0 = r0 / kSliceRows, q1 = q0 + kHaloRows / kSliceRows;
    const int64_t e0 = slice_ptr[q0], e1 = slice_ptr[q1];
    for (int64_t e = e0 + tid; e < e1; e += kHaloThreads) {
        const int32_t c = col[e];
        if (c >= r0 && c < r0 + kHaloRows) continue;       // own rows come first
        unsigned h = halo_slot(c);
        for (int probe = 0; probe < kHaloHash; ++probe) {  // bounded: the set has kHaloHash slots
            const int32_t prev = atomicCAS(&keys[h], -1, c);
            if (prev == -1) {
                const int at = atomicAdd(n_ext, 1);
                if (at < kHaloMaxExt) ext[at] = c; else *overflow = 1;
                break;
            }
            if (prev == c) break;
            h = (h + 1) & (kHaloHash - 1);
            if (probe == kHaloHash - 1) *overflow = 1;
        }
    }
    __syncthreads();
    if (!sort) return;
    const int n = min(*n_ext, kHaloMaxExt);
    int n2 = 32;
    while (n2 < n) n2 <<= 1;
    for (int k = n + tid; k < n2; k += kHaloThreads) ext[k] = INT32_MAX;
    __syncthreads();
    // bitonic sort of ext[0 .. n2)
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = tid; k < n2 / 2; k += kHaloThreads) {
                const int lo = 2 * k - (k & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const int32_t x = ext[lo], y = ext[hi];
                if ((x > y) == up) { ext[lo] = y; ext[hi] = x; }
            }
            __syncthreads();
        }
    }
}

// Packed entries of each slice: 32 x (width rounded up to 4).
__global__ void k_packed_slice_entries(int64_t n_slices, const int64_t *slice_ptr, int64_t *ent)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_slices) return;
    const int64_t w = (slice_ptr[q + 1] - slice_ptr[q]) / kSliceRows;
    ent[q] = (w + 3) / 4 * 4 * kSliceRows;
}

// Pass 1: halo size of every block (kHaloRows + distinct external rows), or
// -1 when the block overflows the set.
__global__ void __launch_bounds__(kHaloThreads) k_halo_count(const int64_t *slice_ptr,
                                                             const int32_t *col, int64_t *size)
{
    __shared__ int32_t keys[kHaloHash];
    __shared__ int32_t ext[kHaloMaxExt];
    __shared__ int n_ext, overflow;
    halo_collect(blockIdx.x, slice_ptr, col, keys, ext, &n_ext, &overflow, false);
    if (threadIdx.x == 0) size[blockIdx.x] = overflow ? -1 : (int64_t)kHaloRows + n_ext;
}

// Bank-parity colouring of the external halo slots.  The pipelined term
// kernel reads a neighbour's lanes with the row's C threads, so one
// quarter-warp reads the neighbours of rows 2m and 2m+1 of a slice at the
// same entry k; with 64-byte rows the two reads fall on the same half of
// the shared-memory banks -- one extra wavefront -- when their slots have
// equal parity (reads of the same slot are a broadcast).  The slots of a
// block's external rows are a free permutation, so they are 2-coloured by
// slot parity to cut the pair graph (a node per halo row, an edge per pair
// and entry): greedy local moves in index order for a few passes, the
// colour counts kept within a few of the slot counts, then restored by the
// least harmful moves.  Own rows keep slots 0 .. kHaloRows-1.  Integer
// gains and a fixed order: the layout depends on the matrix alone.
constexpr int kColorMaxEnt = 12288;      // packed entries of the blocks that are coloured
constexpr int kColorPasses = 2;          // (a 12 nm flake: 39.6 % equal-parity pairs, 4 passes 39.4 %)
constexpr int kColorMaxNodes = kHaloRows + kHaloMaxExt;
constexpr int kColorSmem = (kColorMaxNodes + 1) * 4 + kColorMaxNodes * 4 + kColorMaxEnt * 2 * 2 +
                           kColorMaxNodes * 2 + kColorMaxNodes;

// Pass 2: the lists (at halo_ptr[hb]) and the per-entry positions, packed.
__global__ void __launch_bounds__(kHaloThreads) k_halo_fill(const int64_t *slice_ptr,
                                                            const int32_t *col,
                                                            const int64_t *halo_ptr,
                                                            const int64_t *pslice,
                                                            int32_t *halo_rows, uint16_t *lcol)
{
    __shared__ int32_t keys[kHaloHash];
    __shared__ int32_t ext[kHaloMaxExt];
    __shared__ int n_ext, overflow;
    extern __shared__ __align__(16) unsigned char dyn[];
    int32_t *offs = reinterpret_cast<int32_t *>(dyn);                   // [nodes + 1]
    int32_t *cursor = offs + (kColorMaxNodes + 1);                      // [nodes]
    uint16_t *posbuf = reinterpret_cast<uint16_t *>(cursor + kColorMaxNodes);  // [entries]
    uint16_t *adj = posbuf + kColorMaxEnt;                              // [entries]
    uint16_t *slot = adj + kColorMaxEnt;                                // [nodes]
    uint8_t *color = reinterpret_cast<uint8_t *>(slot + kColorMaxNodes);       // [nodes]
    const int tid = threadIdx.x;
    const int64_t hb = blockIdx.x;
    halo_collect(hb, slice_ptr, col, keys, ext, &n_ext, &overflow, true);
    const int n = n_ext;
    const int H = kHaloRows + n;
    const int64_t r0 = hb * kHaloRows;
    const int64_t q0 = r0 / kSliceRows;
    constexpr int SPB = kHaloRows / kSliceRows;
    const int64_t pb = pslice[q0];
    const int64_t E = pslice[q0 + SPB] - pb;
    const bool colour = E <= kColorMaxEnt && n > 1;
    // node of every packed entry: the own row (its local index), or
    // kHaloRows + its index in ext
    for (int qq = 0; qq < SPB; ++qq) {
        const int64_t q = q0 + qq;
        const int64_t e0 = slice_ptr[q];
        const int w = (int)((slice_ptr[q + 1] - e0) / kSliceRows);
        const int w4 = (w + 3) / 4 * 4;
        for (int idx = tid; idx < w4 * kSliceRows; idx += kHaloThreads) {
            const int k = idx / kSliceRows, lr = idx % kSliceRows;
            int pos = qq * kSliceRows + lr;                 // padding: the own row
            if (k < w) {
                const int32_t c = col[e0 + idx];
                if (c >= r0 && c < r0 + kHaloRows) {
                    pos = (int)(c - r0);
                } else {
                    int lo = 0, hi = n - 1;                 // ext is sorted and holds c
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (ext[mid] < c) lo = mid + 1; else hi = mid;
                    }
                    pos = kHaloRows + lo;
                }
            }
            const int64_t at = pslice[q] + (k / 4) * (4 * kSliceRows) + lr * 4 + k % 4;
            if (colour) posbuf[at - pb] = (uint16_t)pos;
            else lcol[at] = (uint16_t)pos;
        }
    }
    int32_t *out = halo_rows + halo_ptr[hb];
    for (int k = tid; k < kHaloRows; k += kHaloThreads) out[k] = (int32_t)(r0 + k);
    if (!colour) {
        for (int i = tid; i < n; i += kHaloThreads) out[kHaloRows + i] = ext[i];
        return;
    }
    // the pair graph in CSR form (edges of equal nodes are broadcasts: left out)
    for (int v = tid; v < H; v += kHaloThreads) cursor[v] = 0;
    __syncthreads();
    auto for_pairs = [&](auto fn) {
        for (int qq = 0; qq < SPB; ++qq) {
            const int base = (int)(pslice[q0 + qq] - pb);
            const int w4 = (int)((pslice[q0 + qq + 1] - pslice[q0 + qq]) / kSliceRows);
            for (int idx = tid; idx < w4 * (kSliceRows / 2); idx += kHaloThreads) {
                const int k = idx / (kSliceRows / 2), m = idx % (kSliceRows / 2);
                const int i0 = base + (k / 4) * (4 * kSliceRows) + (2 * m) * 4 + k % 4;
                const int u = posbuf[i0], v = posbuf[i0 + 4];   // rows 2m and 2m+1
                if (u != v) fn(u, v);
            }
        }
    };
    for_pairs([&](int u, int v) {
        atomicAdd(&cursor[u], 1);
        atomicAdd(&cursor[v], 1);
    });
    __syncthreads();
    if (tid < 32) {                                     // exclusive scan of the degrees
        int run = 0;
        for (int v0 = 0; v0 < H; v0 += 32) {
            const int v = v0 + tid;
            const int d = v < H ? cursor[v] : 0;
            int incl = d;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += t;
            }
            if (v < H) offs[v] = cursor[v] = run + incl - d;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (tid == 0) offs[H] = run;
    }
    __syncthreads();
    for_pairs([&](int u, int v) {
        adj[atomicAdd(&cursor[u], 1)] = (uint16_t)v;
        adj[atomicAdd(&cursor[v], 1)] = (uint16_t)u;
    });
    for (int v = tid; v < H; v += kHaloThreads)
        color[v] = (uint8_t)(v < kHaloRows ? (v & 1) : ((v - kHaloRows) & 1));   // the sorted layout
    __syncthreads();
    if (tid < 32) {
        const int target = (n + 1) / 2;                 // even slots among kHaloRows .. H-1
        const int cap = 2 + n / 32;
        int e0 = target;                                // colour-0 external rows
        // cut gained by moving v to the other colour, summed by the warp
        auto gain = [&](int v) {
            const int cv = color[v];
            int s = 0;
            for (int e = offs[v] + tid; e < offs[v + 1]; e += 32) s += color[adj[e]] == cv ? 1 : -1;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            return s;
        };
        for (int pass = 0; pass < kColorPasses; ++pass) {
            bool moved = false;
            for (int v = kHaloRows; v < H; ++v) {
                const int g = gain(v);
                const int ne0 = e0 + (color[v] == 0 ? -1 : 1);
                __syncwarp();
                if (g > 0 && abs(ne0 - target) <= cap) {
                    if (tid == 0) color[v] ^= 1;
                    e0 = ne0;
                    moved = true;
                }
                __syncwarp();
            }
            if (!moved) break;
        }
        // restore the counts: move the majority colour's least harmful rows
        while (e0 != target) {
            const int cm = e0 > target ? 0 : 1;
            int best = INT32_MAX, bg = INT32_MIN;
            for (int v = kHaloRows + tid; v < H; v += 32) {
                if (color[v] != cm) continue;
                int s = 0;
                for (int e = offs[v]; e < offs[v + 1]; ++e) s += color[adj[e]] == cm ? 1 : -1;
                if (s > bg) { bg = s; best = v; }
            }
            for (int o = 16; o > 0; o >>= 1) {          // largest gain, then lowest row
                const int og = __shfl_xor_sync(0xffffffffu, bg, o);
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                if (og > bg || (og == bg && ob < best)) { bg = og; best = ob; }
            }
            __syncwarp();
            if (tid == 0) color[best] ^= 1;
            __syncwarp();
            e0 += cm == 0 ? -1 : 1;
        }
        // slots: colour c takes kHaloRows + c, + 2 + c, ... in row order
        int c0 = 0, c1 = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + tid;
            const int c = i < n ? color[kHaloRows + i] : 0;
            const unsigned m1 = __ballot_sync(0xffffffffu, i < n && c == 1);
            const unsigned m0 = __ballot_sync(0xffffffffu, i < n && c == 0);
            const unsigned below = (1u << tid) - 1u;
            if (i < n) {
                const int rk = c ? c1 + __popc(m1 & below) : c0 + __popc(m0 & below);
                slot[kHaloRows + i] = (uint16_t)(kHaloRows + 2 * rk + c);
            }
            c0 += __popc(m0);
            c1 += __popc(m1);
        }
    }
    for (int v = tid; v < kHaloRows; v += kHaloThreads) slot[v] = (uint16_t)v;
    __syncthreads();
    for (int i = tid; i < n; i += kHaloThreads) out[slot[kHaloRows + i]] = ext[i];
    for (int e = tid; e < (int)E; e += kHaloThreads) lcol[pb + e] = slot[posbuf[e]];
}

// Packed copy of the values (see above), padding slots 0.
template <typename T>
__global__ void k_pack_values(int64_t n_rows, const int64_t *slice_ptr, const int64_t *pslice,
                              const T *val, T *vpack)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t q = r / kSliceRows;
    const int lr = (int)(r % kSliceRows);
    const int64_t e0 = slice_ptr[q];
    const int w = (int)((slice_ptr[q + 1] - e0) / kSliceRows);
    const int w4 = (w + 3) / 4 * 4;
    for (int k = 0; k < w4; ++k)
        vpack[pslice[q] + (k / 4) * (4 * kSliceRows) + lr * 4 + k % 4] =
            k < w ? val[e0 + (int64_t)k * kSliceRows + lr] : (T)0;
}

}  // namespace

int build_halo(BuildOutput &b, cudaStream_t st, std::string &msg)
{
    if (b.halo_ptr) return TBPM_OK;
    if (b.n_rows % kHaloRows) { msg = "rows are not a multiple of the halo block"; return TBPM_E_UNSUPPORTED; }
    const int64_t nb = b.n_rows / kHaloRows;
    const int64_t ns = b.n_slices;
    int64_t *size = nullptr, *ent = nullptr, *pslice = nullptr;
    CK(cudaMalloc(&size, (nb + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&ent, (ns + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&pslice, (ns + 1) * sizeof(int64_t)));
    // packed slice offsets
    k_packed_slice_entries<<<blocks_for(ns, 256), 256, 0, st>>>(ns, b.slice_ptr, ent);
    CK(cudaGetLastError());
    int rc0 = scan_exclusive(ent, pslice, ns, st, msg);
    cudaFree(ent);
    if (rc0) { cudaFree(size); cudaFree(pslice); return rc0; }
    std::vector<int64_t> hp(ns + 1);
    CK(cudaMemcpyAsync(hp.data(), pslice, (ns + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    k_halo_count<<<(unsigned)nb, kHaloThreads, 0, st>>>(b.slice_ptr, b.col, size);
    CK(cudaGetLastError());
    std::vector<int64_t> hs(nb);
    CK(cudaMemcpyAsync(hs.data(), size, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int spb = kHaloRows / kSliceRows;          // slices per halo block
    int64_t emx = 0;
    for (int64_t k = 0; k < nb; ++k) emx = std::max(emx, hp[(k + 1) * spb] - hp[k * spb]);
    int64_t mx = 0;
    for (int64_t k = 0; k < nb; ++k) {
        if (hs[k] < 0) {
            cudaFree(size);
            cudaFree(pslice);
            msg = "a row block references more than " + std::to_string(kHaloMaxExt) +
                  " other rows: no halo lists for this matrix";
            return TBPM_E_UNSUPPORTED;
        }
        mx = std::max(mx, hs[k]);
    }
    int64_t *ptr = nullptr;
    CK(cudaMalloc(&ptr, (nb + 1) * sizeof(int64_t)));
    int rc = scan_exclusive(size, ptr, nb, st, msg);
    cudaFree(size);
    if (rc) { cudaFree(ptr); cudaFree(pslice); return rc; }
    int64_t total = 0;
    CK(cudaMemcpyAsync(&total, ptr + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int32_t *rows = nullptr;
    uint16_t *lc = nullptr;
    const int64_t npack = hp[ns];
    cudaError_t e = cudaMalloc(&rows, total * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&lc, (npack > 0 ? npack : 1) * sizeof(uint16_t));
    if (e != cudaSuccess) {
        cudaFree(ptr); cudaFree(rows); cudaFree(lc); cudaFree(pslice);
        msg = std::string("halo lists: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TBPM_E_OOM : TBPM_E_CUDA;
    }
    e = cudaFuncSetAttribute(k_halo_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, kColorSmem);
    if (e == cudaSuccess) {
        k_halo_fill<<<(unsigned)nb, kHaloThreads, kColorSmem, st>>>(b.slice_ptr, b.col, ptr, pslice,
                                                                     rows, lc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(ptr); cudaFree(rows); cudaFree(lc); cudaFree(pslice);
        msg = std::string("halo lists: ") + cudaGetErrorString(e);
        return TBPM_E_CUDA;
    }
    b.halo_ptr = ptr;
    b.halo_rows = rows;
    b.lcol = lc;
    b.pslice = pslice;
    b.n_packed = npack;
    b.halo_max = (int)mx;
    b.halo_ent_max = (int)std::min<int64_t>(emx, INT32_MAX);
    b.halo_total = total;
    return TBPM_OK;
}

int build_packed_values(BuildOutput &b, int fp32, cudaStream_t st, std::string &msg)
{
    if (!b.pslice) { msg = "no halo lists"; return TBPM_E_STATE; }
    if (b.vpack[fp32]) return TBPM_OK;
    const void *val = fp32 ? (const void *)b.val32 : (const void *)b.val64;
    if (!val || b.cplx) { msg = "no real values of this precision"; return TBPM_E_STATE; }
    const size_t bytes = (size_t)std::max<int64_t>(b.n_packed, 1) * (fp32 ? 4 : 8);
    void *vp = nullptr;
    CK(cudaMalloc(&vp, bytes));
    if (fp32)
        k_pack_values<float><<<blocks_for(b.n_rows, 256), 256, 0, st>>>(
            b.n_rows, b.slice_ptr, b.pslice, (const float *)val, (float *)vp);
    else
        k_pack_values<double><<<blocks_for(b.n_rows, 256), 256, 0, st>>>(
            b.n_rows, b.slice_ptr, b.pslice, (const double *)val, (double *)vp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(vp);
        msg = std::string("packed values: ") + cudaGetErrorString(e);
        return TBPM_E_CUDA;
    }
    b.vpack[fp32] = vp;
    return TBPM_OK;
}

namespace {
__global__ void k_twice(int64_t n, const double *src, double *dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + src[i];
}
}  // namespace

int build_diag2(BuildOutput &b, cudaStream_t st, std::string &msg)
{
    if (b.diag2_64) return TBPM_OK;
    if (!b.diag64) { msg = "no FP64 diagonal"; return TBPM_E_STATE; }
    double *d2 = nullptr;
    CK(cudaMalloc(&d2, (size_t)std::max<int64_t>(b.n_rows, 1) * sizeof(double)));
    k_twice<<<blocks_for(b.n_rows, 256), 256, 0, st>>>(b.n_rows, b.diag64, d2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(d2);
        msg = std::string("2 d: ") + cudaGetErrorString(e);
        return TBPM_E_CUDA;
    }
    b.diag2_64 = d2;
    return TBPM_OK;
}

void free_build(BuildOutput &b)
{
    cudaFree(b.diag2_64);
    cudaFree(b.user_to_row);
    cudaFree(b.orb_sample);
    cudaFree(b.slice_ptr);
    cudaFree(b.col);
    cudaFree(b.val64);
    cudaFree(b.val32);
    cudaFree(b.diag64);
    cudaFree(b.diag32);
    cudaFree(b.chunk_sample);
    cudaFree(b.bond_rows);
    cudaFree(b.halo_ptr);
    cudaFree(b.halo_rows);
    cudaFree(b.lcol);
    cudaFree(b.pslice);
    cudaFree(b.vpack[0]);
    cudaFree(b.vpack[1]);
    b = BuildOutput();
}

int build_sell(const BuildInput &in, int keep64, int keep32, int detect_uniform,
               int keep_bond_map, BuildOutput &out, cudaStream_t st, std::string &msg)
{
    const int T = 256;
    const int vw = in.cplx ? 2 : 1;      // doubles per stored value
    std::vector<int64_t> row_off(in.n_samples + 1);
    CK(cudaMemcpyAsync(row_off.data(), in.d_sample_row_off,
                       (in.n_samples + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t n_rows = row_off[in.n_samples];
    const int64_t n_slices = n_rows / kSliceRows;
    out.n_rows = n_rows;
    out.n_slices = n_slices;
    out.n_orb_user = in.n_orb;

    CK(cudaMalloc(&out.user_to_row, in.n_orb * sizeof(int32_t)));
    CK(cudaMalloc(&out.orb_sample, in.n_orb * sizeof(int32_t)));
    k_map_orbitals<<<blocks_for(in.n_orb, T), T, 0, st>>>(
        in.n_orb, in.n_samples, in.d_sample_off, in.d_sample_row_off, in.d_perm,
        out.user_to_row, out.orb_sample);
    CK(cudaGetLastError());

    int32_t *deg = nullptr, *fill = nullptr;
    int64_t *entries = nullptr;
    int *err = nullptr;           // [0] error bits, [1] max width
    unsigned long long *gbits = nullptr;   // [0] Gershgorin bits, [1] bandwidth
    CK(cudaMalloc(&deg, n_rows * sizeof(int32_t)));
    CK(cudaMalloc(&fill, n_rows * sizeof(int32_t)));
    CK(cudaMalloc(&entries, (n_slices + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&err, 2 * sizeof(int)));
    CK(cudaMalloc(&gbits, 2 * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(deg, 0, n_rows * sizeof(int32_t), st));
    CK(cudaMemsetAsync(fill, 0, n_rows * sizeof(int32_t), st));
    CK(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(gbits, 0, 2 * sizeof(unsigned long long), st));

    if (in.n_hop > 0) {
        k_count<<<blocks_for(in.n_hop, T), T, 0, st>>>(in.n_hop, in.n_orb, in.hop_i, in.hop_j,
                                                       in.hop_v, vw, out.user_to_row,
                                                       out.orb_sample, deg, err);
        CK(cudaGetLastError());
    }
    int h_err[2] = {0, 0};
    CK(cudaMemcpyAsync(h_err, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    auto cleanup = [&]() {
        cudaFree(deg); cudaFree(fill); cudaFree(entries); cudaFree(err); cudaFree(gbits);
    };
    if (h_err[0]) {
        msg = "invalid bond list:";
        if (h_err[0] & 1) msg += " index out of range;";
        if (h_err[0] & 2) msg += " bond from an orbital to itself;";
        if (h_err[0] & 4) msg += " bond joins two samples;";
        if (h_err[0] & 8) msg += " non-finite hopping;";
        cleanup();
        return TBPM_E_INVALID_ARG;
    }
    k_slice_width<<<blocks_for(n_slices * 32, T), T, 0, st>>>(n_slices, deg, entries, err + 1);
    CK(cudaGetLastError());
    CK(cudaMalloc(&out.slice_ptr, (n_slices + 1) * sizeof(int64_t)));
    int rc = scan_exclusive(entries, out.slice_ptr, n_slices, st, msg);
    if (rc) { cleanup(); return rc; }
    CK(cudaMemcpyAsync(&out.nnz_pad, out.slice_ptr + n_slices, sizeof(int64_t),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&out.max_width, err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out.nnz_true = 2 * in.n_hop;
    // Fixed-width layout when padding every slice to the widest costs at most
    // 10 % more slots (lattices: nearly every slice has the maximum width):
    // the term kernels then compute a slice's base instead of loading it.
    out.fixed_width = 0;
    if (out.max_width > 0 && (double)n_slices * kSliceRows * out.max_width <= 1.1 * out.nnz_pad) {
        k_fixed_slices<<<blocks_for(n_slices + 1, T), T, 0, st>>>(n_slices, out.max_width,
                                                                   out.slice_ptr);
        CK(cudaGetLastError());
        out.fixed_width = out.max_width;
        out.nnz_pad = n_slices * kSliceRows * (int64_t)out.max_width;
    }
    if (out.nnz_pad > (int64_t)1 << 40) { msg = "matrix too large"; cleanup(); return TBPM_E_OOM; }

    int64_t nnz_alloc = out.nnz_pad > 0 ? out.nnz_pad : 1;
    CK(cudaMalloc(&out.col, nnz_alloc * sizeof(int32_t)));
    // values go straight to their kept precision: FP64 (and FP32 converted
    // from it afterwards) or, without the FP64 copy, FP32 only
    const bool direct32 = !keep64;
    if (direct32)
        CK(cudaMalloc(&out.val32, nnz_alloc * vw * sizeof(float)));
    else
        CK(cudaMalloc(&out.val64, nnz_alloc * vw * sizeof(double)));
    out.cplx = in.cplx;
    CK(cudaMalloc(&out.diag64, n_rows * sizeof(double)));
    CK(cudaMemsetAsync(out.diag64, 0, n_rows * sizeof(double), st));
    auto fill_all = [&](auto *val) -> cudaError_t {
        typedef typename std::remove_pointer<decltype(val)>::type VT;
        if (vw == 2)
            k_pad_fill<2, VT><<<blocks_for(n_rows, T), T, 0, st>>>(n_rows, out.slice_ptr, out.col, val);
        else
            k_pad_fill<1, VT><<<blocks_for(n_rows, T), T, 0, st>>>(n_rows, out.slice_ptr, out.col, val);
        if (in.n_hop > 0) {
            if (vw == 2)
                k_fill<2, VT><<<blocks_for(in.n_hop, T), T, 0, st>>>(
                    in.n_hop, in.hop_i, in.hop_j, in.hop_v, in.inv_s, out.user_to_row,
                    out.slice_ptr, fill, out.col, val);
            else
                k_fill<1, VT><<<blocks_for(in.n_hop, T), T, 0, st>>>(
                    in.n_hop, in.hop_i, in.hop_j, in.hop_v, in.inv_s, out.user_to_row,
                    out.slice_ptr, fill, out.col, val);
        }
        k_diag<<<blocks_for(in.n_orb, T), T, 0, st>>>(in.n_orb, in.onsite, in.inv_s,
                                                      out.user_to_row, out.diag64);
        if (vw == 2)
            k_sort_rows<2, VT><<<blocks_for(n_rows, T), T, 0, st>>>(
                n_rows, out.slice_ptr, deg, out.diag64, out.col, val, gbits, gbits + 1);
        else
            k_sort_rows<1, VT><<<blocks_for(n_rows, T), T, 0, st>>>(
                n_rows, out.slice_ptr, deg, out.diag64, out.col, val, gbits, gbits + 1);
        return cudaGetLastError();
    };
    CK(direct32 ? fill_all(out.val32) : fill_all(out.val64));
    unsigned long long hg[2] = {0, 0};
    CK(cudaMemcpyAsync(hg, gbits, sizeof(hg), cudaMemcpyDeviceToHost, st));

    // chunk -> sample table
    int64_t n_chunks = n_rows / kChunkRows;
    std::vector<int32_t> cs(n_chunks > 0 ? n_chunks : 1);
    for (int s = 0; s < in.n_samples; ++s)
        for (int64_t c = row_off[s] / kChunkRows; c < row_off[s + 1] / kChunkRows; ++c)
            cs[c] = s;
    CK(cudaMalloc(&out.chunk_sample, cs.size() * sizeof(int32_t)));
    CK(cudaMemcpyAsync(out.chunk_sample, cs.data(), cs.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice, st));

    out.n_hop = in.n_hop;
    out.zero_diag = in.onsite == nullptr;
    if (in.onsite) {          // a diagonal of zeros passed explicitly
        CK(cudaMemsetAsync(err, 0xff, sizeof(int), st));
        k_zero_onsite<<<blocks_for(in.n_orb, T), T, 0, st>>>(in.n_orb, in.onsite, err);
        CK(cudaGetLastError());
        int zero = 0;
        CK(cudaMemcpyAsync(&zero, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out.zero_diag = zero != 0;
    }
    if (detect_uniform && in.n_hop > 0 && vw == 1) {
        // one hopping value everywhere (e.g. pristine or onsite-disordered
        // lattices): the term kernels then need no value loads
        CK(cudaMemsetAsync(err, 0xff, sizeof(int), st));
        k_uniform<<<blocks_for(in.n_hop, T), T, 0, st>>>(in.n_hop, in.hop_v, in.inv_s, err);
        CK(cudaGetLastError());
        int same = 0;
        double v0 = 0.0;
        CK(cudaMemcpyAsync(&same, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&v0, in.hop_v, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out.uniform = same != 0;
        out.h_uniform = v0 * in.inv_s;
    }
    if (in.n_hop > 0 && keep_bond_map) {  // bond -> rows: the adjoint's gradients, the bond vectors
        CK(cudaMalloc(&out.bond_rows, 2 * in.n_hop * sizeof(int32_t)));
        k_bond_rows<<<blocks_for(in.n_hop, T), T, 0, st>>>(in.n_hop, in.hop_i, in.hop_j,
                                                           out.user_to_row, out.bond_rows);
        CK(cudaGetLastError());
    }
    if (keep32) {
        if (!direct32) CK(cudaMalloc(&out.val32, nnz_alloc * vw * sizeof(float)));
        CK(cudaMalloc(&out.diag32, n_rows * sizeof(float)));
        if (out.nnz_pad > 0 && !direct32)
            k_to_f32<<<blocks_for(out.nnz_pad * vw, T), T, 0, st>>>(out.nnz_pad * vw, out.val64,
                                                                    out.val32);
        k_to_f32<<<blocks_for(n_rows, T), T, 0, st>>>(n_rows, out.diag64, out.diag32);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(st));
    double g;
    memcpy(&g, &hg[0], sizeof(g));
    out.gershgorin = g;
    out.bandwidth = (int64_t)hg[1];
    if (!keep64) {
        cudaFree(out.val64);
        cudaFree(out.diag64);
        out.val64 = nullptr;
        out.diag64 = nullptr;
    }
    cleanup();
    return TBPM_OK;
}

}  // namespace tbpm
