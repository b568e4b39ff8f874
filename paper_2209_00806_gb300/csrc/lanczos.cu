// a1, spectral bound: Lanczos estimate of the extreme eigenvalues of H~.
//
// The expansion of Sec. 2.2 holds for H~ = H / s with its spectrum inside
// [-1, 1]; the Chebyshev series of exp(-i z x) grows without bound outside.
// The builder's Gershgorin bound is safe but loose (it counts every
// |H_ij|); the Lanczos process on a fixed start vector gives Ritz values
// that lie inside the spectrum and approach its ends within tens of steps,
// so max |Ritz value| is a lower bound on the spectral radius that is close
// to it.  Each step is one sparse product and two deterministic FP64
// reductions on the GPU; the tridiagonal matrix of the Lanczos coefficients
// is solved for its extreme eigenvalues on the host by bisection with Sturm
// counts.
//
// Start vector: v_u = (U_2u - 1/2) + i (U_2u+1 - 1/2) in caller order u,
// normalised, with U_k = top 53 bits of the SplitMix64 output function
// (Steele, Lea & Flood, OOPSLA 2014) of key + GAMMA (k + 1), key = mix(seed +
// GAMMA (stream + 1)), seed kLanczosSeed, stream kLanczosStream -- so any
// other implementation of that published generator draws the same vector.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kLzThreads = 256;
constexpr int kLzBlocks = 1024;         // blocks of the reductions (grid-stride)

__host__ __device__ inline uint64_t mix64(uint64_t x)
{
    uint64_t y = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    uint64_t z = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ inline double unit53(uint64_t key, uint64_t k)
{
    return (double)(mix64(key + kGamma * (k + 1)) >> 11) * 0x1.0p-53;
}

__global__ void k_lz_start(int64_t n_orb, const int32_t *user_to_row, uint64_t key, double2 *v)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n_orb) return;
    v[user_to_row[u]] = make_double2(unit53(key, 2 * (uint64_t)u) - 0.5,
                                     unit53(key, 2 * (uint64_t)u + 1) - 0.5);
}

// Sum of the block's per-thread values in a fixed tree; thread 0 returns it.
__device__ inline double block_sum(double x)
{
    __shared__ double w[kLzThreads / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (threadIdx.x % 32 == 0) w[threadIdx.x / 32] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kLzThreads / 32; ++k) s += w[k];
    __syncthreads();
    return s;
}

// w = H~ v - beta v_prev (complex v, real or complex values of type T), and
// the block partial of Re <v|w>.  Rows in a fixed grid-stride assignment.
template <typename T>
__global__ void __launch_bounds__(kLzThreads) k_lz_apply(SellView H, int cplx, int64_t n_rows,
                                                         const double2 *v, const double2 *vprev,
                                                         const double *beta, double2 *w,
                                                         double *partial)
{
    const double b = *beta;
    double acc = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)kLzThreads + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * kLzThreads) {
        const int64_t q = r / kSliceRows;
        const int64_t base = H.slice_ptr[q] + r % kSliceRows;
        const int wd = (int)((H.slice_ptr[q + 1] - H.slice_ptr[q]) / kSliceRows);
        const double d = (double)reinterpret_cast<const T *>(H.diag)[r];
        const double2 vr = v[r];
        double yr = d * vr.x, yi = d * vr.y;
        for (int k = 0; k < wd; ++k) {
            const int64_t e = base + (int64_t)k * kSliceRows;
            const int32_t c = H.col[e];
            const double2 x = v[c];
            double hr, hi = 0.0;
            if (cplx) {
                hr = (double)reinterpret_cast<const T *>(H.val)[2 * e];
                hi = (double)reinterpret_cast<const T *>(H.val)[2 * e + 1];
            } else {
                hr = (double)reinterpret_cast<const T *>(H.val)[e];
            }
            yr += hr * x.x - hi * x.y;
            yi += hr * x.y + hi * x.x;
        }
        const double2 p = vprev[r];
        const double2 o = make_double2(yr - b * p.x, yi - b * p.y);
        w[r] = o;
        acc += vr.x * o.x + vr.y * o.y;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// w -= alpha v (alpha = *alpha_p); block partial of |w|^2.
__global__ void __launch_bounds__(kLzThreads) k_lz_orth(int64_t n_rows, const double2 *v,
                                                        const double *alpha_p, double2 *w,
                                                        double *partial)
{
    const double a = alpha_p ? *alpha_p : 0.0;
    double acc = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)kLzThreads + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * kLzThreads) {
        const double2 x = v[r];
        double2 o = w[r];
        o.x -= a * x.x;
        o.y -= a * x.y;
        w[r] = o;
        acc += o.x * o.x + o.y * o.y;
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out = sum of the n partials in a fixed order (one block).
__global__ void __launch_bounds__(kLzThreads) k_lz_total(const double *partial, int n, double *out,
                                                         int take_sqrt)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += kLzThreads) acc += partial[k];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : s;
}

// v_next = w / beta into dst (may be w itself).
__global__ void k_lz_scale(int64_t n_rows, const double2 *w, const double *beta, double2 *dst)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const double inv = 1.0 / *beta;
    const double2 x = w[r];
    dst[r] = make_double2(x.x * inv, x.y * inv);
}

// Number of eigenvalues of the symmetric tridiagonal matrix (diagonal a,
// off-diagonal b[1..m-1]) below x (Sturm sequence of the LDL^T pivots).
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i ? b[i] * b[i] / q : 0.0;
        q = a[i] - x - off;
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

}  // namespace

int lanczos_extremes(const BuildOutput &H, int n_iter, cudaStream_t st, double *lo, double *hi,
                     int *steps, std::string &msg)
{
    const int64_t n = H.n_rows;
    double2 *buf[3] = {nullptr, nullptr, nullptr};
    double *part = nullptr, *scal = nullptr;      // scal: [0] alpha, [1] beta, [2] zero
    auto release = [&]() {
        for (auto &p : buf) cudaFree(p);
        cudaFree(part);
        cudaFree(scal);
    };
#define LZ_CK(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            release();                                                                \
            msg = std::string("Lanczos: ") + #call + ": " + cudaGetErrorString(e_);   \
            return e_ == cudaErrorMemoryAllocation ? TBPM_E_OOM : TBPM_E_CUDA;        \
        }                                                                             \
    } while (0)
    for (auto &p : buf) LZ_CK(cudaMalloc(&p, n * sizeof(double2)));
    LZ_CK(cudaMalloc(&part, kLzBlocks * sizeof(double)));
    LZ_CK(cudaMalloc(&scal, 4 * sizeof(double)));
    LZ_CK(cudaMemsetAsync(scal, 0, 4 * sizeof(double), st));
    for (auto &p : buf) LZ_CK(cudaMemsetAsync(p, 0, n * sizeof(double2), st));
    const uint64_t key = mix64((uint64_t)kLanczosSeed + kGamma * (uint64_t)(kLanczosStream + 1));
    const int64_t n_orb = H.n_orb_user;
    k_lz_start<<<(unsigned)((n_orb + 255) / 256), 256, 0, st>>>(n_orb, H.user_to_row, key, buf[1]);
    const unsigned nb = (unsigned)std::min<int64_t>(kLzBlocks, (n + kLzThreads - 1) / kLzThreads);
    // normalise the start vector
    k_lz_orth<<<nb, kLzThreads, 0, st>>>(n, buf[1], nullptr, buf[1], part);
    k_lz_total<<<1, kLzThreads, 0, st>>>(part, (int)nb, scal + 1, 1);
    k_lz_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, buf[1], scal + 1, buf[1]);
    LZ_CK(cudaMemsetAsync(scal + 1, 0, sizeof(double), st));   // beta_0 = 0
    LZ_CK(cudaGetLastError());
    const bool f32 = H.val64 == nullptr;
    SellView hv;
    hv.slice_ptr = H.slice_ptr;
    hv.col = H.col;
    hv.val = f32 ? (const void *)H.val32 : (const void *)H.val64;
    hv.diag = f32 ? (const void *)H.diag32 : (const void *)H.diag64;
    std::vector<double> a, b(1, 0.0);
    int prev = 0, cur = 1, wk = 2;          // v_{j-1}, v_j, w
    double ab[2];
    for (int j = 0; j < n_iter; ++j) {
        if (f32)
            k_lz_apply<float><<<nb, kLzThreads, 0, st>>>(hv, H.cplx, n, buf[cur], buf[prev],
                                                         scal + 1, buf[wk], part);
        else
            k_lz_apply<double><<<nb, kLzThreads, 0, st>>>(hv, H.cplx, n, buf[cur], buf[prev],
                                                          scal + 1, buf[wk], part);
        k_lz_total<<<1, kLzThreads, 0, st>>>(part, (int)nb, scal + 0, 0);
        k_lz_orth<<<nb, kLzThreads, 0, st>>>(n, buf[cur], scal + 0, buf[wk], part);
        k_lz_total<<<1, kLzThreads, 0, st>>>(part, (int)nb, scal + 1, 1);
        LZ_CK(cudaGetLastError());
        LZ_CK(cudaMemcpyAsync(ab, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        LZ_CK(cudaStreamSynchronize(st));
        if (!std::isfinite(ab[0]) || !std::isfinite(ab[1])) {
            release();
            msg = "Lanczos: non-finite coefficient (non-finite matrix values?)";
            return TBPM_E_NONFINITE;
        }
        a.push_back(ab[0]);
        const double scale = std::fabs(ab[0]) + (b.size() > 1 ? b.back() : 0.0) + 1e-300;
        if (j + 1 == n_iter || ab[1] <= 1e-12 * scale) break;   // done or invariant subspace
        b.push_back(ab[1]);
        k_lz_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, buf[wk], scal + 1, buf[wk]);
        const int t = prev;
        prev = cur;
        cur = wk;
        wk = t;
    }
    LZ_CK(cudaStreamSynchronize(st));
    release();
#undef LZ_CK
    // extreme eigenvalues of T by bisection on the Gershgorin interval of T
    const int m = (int)a.size();
    double g = 0.0;
    for (int i = 0; i < m; ++i)
        g = std::max(g, std::fabs(a[i]) + (i ? std::fabs(b[i]) : 0.0) +
                            (i + 1 < m ? std::fabs(b[i + 1]) : 0.0));
    auto kth = [&](int k) {          // the k-th smallest eigenvalue (0-based)
        double l = -g - 1e-300, h = g + 1e-300;
        for (int it = 0; it < 200 && h - l > 1e-15 * std::max(1.0, g); ++it) {
            const double mid = 0.5 * (l + h);
            if (sturm_count(a, b, mid) > k) h = mid; else l = mid;
        }
        return 0.5 * (l + h);
    };
    *lo = kth(0);
    *hi = kth(m - 1);
    *steps = m;
    return TBPM_OK;
}

}  // namespace tbpm
