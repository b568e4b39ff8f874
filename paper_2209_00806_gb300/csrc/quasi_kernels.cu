// Quasi-eigenstates (Sec. 2.6, Eq. quasi): after every time step of the
// forward run and of the backward run (H -> -H), each state lane adds
// c_{n,k} psi(t_n) to the accumulator of every energy E_k, where
// c_{n,k} = (tau / 2 pi) w_n e^{i E_k t_n} comes from a host table (FP64 and
// FP32 copies) indexed by the step counter the reduction has just advanced
// (graph-safe).  Then the
// accumulators go to the caller's layout and are normalised per energy,
// state and sample.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

template <typename V> struct QeC;
template <> struct QeC<double> {
    typedef double2 type;
    __device__ static const double *scale(const QeArgs &a) { return a.scale; }
    __device__ static const void *coef(const QeArgs &a) { return a.coef; }
};
template <> struct QeC<float> {
    typedef float2 type;
    __device__ static const float *scale(const QeArgs &a) { return a.scale_f; }
    __device__ static const void *coef(const QeArgs &a) { return a.coef_f; }
};

// One thread per (row, lane); acc is [K][n_rows][S] with this group's lanes
// at s0 .. s0 + B - 1, in the group's precision: FP32 accumulators in the
// FP32 form (GB300 runs FP64 at a small fraction of the FP32 rate; the sum of
// 2N + 1 windowed terms keeps the FP32 states' accuracy), FP64 in the FP64 form.
template <typename V>
__global__ void k_qe_acc(QeArgs a)
{
    typedef typename QeC<V>::type C;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n_rows * a.B) return;
    const int64_t r = t / a.B;
    const int l = (int)(t % a.B);
    const int smp = a.chunk_sample[r / kChunkRows];
    const int n = a.step[smp] - 1;
    C v = __ldg(reinterpret_cast<const C *>(a.psi) + t);
    if (a.scale) {
        const V sc = (V)QeC<V>::scale(a)[(int64_t)smp * a.B + l];
        v.x *= sc;
        v.y *= sc;
    }
    const C *cf = reinterpret_cast<const C *>(QeC<V>::coef(a)) + (int64_t)n * a.K;
    C *acc = reinterpret_cast<C *>(a.acc);
    for (int k = 0; k < a.K; ++k) {
        const C c = cf[k];
        C *q = acc + ((int64_t)k * a.n_rows + r) * a.S + a.s0 + l;
        C o = *q;
        o.x = fma(c.x, v.x, fma(-c.y, v.y, o.x));
        o.y = fma(c.x, v.y, fma(c.y, v.x, o.y));
        *q = o;
    }
}

// out[k][p][i] = acc[k][row(i)][p]
template <typename C>
__global__ void k_qe_store(const C *acc, int K, int S, int64_t n_rows, int64_t n_orb,
                           const int32_t *user_to_row, double2 *out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)K * S * n_orb) return;
    const int64_t i = t % n_orb;
    const int64_t kp = t / n_orb;
    const int p = (int)(kp % S), k = (int)(kp / S);
    const C v = acc[((int64_t)k * n_rows + user_to_row[i]) * S + p];
    out[t] = make_double2((double)v.x, (double)v.y);
}

// Squared norm of out[k][p][off_s .. off_{s+1}) per (k, p, sample s), one
// block each: strided per-thread sums, then a shared-memory tree (fixed order).
constexpr int kQeThreads = 256;
__global__ void __launch_bounds__(kQeThreads) k_qe_norms(const double2 *out, int n_samples,
                                                         int64_t n_orb, const int64_t *orb_off,
                                                         double *norms)
{
    const int64_t kps = blockIdx.x;            // (k * S + p) * n_samples + s
    const int smp = (int)(kps % n_samples);
    const int64_t kp = kps / n_samples;
    const double2 *v = out + kp * n_orb;
    double acc = 0.0;
    for (int64_t i = orb_off[smp] + threadIdx.x; i < orb_off[smp + 1]; i += kQeThreads) {
        const double2 x = v[i];
        acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    __shared__ double red[kQeThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kQeThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) norms[kps] = red[0];
}

__global__ void k_qe_normalise(double2 *out, int K, int S, int n_samples, int64_t n_orb,
                               const int32_t *orb_sample, const double *norms)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)K * S * n_orb) return;
    const int64_t i = t % n_orb;
    const int64_t kp = t / n_orb;
    const double nn = norms[kp * n_samples + orb_sample[i]];
    if (nn > 0.0) {
        const double f = 1.0 / sqrt(nn);
        out[t].x *= f;
        out[t].y *= f;
    }
}

}  // namespace

cudaError_t launch_qe_acc(const QeArgs &a, int fp32, cudaStream_t st)
{
    const int64_t n = a.n_rows * a.B;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (fp32) k_qe_acc<float><<<blocks, 256, 0, st>>>(a);
    else k_qe_acc<double><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_qe_finish(const void *acc, int fp32, int K, int S, int64_t n_rows, int64_t n_orb,
                             int n_samples, const int32_t *user_to_row, const int32_t *orb_sample,
                             const int64_t *orb_off, double2 *out, double *norms, cudaStream_t st)
{
    const int64_t n = (int64_t)K * S * n_orb;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (fp32)
        k_qe_store<float2><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(acc), K, S,
                                                    n_rows, n_orb, user_to_row, out);
    else
        k_qe_store<double2><<<blocks, 256, 0, st>>>(reinterpret_cast<const double2 *>(acc), K, S,
                                                     n_rows, n_orb, user_to_row, out);
    k_qe_norms<<<(unsigned)((int64_t)K * S * n_samples), kQeThreads, 0, st>>>(out, n_samples, n_orb,
                                                                             orb_off, norms);
    k_qe_normalise<<<blocks, 256, 0, st>>>(out, K, S, n_samples, n_orb, orb_sample, norms);
    return cudaGetLastError();
}

}  // namespace tbpm
