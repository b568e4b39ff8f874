// C ABI of the TBPM library: contexts, Hamiltonian build, states, the
// time-step loop of the Chebyshev propagation, correlations and statistics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <string>
#include <vector>

#include "tbpm_internal.cuh"

using namespace tbpm;

namespace {

thread_local std::string g_last_error;

struct Group {
    int B = 0, s0 = 0;
    void *psi0 = nullptr;        // internal layout, precision of the group
    void *buf[3] = {nullptr, nullptr, nullptr};
    double *scale = nullptr;     // [n_samples * B]
    float *scale_f = nullptr;    // FP32 copy
    int cur = 0;                 // buffer holding the current state
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
};

}  // namespace

struct tbpm_ctx {
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t st = nullptr;
    std::string err;

    // Hamiltonian
    bool have_h = false;
    BuildOutput H;
    int64_t n_orb = 0;
    int n_samples = 0;
    double s = 0.0;
    std::vector<int64_t> sample_off, row_off;
    int64_t *d_sample_chunk_off = nullptr;
    double *d_inv_sqrt_n = nullptr;

    // initial states, caller order, complex128 [n_states][n_orb]
    int n_states = 0;
    double2 *d_psi_user = nullptr;

    // propagation state
    int prec = -1;               // precision of the group buffers
    int max_group[2] = {8, 16};  // widest state group per precision
    int threads[2] = {64, 64};   // threads per block per precision (fastest on GB300)
    // term-kernel launch variants (FP64, FP32): the fastest on GB300 for
    // graphene-like lattices; tbpm_autotune re-checks for the actual matrix
    int variant[2] = {kVariantZigZag, kVariantZigZag | kVariantWide | kVariantPrefetch};
    int num_sms = 0;
    double renorm_fp32 = 1e-5, hard_fp32 = 1e-2, hard_fp64 = 1e-6;   // norm policy
    std::vector<Group> groups;
    double *d_partial = nullptr;
    int64_t partial_len = 0;
    double *d_block_partial = nullptr;
    int64_t block_partial_len = 0;
    int *d_chunk_count = nullptr;
    double *d_partial2 = nullptr;          // [n_samples][64][16][3]
    unsigned int *d_sample_ticket = nullptr;
    // wavefront-fused step
    int32_t *d_items = nullptr;
    int64_t items_len = 0;
    int items_key[3] = {-1, -1, -1};       // (J, tile rows, radius) of the table
    int *d_done = nullptr;
    int64_t done_len = 0;
    unsigned long long *d_fcounter = nullptr;
    FusedTerm *d_fterms = nullptr;         // [3][kMaxTerms]
    double *d_tile_partial = nullptr;
    int64_t tile_partial_len = 0;
    int *d_step = nullptr;       // [n_samples]
    int *d_flags = nullptr;      // [0] error bits
    unsigned long long *d_renorm = nullptr;
    double2 *d_corr = nullptr;
    double *d_norms = nullptr;
    int corr_steps = -1;         // n_steps of the buffers above
    double *d_norm_ref = nullptr;          // [n_samples][n_states] squared norms at t = 0
    int64_t norm_ref_len = 0;
    // AC-conductivity correlation
    double *d_bond_dx = nullptr, *d_bond_dy = nullptr;   // [nnz_pad] bond vector per entry
    float *d_bond_dx32 = nullptr, *d_bond_dy32 = nullptr; // FP32 copies
    bool ac_on = false;
    double2 *d_ac_corr = nullptr;          // [n_samples][n_states / 4][4][n_steps + 1]
    double *d_ac_partial = nullptr;        // [n_rows / kAcRows][4][8]
    // quasi-eigenstates
    bool qe_on = false;
    int qe_K = 0;
    double2 *d_qe_acc = nullptr;           // [K][n_rows][n_states]
    const double2 *d_qe_coef = nullptr;    // [n_steps + 1][K] of the current run
    const float2 *d_qe_coef_f = nullptr;   // its FP32 copy
    bool have_run = false;
    std::vector<cudaEvent_t> events;
    tbpm_stats stats;
};

namespace {

int fail(tbpm_ctx *c, int code, const std::string &m)
{
    if (c) c->err = m;
    g_last_error = m;
    return code;
}

#define CUDA_OR_FAIL(ctx, call)                                                    \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? TBPM_E_OOM : TBPM_E_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

template <typename T>
int dalloc(tbpm_ctx *c, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? TBPM_E_OOM : TBPM_E_CUDA,
                    std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                        " bytes: " + cudaGetErrorString(e));
    }
    return TBPM_OK;
}

void free_groups(tbpm_ctx *c)
{
    for (auto &g : c->groups) {
        cudaFree(g.psi0);
        for (int k = 0; k < 3; ++k) {
            cudaFree(g.buf[k]);
            if (g.graph[k]) cudaGraphExecDestroy(g.graph[k]);
        }
        cudaFree(g.scale);
        cudaFree(g.scale_f);
    }
    c->groups.clear();
    c->prec = -1;
    c->have_run = false;
}

void free_outputs(tbpm_ctx *c)
{
    cudaFree(c->d_corr);
    cudaFree(c->d_norms);
    c->d_corr = nullptr;
    c->d_norms = nullptr;
    c->corr_steps = -1;
}

void free_hamiltonian(tbpm_ctx *c)
{
    free_groups(c);
    free_outputs(c);
    free_build(c->H);
    cudaFree(c->d_sample_chunk_off);
    cudaFree(c->d_inv_sqrt_n);
    cudaFree(c->d_psi_user);
    cudaFree(c->d_partial);
    cudaFree(c->d_block_partial);
    cudaFree(c->d_chunk_count);
    cudaFree(c->d_partial2);
    cudaFree(c->d_sample_ticket);
    c->d_partial2 = nullptr;
    c->d_sample_ticket = nullptr;
    cudaFree(c->d_items);
    cudaFree(c->d_done);
    cudaFree(c->d_fcounter);
    cudaFree(c->d_fterms);
    cudaFree(c->d_tile_partial);
    c->d_items = nullptr;
    c->d_done = nullptr;
    c->d_fcounter = nullptr;
    c->d_fterms = nullptr;
    c->d_tile_partial = nullptr;
    c->items_len = c->done_len = c->tile_partial_len = 0;
    c->items_key[0] = c->items_key[1] = c->items_key[2] = -1;
    cudaFree(c->d_step);
    cudaFree(c->d_norm_ref);
    cudaFree(c->d_bond_dx);
    cudaFree(c->d_bond_dy);
    cudaFree(c->d_bond_dx32);
    cudaFree(c->d_bond_dy32);
    c->d_norm_ref = nullptr;
    c->norm_ref_len = 0;
    c->d_bond_dx = c->d_bond_dy = nullptr;
    c->d_bond_dx32 = c->d_bond_dy32 = nullptr;
    c->d_block_partial = nullptr;
    c->d_chunk_count = nullptr;
    c->block_partial_len = 0;
    c->d_sample_chunk_off = nullptr;
    c->d_inv_sqrt_n = nullptr;
    c->d_psi_user = nullptr;
    c->d_partial = nullptr;
    c->d_step = nullptr;
    c->partial_len = 0;
    c->n_states = 0;
    c->have_h = false;
}

// Order our stream after the user's stream.
int enter(tbpm_ctx *c)
{
    CUDA_OR_FAIL(c, cudaSetDevice(c->device));
    cudaEvent_t e;
    CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CUDA_OR_FAIL(c, cudaEventRecord(e, c->user));
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->st, e, 0));
    cudaEventDestroy(e);
    return TBPM_OK;
}

// Make the user's stream wait for our work.
int leave(tbpm_ctx *c)
{
    cudaEvent_t e;
    CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CUDA_OR_FAIL(c, cudaEventRecord(e, c->st));
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->user, e, 0));
    cudaEventDestroy(e);
    return TBPM_OK;
}

// Copy `bytes` from host or device memory into a fresh device buffer.
template <typename T>
int stage(tbpm_ctx *c, const T *src, size_t count, int where, T **dst, bool *owned)
{
    *owned = false;
    *dst = nullptr;
    if (!src) return TBPM_OK;
    if (where == TBPM_DEVICE) {
        *dst = const_cast<T *>(src);
        return TBPM_OK;
    }
    int rc = dalloc(c, dst, count);
    if (rc) return rc;
    *owned = true;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c->st));
    return TBPM_OK;
}

// Reverse Cuthill-McKee order of one sample's orbitals [lo, hi): BFS from a
// minimum-degree unvisited orbital, neighbours in increasing degree, order
// reversed.  perm[u] = position of orbital u within its sample.
void rcm_sample(int64_t lo, int64_t hi, const std::vector<int64_t> &adj_ptr,
                const std::vector<int32_t> &adj, std::vector<int32_t> &perm)
{
    const int64_t n = hi - lo;
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> seen(n, 0);
    std::vector<int64_t> by_deg(n);
    for (int64_t k = 0; k < n; ++k) by_deg[k] = k;
    auto deg = [&](int64_t u) { return adj_ptr[lo + u + 1] - adj_ptr[lo + u]; };
    std::stable_sort(by_deg.begin(), by_deg.end(),
                     [&](int64_t a, int64_t b) { return deg(a) < deg(b); });
    std::vector<int32_t> nb;
    for (int64_t start : by_deg) {
        if (seen[start]) continue;
        size_t head = order.size();
        order.push_back((int32_t)start);
        seen[start] = 1;
        while (head < order.size()) {
            int64_t u = order[head++];
            nb.clear();
            for (int64_t e = adj_ptr[lo + u]; e < adj_ptr[lo + u + 1]; ++e) {
                int64_t v = adj[e] - lo;
                if (!seen[v]) { seen[v] = 1; nb.push_back((int32_t)v); }
            }
            std::stable_sort(nb.begin(), nb.end(),
                             [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
            order.insert(order.end(), nb.begin(), nb.end());
        }
    }
    for (int64_t k = 0; k < n; ++k) perm[lo + order[n - 1 - k]] = (int32_t)k;
}

// Cluster order on top of RCM: walk the nodes in RCM order; each node not
// yet placed seeds a breadth-first ball of up to kClusterRows unplaced nodes
// (neighbours taken in RCM order), and the ball's nodes follow in RCM order.
// On geometric lattices a ball is a compact patch, so a block of rows
// gathers from a few hundred distinct rows (the patch and its rim) instead
// of the two RCM fronts around it: the gathers stay in L1.
constexpr int kClusterRows = 128;

void cluster_sample(int64_t lo, int64_t hi, const std::vector<int64_t> &adj_ptr,
                    const std::vector<int32_t> &adj, std::vector<int32_t> &perm)
{
    const int64_t n = hi - lo;
    std::vector<int32_t> by_rcm(n);                // RCM position -> local node
    for (int64_t u = 0; u < n; ++u) by_rcm[perm[lo + u]] = (int32_t)u;
    std::vector<char> placed(n, 0);
    std::vector<int32_t> ball, nb, out;
    out.reserve(n);
    for (int64_t k = 0; k < n; ++k) {
        const int32_t seed = by_rcm[k];
        if (placed[seed]) continue;
        ball.clear();
        ball.push_back(seed);
        placed[seed] = 1;
        for (size_t head = 0; head < ball.size() && ball.size() < (size_t)kClusterRows; ++head) {
            const int64_t u = ball[head];
            nb.clear();
            for (int64_t e = adj_ptr[lo + u]; e < adj_ptr[lo + u + 1]; ++e) {
                const int32_t v = (int32_t)(adj[e] - lo);
                if (!placed[v]) nb.push_back(v);
            }
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return perm[lo + a] < perm[lo + b];
            });
            nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
            for (int32_t v : nb) {
                if (ball.size() >= (size_t)kClusterRows) break;
                placed[v] = 1;
                ball.push_back(v);
            }
        }
        std::sort(ball.begin(), ball.end(), [&](int32_t a, int32_t b) {
            return perm[lo + a] < perm[lo + b];
        });
        out.insert(out.end(), ball.begin(), ball.end());
    }
    for (int64_t k = 0; k < n; ++k) perm[lo + out[k]] = (int32_t)k;
}

}  // namespace

void tbpm::set_thread_error(const std::string &m) { g_last_error = m; }

// ---------------------------------------------------------------------------

extern "C" int tbpm_version(void) { return 10200; }

extern "C" int tbpm_kernel_binary_version(int *version)
{
    if (!version) return fail(nullptr, TBPM_E_INVALID_ARG, "version is NULL");
    cudaError_t e = kernel_binary_version(version);
    if (e != cudaSuccess)
        return fail(nullptr, TBPM_E_CUDA, std::string("cudaFuncGetAttributes: ") + cudaGetErrorString(e));
    return TBPM_OK;
}

extern "C" const char *tbpm_last_error(const tbpm_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

extern "C" int tbpm_create(tbpm_ctx **out, int device, void *stream)
{
    if (!out) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx pointer is NULL");
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || n_dev == 0)
        return fail(nullptr, TBPM_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (device < 0 || device >= n_dev)
        return fail(nullptr, TBPM_E_INVALID_ARG, "device index out of range");
    tbpm_ctx *c = new tbpm_ctx();
    c->device = device;
    c->user = (cudaStream_t)stream;
    memset(&c->stats, 0, sizeof(c->stats));
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_renorm, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        std::string m = std::string("context setup: ") + cudaGetErrorString(e);
        tbpm_destroy(c);
        return fail(nullptr, TBPM_E_CUDA, m);
    }
    *out = c;
    return TBPM_OK;
}

extern "C" void tbpm_destroy(tbpm_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->st) cudaStreamSynchronize(c->st);
    free_hamiltonian(c);
    cudaFree(c->d_flags);
    cudaFree(c->d_renorm);
    for (auto e : c->events) cudaEventDestroy(e);
    if (c->st) cudaStreamDestroy(c->st);
    delete c;
}

extern "C" int tbpm_build_hamiltonian(tbpm_ctx *c, int64_t n_orb, const double *onsite,
                                      int64_t n_hop, const int64_t *hop_i,
                                      const int64_t *hop_j, const double *hop_v, double s,
                                      int n_samples, const int64_t *sample_offsets, int where,
                                      int flags)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (n_orb < 1 || n_orb > INT32_MAX - (int64_t)kChunkRows * 64)
        return fail(c, TBPM_E_INVALID_ARG, "n_orb out of range");
    if (n_hop < 0 || (n_hop > 0 && (!hop_i || !hop_j || !hop_v)))
        return fail(c, TBPM_E_INVALID_ARG, "bond arrays missing");
    if (!(s > 0.0) || !std::isfinite(s)) return fail(c, TBPM_E_INVALID_ARG, "s must be > 0");
    if (n_samples < 1 || (n_samples > 1 && !sample_offsets))
        return fail(c, TBPM_E_INVALID_ARG, "bad sample description");
    if (where != TBPM_HOST && where != TBPM_DEVICE)
        return fail(c, TBPM_E_INVALID_ARG, "where must be TBPM_HOST or TBPM_DEVICE");
    if ((flags & TBPM_BUILD_NO_FP64) && (flags & TBPM_BUILD_NO_FP32))
        return fail(c, TBPM_E_INVALID_ARG, "both value precisions dropped");
    std::vector<int64_t> off(n_samples + 1);
    if (sample_offsets) {
        for (int k = 0; k <= n_samples; ++k) off[k] = sample_offsets[k];
    } else {
        off[0] = 0;
        off[1] = n_orb;
    }
    if (off[0] != 0 || off[n_samples] != n_orb)
        return fail(c, TBPM_E_INVALID_ARG, "sample offsets must run from 0 to n_orb");
    for (int k = 0; k < n_samples; ++k)
        if (off[k + 1] <= off[k]) return fail(c, TBPM_E_INVALID_ARG, "empty or unsorted sample");
    int rc = enter(c);
    if (rc) return rc;
    free_hamiltonian(c);

    std::vector<int64_t> row_off(n_samples + 1, 0);
    for (int k = 0; k < n_samples; ++k) {
        int64_t n_k = off[k + 1] - off[k];
        row_off[k + 1] = row_off[k] + (n_k + kChunkRows - 1) / kChunkRows * kChunkRows;
    }
    if (row_off[n_samples] > INT32_MAX) return fail(c, TBPM_E_INVALID_ARG, "too many rows");

    // optional reverse Cuthill-McKee order per sample (host)
    std::vector<int32_t> perm;
    if (flags & (TBPM_BUILD_REORDER_RCM | TBPM_BUILD_REORDER_CLUSTER)) {
        std::vector<int64_t> hi(n_hop), hj(n_hop);
        if (where == TBPM_DEVICE) {
            CUDA_OR_FAIL(c, cudaMemcpy(hi.data(), hop_i, n_hop * sizeof(int64_t), cudaMemcpyDeviceToHost));
            CUDA_OR_FAIL(c, cudaMemcpy(hj.data(), hop_j, n_hop * sizeof(int64_t), cudaMemcpyDeviceToHost));
        } else {
            memcpy(hi.data(), hop_i, n_hop * sizeof(int64_t));
            memcpy(hj.data(), hop_j, n_hop * sizeof(int64_t));
        }
        std::vector<int64_t> ptr(n_orb + 1, 0);
        for (int64_t b = 0; b < n_hop; ++b) {
            if (hi[b] < 0 || hi[b] >= n_orb || hj[b] < 0 || hj[b] >= n_orb)
                return fail(c, TBPM_E_INVALID_ARG, "invalid bond list: index out of range");
            ++ptr[hi[b] + 1];
            ++ptr[hj[b] + 1];
        }
        for (int64_t u = 0; u < n_orb; ++u) ptr[u + 1] += ptr[u];
        std::vector<int32_t> adj(ptr[n_orb]);
        std::vector<int64_t> fillp(ptr.begin(), ptr.end() - 1);
        for (int64_t b = 0; b < n_hop; ++b) {
            adj[fillp[hi[b]]++] = (int32_t)hj[b];
            adj[fillp[hj[b]]++] = (int32_t)hi[b];
        }
        for (int k = 0; k < n_samples; ++k)
            for (int64_t u = off[k]; u < off[k + 1]; ++u)
                for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e)
                    if (adj[e] < off[k] || adj[e] >= off[k + 1])
                        return fail(c, TBPM_E_INVALID_ARG, "invalid bond list: bond joins two samples");
        perm.assign(n_orb, 0);
        for (int k = 0; k < n_samples; ++k) {
            rcm_sample(off[k], off[k + 1], ptr, adj, perm);
            if (flags & TBPM_BUILD_REORDER_CLUSTER) cluster_sample(off[k], off[k + 1], ptr, adj, perm);
        }
    }

    // stage inputs on the device
    const double *d_on = nullptr, *d_hv = nullptr;
    const int64_t *d_hi = nullptr, *d_hj = nullptr;
    bool o1, o2, o3, o4;
    rc = stage(c, onsite, n_orb, where, const_cast<double **>(&d_on), &o1);
    if (!rc) rc = stage(c, hop_i, n_hop, where, const_cast<int64_t **>(&d_hi), &o2);
    if (!rc) rc = stage(c, hop_j, n_hop, where, const_cast<int64_t **>(&d_hj), &o3);
    const bool cplx = (flags & TBPM_BUILD_COMPLEX_HOPS) != 0;
    if (!rc) rc = stage(c, hop_v, (size_t)n_hop * (cplx ? 2 : 1), where,
                        const_cast<double **>(&d_hv), &o4);
    int64_t *d_off = nullptr, *d_row_off = nullptr;
    int32_t *d_perm = nullptr;
    if (!rc) rc = dalloc(c, &d_off, n_samples + 1);
    if (!rc) rc = dalloc(c, &d_row_off, n_samples + 1);
    if (!rc && !perm.empty()) rc = dalloc(c, &d_perm, n_orb);
    auto release = [&]() {
        if (o1) cudaFree((void *)d_on);
        if (o2) cudaFree((void *)d_hi);
        if (o3) cudaFree((void *)d_hj);
        if (o4) cudaFree((void *)d_hv);
        cudaFree(d_off);
        cudaFree(d_row_off);
        cudaFree(d_perm);
    };
    if (rc) { release(); return rc; }
    cudaMemcpyAsync(d_off, off.data(), (n_samples + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(d_row_off, row_off.data(), (n_samples + 1) * sizeof(int64_t),
                    cudaMemcpyHostToDevice, c->st);
    if (d_perm)
        cudaMemcpyAsync(d_perm, perm.data(), n_orb * sizeof(int32_t), cudaMemcpyHostToDevice, c->st);

    BuildInput in;
    in.n_orb = n_orb;
    in.onsite = d_on;
    in.n_hop = n_hop;
    in.hop_i = d_hi;
    in.hop_j = d_hj;
    in.hop_v = d_hv;
    in.inv_s = 1.0 / s;
    in.n_samples = n_samples;
    in.d_sample_off = d_off;
    in.d_sample_row_off = d_row_off;
    in.d_perm = d_perm;
    in.cplx = cplx ? 1 : 0;
    std::string msg;
    rc = build_sell(in, !(flags & TBPM_BUILD_NO_FP64), !(flags & TBPM_BUILD_NO_FP32),
                    !(flags & TBPM_BUILD_NO_UNIFORM), !(flags & TBPM_BUILD_NO_BOND_MAP), c->H,
                    c->st, msg);
    cudaStreamSynchronize(c->st);
    release();
    if (rc) {
        free_build(c->H);
        return fail(c, rc, msg);
    }
    c->n_orb = n_orb;
    c->n_samples = n_samples;
    c->s = s;
    c->sample_off = off;
    c->row_off = row_off;
    std::vector<int64_t> chunk_off(n_samples + 1);
    std::vector<double> inv_sqrt(n_samples);
    for (int k = 0; k <= n_samples; ++k) chunk_off[k] = row_off[k] / kChunkRows;
    for (int k = 0; k < n_samples; ++k) inv_sqrt[k] = 1.0 / sqrt((double)(off[k + 1] - off[k]));
    rc = dalloc(c, &c->d_sample_chunk_off, n_samples + 1);
    if (!rc) rc = dalloc(c, &c->d_inv_sqrt_n, n_samples);
    if (!rc) rc = dalloc(c, &c->d_step, n_samples);
    if (rc) { free_hamiltonian(c); return rc; }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_sample_chunk_off, chunk_off.data(),
                                    (n_samples + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_inv_sqrt_n, inv_sqrt.data(), n_samples * sizeof(double),
                                    cudaMemcpyHostToDevice, c->st));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));
    c->have_h = true;
    c->stats.gershgorin = c->H.gershgorin;
    c->stats.n_rows = c->H.n_rows;
    c->stats.nnz = c->H.nnz_pad;
    c->stats.nnz_true = c->H.nnz_true;
    if ((flags & TBPM_BUILD_STRICT_BOUND) && c->H.gershgorin > 1.0) {
        char buf[160];
        snprintf(buf, sizeof buf, "Gershgorin bound of H is %.6g eV, above s = %.6g eV",
                 c->H.gershgorin * s, s);
        free_hamiltonian(c);
        return fail(c, TBPM_E_SPECTRAL_BOUND, buf);
    }
    c->stats.lanczos_radius = 0.0;
    if (!(flags & TBPM_BUILD_NO_SPECTRAL_CHECK) && c->H.gershgorin > 1.0 / 1.01) {
        // the Gershgorin bound does not clear s: estimate the spectral radius
        double lo = 0, hi = 0;
        int steps = 0;
        std::string msg;
        rc = lanczos_extremes(c->H, kLanczosSteps, c->st, &lo, &hi, &steps, msg);
        if (rc) { free_hamiltonian(c); return fail(c, rc, msg); }
        const double rho = std::max(std::fabs(lo), std::fabs(hi));
        c->stats.lanczos_radius = rho;
        if (1.01 * rho > 1.0) {
            char buf[240];
            snprintf(buf, sizeof buf,
                     "s = %.6g eV is below 1.01 x the Lanczos estimate %.6g eV of the spectral "
                     "radius of H (extreme Ritz values %.6g, %.6g eV): the Chebyshev series "
                     "would diverge",
                     s, rho * s, lo * s, hi * s);
            free_hamiltonian(c);
            return fail(c, TBPM_E_SPECTRAL_BOUND, buf);
        }
    }
    c->err.clear();
    return leave(c);
}

static int set_states_common(tbpm_ctx *c, int n_states, const double *src, int where,
                             bool phases)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h) return fail(c, TBPM_E_STATE, "build the Hamiltonian first");
    if (n_states < 1 || n_states > kMaxStates || !src)
        return fail(c, TBPM_E_INVALID_ARG, "n_states must be 1..64 with data");
    if (where != TBPM_HOST && where != TBPM_DEVICE)
        return fail(c, TBPM_E_INVALID_ARG, "where must be TBPM_HOST or TBPM_DEVICE");
    int rc = enter(c);
    if (rc) return rc;
    free_groups(c);
    cudaFree(c->d_psi_user);
    c->d_psi_user = nullptr;
    c->n_states = 0;
    const size_t count = (size_t)n_states * c->n_orb;
    rc = dalloc(c, &c->d_psi_user, count);
    if (rc) return rc;
    if (phases) {
        const double *d_theta = nullptr;
        bool owned = false;
        rc = stage(c, src, count, where, const_cast<double **>(&d_theta), &owned);
        if (rc) return rc;
        CUDA_OR_FAIL(c, launch_phase_user(d_theta, c->n_orb, n_states, c->d_inv_sqrt_n,
                                          c->H.orb_sample, c->d_psi_user, c->st));
        if (owned) {
            cudaStreamSynchronize(c->st);
            cudaFree((void *)d_theta);
        }
    } else {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_psi_user, src, count * sizeof(double2),
                                        where == TBPM_HOST ? cudaMemcpyHostToDevice
                                                           : cudaMemcpyDeviceToDevice,
                                        c->st));
    }
    c->n_states = n_states;
    c->err.clear();
    return leave(c);
}

extern "C" int tbpm_spectral_bounds(tbpm_ctx *c, int n_iter, double *e_min, double *e_max,
                                    int *steps)
{
    if (!c || !e_min || !e_max) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    if (!c->have_h) return fail(c, TBPM_E_STATE, "build the Hamiltonian first");
    if (n_iter < 1 || n_iter > 10000) return fail(c, TBPM_E_INVALID_ARG, "n_iter must be 1..10000");
    int rc = enter(c);
    if (rc) return rc;
    double lo = 0, hi = 0;
    int m = 0;
    std::string msg;
    rc = lanczos_extremes(c->H, n_iter, c->st, &lo, &hi, &m, msg);
    if (rc) return fail(c, rc, msg);
    *e_min = lo * c->s;
    *e_max = hi * c->s;
    if (steps) *steps = m;
    c->err.clear();
    return leave(c);
}

extern "C" int tbpm_set_states(tbpm_ctx *c, int n_states, const double *psi0, int where)
{
    return set_states_common(c, n_states, psi0, where, false);
}

extern "C" int tbpm_set_phase_states(tbpm_ctx *c, int n_states, const double *theta, int where)
{
    return set_states_common(c, n_states, theta, where, true);
}

extern "C" int tbpm_set_launch_config(tbpm_ctx *c, int precision, int max_group, int threads,
                                      int variant)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (precision != TBPM_FP64 && precision != TBPM_FP32)
        return fail(c, TBPM_E_INVALID_ARG, "bad precision");
    const int cap = precision == TBPM_FP64 ? 8 : 16;
    if (max_group < 1 || max_group > cap || (max_group & (max_group - 1)))
        return fail(c, TBPM_E_INVALID_ARG, "group width must be a power of two within the cap");
    if (threads < 64 || threads > 256 || (threads & (threads - 1)))
        return fail(c, TBPM_E_INVALID_ARG, "threads must be 64, 128 or 256");
    if (variant < 0 || variant > (kVariantZigZag | kVariantStreamHints | kVariantTma | kVariantFused |
                                  (3 << kVariantFusedTileShift) | kVariantWide | kVariantSplit2 |
                                  kVariantSplit4 | kVariantHalo | kVariantPipe |
                                  kVariantCluster | kVariantStaged | kVariantPrefetch) ||
        ((variant >> kVariantFusedTileShift) & 3) == 3 ||
        ((variant & kVariantSplit2) && (variant & kVariantSplit4)))
        return fail(c, TBPM_E_INVALID_ARG, "unknown launch variant bits");
    if (c->max_group[precision] != max_group || c->threads[precision] != threads) free_groups(c);
    c->max_group[precision] = max_group;
    c->threads[precision] = threads;
    c->variant[precision] = variant;
    return TBPM_OK;
}

extern "C" int tbpm_set_norm_policy(tbpm_ctx *c, double renorm_fp32, double hard_fp32,
                                    double hard_fp64)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!(renorm_fp32 > 0.0) || !(hard_fp32 > 0.0) || !(hard_fp64 > 0.0))
        return fail(c, TBPM_E_INVALID_ARG, "norm bounds must be > 0");
    c->renorm_fp32 = renorm_fp32;
    c->hard_fp32 = hard_fp32;
    c->hard_fp64 = hard_fp64;
    return TBPM_OK;
}

// Allocate the state groups for `prec`, splitting n_states into power-of-two
// widths no wider than the cap (e.g. 3 -> 2 + 1).
static int ensure_groups(tbpm_ctx *c, int prec)
{
    if (c->prec == prec && !c->groups.empty()) return TBPM_OK;
    free_groups(c);
    const size_t cs = prec == TBPM_FP64 ? 16 : 8;
    int left = c->n_states, s0 = 0;
    while (left > 0) {
        int B = 1;
        while (B * 2 <= left && B * 2 <= c->max_group[prec]) B *= 2;
        Group g;
        g.B = B;
        g.s0 = s0;
        c->groups.push_back(g);
        left -= B;
        s0 += B;
    }
    if ((int)c->groups.size() > kMaxGroups) {
        free_groups(c);
        return fail(c, TBPM_E_UNSUPPORTED, "too many state groups");
    }
    for (auto &g : c->groups) {
        const size_t bytes = (size_t)c->H.n_rows * g.B * cs;
        int rc = dalloc(c, (char **)&g.psi0, bytes);
        for (int k = 0; k < 3 && !rc; ++k) rc = dalloc(c, (char **)&g.buf[k], bytes);
        if (!rc && prec == TBPM_FP32) rc = dalloc(c, &g.scale, (size_t)c->n_samples * g.B);
        if (!rc && prec == TBPM_FP32) rc = dalloc(c, &g.scale_f, (size_t)c->n_samples * g.B);
        if (rc) { free_groups(c); return rc; }
        for (int k = 0; k < 3; ++k) cudaMemsetAsync(g.buf[k], 0, bytes, c->st);
        cudaMemsetAsync(g.psi0, 0, bytes, c->st);
    }
    int maxB = 1;
    for (auto &g : c->groups) maxB = std::max(maxB, g.B);
    const int64_t need = c->H.n_rows / kChunkRows * maxB * 3;
    if (need > c->partial_len) {
        cudaFree(c->d_partial);
        c->d_partial = nullptr;
        int rc = dalloc(c, &c->d_partial, need);
        if (rc) { free_groups(c); return rc; }
        c->partial_len = need;
    }
    // block partials of the closing term: one per block of the launch shape
    int64_t need_b = 0;
    for (auto &g : c->groups) {
        const int L = prec == TBPM_FP64 ? g.B : std::max(1, g.B / 2);
        need_b = std::max<int64_t>(need_b, c->H.n_rows * L / 128 * g.B * 3);   // closing-term blocks of 128
    }
    if (need_b > c->block_partial_len) {
        cudaFree(c->d_block_partial);
        c->d_block_partial = nullptr;
        int rc = dalloc(c, &c->d_block_partial, need_b);
        if (rc) { free_groups(c); return rc; }
        c->block_partial_len = need_b;
    }
    if (!c->d_chunk_count) {
        int rc = dalloc(c, &c->d_chunk_count, c->H.n_rows / kChunkRows);
        if (rc) { free_groups(c); return rc; }
        cudaMemsetAsync(c->d_chunk_count, 0, c->H.n_rows / kChunkRows * sizeof(int), c->st);
    }
    if (!c->d_partial2) {
        int rc = dalloc(c, &c->d_partial2, (size_t)c->n_samples * 64 * 16 * 3);
        if (!rc) rc = dalloc(c, &c->d_sample_ticket, (size_t)c->n_samples);
        if (rc) { free_groups(c); return rc; }
        cudaMemsetAsync(c->d_sample_ticket, 0, c->n_samples * sizeof(unsigned int), c->st);
    }
    c->prec = prec;
    return TBPM_OK;
}

namespace {

struct Slot {
    int buf;      // buffer index holding the stored part, or -1
    double beta;  // plus beta * psi
};

struct Launch {
    bool final_term;
    int x, z, out;   // buffer indices; x == -1 means psi
    double c, gamma;
    bool interior;   // full term: gathered buffer x, z present
};

// Clenshaw schedule of one step for M coefficients a[0..M-1], given the
// buffer `cur` that holds psi.  b_{M-1} = a_{M-1} psi is never stored.
std::vector<Launch> schedule(const std::vector<double> &a, int cur, int *next_cur)
{
    const int M = (int)a.size();
    std::vector<Slot> b(M + 2, Slot{-1, 0.0});
    b[M - 1] = Slot{-1, a[M - 1]};
    int scratch[2], ns = 0;
    for (int k = 0; k < 3; ++k)
        if (k != cur) scratch[ns++] = k;
    std::vector<Launch> out;
    for (int m = M - 2; m >= 0; --m) {
        const Slot x = b[m + 1], zz = b[m + 2];
        Launch L;
        L.final_term = (m == 0);
        const double g = L.final_term ? 1.0 : 2.0;
        if (x.buf < 0) {
            L.x = -1;
            L.gamma = g * x.beta;
        } else {
            L.x = x.buf;
            L.gamma = g;
        }
        L.c = a[m] + zz.beta;
        L.z = zz.buf;
        if (zz.buf >= 0)
            L.out = zz.buf;
        else
            L.out = (scratch[0] != x.buf) ? scratch[0] : scratch[1];
        L.interior = !L.final_term && x.buf >= 0 && zz.buf >= 0;
        out.push_back(L);
        b[m] = Slot{L.out, 0.0};
    }
    *next_cur = out.back().out;
    return out;
}

// FP64 one-value form of one term: gh = gamma h (rounded once, here), and
// gamma d read from d or 2 d with a sign bit when that is exact (|gamma| of
// 1 or 2: the closing and interior terms), else multiplied on the device.
void one_value_terms(const BuildOutput &H, double gamma, double *gh, const double **gdiag,
                     unsigned long long *sign)
{
    *gh = gamma * H.h_uniform;
    *gdiag = nullptr;
    *sign = gamma < 0 ? (1ull << 63) : 0ull;
    const double ag = fabs(gamma);
    if (ag == 1.0) *gdiag = H.diag64;
    else if (ag == 2.0) *gdiag = H.diag2_64;
}

void one_value_table(const BuildOutput &H, FusedTerm &ft)
{
    const double *gd = nullptr;
    one_value_terms(H, ft.gamma, &ft.gh, &gd, &ft.gd_sign);
    const double ag = fabs(ft.gamma);
    ft.gd_sel = ag == 2.0 ? 2 : ag == 1.0 ? 1 : 0;
}

void split_coeff(double c, int fp32, double *hi, double *lo)
{
    if (fp32) {
        float h = (float)c;
        *hi = (double)h;
        *lo = (double)(float)(c - (double)h);
    } else {
        *hi = c;
        *lo = 0.0;
    }
}

}  // namespace

// Item table of the wavefront-fused step: every (term j, tile t) ordered by
// the key t + j D with D = radius + 1 + lag, so each item's dependencies --
// (j-1, t') for |t' - t| <= radius -- come earlier; items of equal key are
// independent.  The extra lag (twice the grid's blocks per term) lets term
// j-1 run far enough ahead that an item's dependencies are normally finished
// by the time it is handed out, so the resident blocks do not queue behind
// one another.
static int ensure_fused(tbpm_ctx *c, int J, int R, int radius, int maxB, int grid)
{
    const int64_t T = c->H.n_rows / R;
    if (T >= ((int64_t)1 << 25) || J >= 128)
        return fail(c, TBPM_E_UNSUPPORTED, "fused step: too many tiles or terms");
    const int D = radius + 1 + (2 * grid + J - 1) / J;
    if (c->items_key[0] != J || c->items_key[1] != R || c->items_key[2] != D) {
        std::vector<int32_t> items;
        items.reserve((size_t)J * T);
        const int64_t kmax = (T - 1) + (int64_t)(J - 1) * D;
        for (int64_t k = 0; k <= kmax; ++k)
            for (int j = 0; j < J; ++j) {
                const int64_t t = k - (int64_t)j * D;
                if (t >= 0 && t < T) items.push_back((int32_t)(((uint32_t)j << 25) | (uint32_t)t));
            }
        cudaFree(c->d_items);
        c->d_items = nullptr;
        int rc = dalloc(c, &c->d_items, items.size());
        if (rc) return rc;
        CUDA_OR_FAIL(c, cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice));
        c->items_len = (int64_t)items.size();
        c->items_key[0] = J;
        c->items_key[1] = R;
        c->items_key[2] = D;
    }
    if (c->done_len < (int64_t)J * T) {
        cudaFree(c->d_done);
        c->d_done = nullptr;
        int rc = dalloc(c, &c->d_done, (size_t)J * T);
        if (rc) return rc;
        c->done_len = (int64_t)J * T;
    }
    if (!c->d_fcounter) {
        int rc = dalloc(c, &c->d_fcounter, 1);
        if (!rc) rc = dalloc(c, &c->d_fterms, 3 * (size_t)kMaxTerms);
        if (rc) return rc;
    }
    if (c->tile_partial_len < T * maxB * 3) {
        cudaFree(c->d_tile_partial);
        c->d_tile_partial = nullptr;
        int rc = dalloc(c, &c->d_tile_partial, (size_t)T * maxB * 3);
        if (rc) return rc;
        c->tile_partial_len = T * maxB * 3;
    }
    return TBPM_OK;
}

static int get_events(tbpm_ctx *c, size_t n)
{
    while (c->events.size() < n) {
        cudaEvent_t e;
        CUDA_OR_FAIL(c, cudaEventCreate(&e));
        c->events.push_back(e);
    }
    return TBPM_OK;
}

extern "C" int tbpm_propagate(tbpm_ctx *c, double z, int n_steps, int precision,
                              double *corr_out, int where_out, int flags)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    if (precision != TBPM_FP64 && precision != TBPM_FP32)
        return fail(c, TBPM_E_INVALID_ARG, "precision must be TBPM_FP64 or TBPM_FP32");
    if (n_steps < 0) return fail(c, TBPM_E_INVALID_ARG, "n_steps < 0");
    if (corr_out && where_out != TBPM_HOST && where_out != TBPM_DEVICE)
        return fail(c, TBPM_E_INVALID_ARG, "bad where_out");
    const int fp32 = precision == TBPM_FP32;
    if ((fp32 && !c->H.val32) || (!fp32 && !c->H.val64))
        return fail(c, TBPM_E_STATE, "the Hamiltonian was built without this precision");
    const bool resume = (flags & TBPM_PROP_RESUME) != 0;
    if (resume && (!c->have_run || c->prec != precision))
        return fail(c, TBPM_E_STATE, "nothing to resume in this precision");
    const bool profile = (flags & TBPM_PROP_PROFILE) != 0;
    const bool graph = (flags & TBPM_PROP_GRAPH) != 0 && !profile;
    const bool fused = !c->H.cplx && ((c->variant[precision] & kVariantFused) != 0 ||
                                      (flags & TBPM_PROP_PERSISTENT) != 0);
    const double tsign = (flags & TBPM_PROP_BACKWARD) ? -1.0 : 1.0;   // e^{+iH tau} per step
    if (c->H.cplx && (flags & TBPM_PROP_PERSISTENT))
        return fail(c, TBPM_E_UNSUPPORTED, "the fused step takes real hoppings only");

    std::vector<double> J(kMaxTerms);
    int M = 0;
    if (bessel_miller(z, 1e-15, kMaxTerms, J.data(), &M) != TBPM_OK || M < 2)
        return fail(c, TBPM_E_INVALID_ARG, "z out of range for the coefficient table");
    std::vector<double> a(M);
    a[0] = J[0];
    for (int m = 1; m < M; ++m) a[m] = 2.0 * J[m];

    int rc = enter(c);
    if (rc) return rc;
    rc = ensure_groups(c, precision);
    if (rc) return rc;
    if (c->corr_steps != n_steps) {
        free_outputs(c);
        const size_t cnt = (size_t)c->n_samples * c->n_states * (n_steps + 1);
        rc = dalloc(c, &c->d_corr, cnt);
        if (!rc) rc = dalloc(c, &c->d_norms, cnt);
        if (rc) return rc;
        c->corr_steps = n_steps;
    }
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), c->st));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_renorm, 0, sizeof(unsigned long long), c->st));
    {
        const int64_t need = (int64_t)c->n_samples * c->n_states;
        if (need > c->norm_ref_len) {
            if (resume) return fail(c, TBPM_E_STATE, "nothing to resume for these states");
            cudaFree(c->d_norm_ref);
            c->d_norm_ref = nullptr;
            c->norm_ref_len = 0;
            rc = dalloc(c, &c->d_norm_ref, need);
            if (rc) return rc;
            c->norm_ref_len = need;
        }
    }
    if (c->ac_on && (!c->d_ac_corr || !c->d_ac_partial || !c->d_bond_dx))
        return fail(c, TBPM_E_STATE, "AC buffers missing");

    const size_t cs = fp32 ? 8 : 16;
    const int threads = c->threads[precision];
    // staged-gather variant: halo lists built on first use; a matrix whose
    // row blocks reference too many other rows keeps the plain kernels
    bool halo = (c->variant[precision] & kVariantHalo) && !c->H.cplx &&
                !(c->variant[precision] & (kVariantTma | kVariantFused));
    if (halo && !c->H.halo_ptr) {
        std::string msg;
        rc = build_halo(c->H, c->st, msg);
        if (rc == TBPM_E_UNSUPPORTED) halo = false;
        else if (rc) return fail(c, rc, msg);
    }
    if (halo && (c->variant[precision] & (kVariantPipe | kVariantStaged)) && !c->H.uniform &&
        !c->H.vpack[fp32]) {
        std::string msg;
        rc = build_packed_values(c->H, fp32, c->st, msg);
        if (rc) return fail(c, rc, msg);
    }
    // FP64 one-value form: 2 d for the interior terms' gamma d
    if (!fp32 && c->H.uniform && !c->H.zero_diag && !c->H.diag2_64) {
        std::string msg;
        rc = build_diag2(c->H, c->st, msg);
        if (rc) return fail(c, rc, msg);
    }
    SellView Hv;
    Hv.slice_ptr = c->H.slice_ptr;
    Hv.col = c->H.col;
    Hv.val = fp32 ? (const void *)c->H.val32 : (const void *)c->H.val64;
    Hv.diag = fp32 ? (const void *)c->H.diag32 : (const void *)c->H.diag64;

    const size_t ev_per_step = 5;
    if (profile) {
        rc = get_events(c, (size_t)(n_steps + 1) * ev_per_step * c->groups.size() + 2);
        if (rc) return rc;
    }
    int64_t launches = 0;
    size_t ev_used = 0;
    cudaEvent_t ev_all0 = nullptr, ev_all1 = nullptr;
    if (profile) {
        ev_all0 = c->events[ev_used++];
        ev_all1 = c->events[ev_used++];
        CUDA_OR_FAIL(c, cudaEventRecord(ev_all0, c->st));
    }
    std::vector<size_t> step_ev;   // index of the first of 5 events per profiled step
    bool cluster_run = false;      // the cluster-resident stepping ran (one launch)

    for (auto &g : c->groups) {
        const size_t bytes = (size_t)c->H.n_rows * g.B * cs;
        if (!resume) {
            CUDA_OR_FAIL(c, launch_set_states(c->d_psi_user, c->n_orb, c->n_states,
                                              c->H.user_to_row, g.s0, g.B, fp32, g.psi0, c->st));
            CUDA_OR_FAIL(c, cudaMemcpyAsync(g.buf[0], g.psi0, bytes, cudaMemcpyDeviceToDevice, c->st));
            g.cur = 0;
            launches += 1;
        }
        for (int k = 0; k < 3; ++k)
            if (g.graph[k]) { cudaGraphExecDestroy(g.graph[k]); g.graph[k] = nullptr; }
        if (g.scale) {
            std::vector<double> ones((size_t)c->n_samples * g.B, 1.0);
            std::vector<float> ones_f((size_t)c->n_samples * g.B, 1.0f);
            CUDA_OR_FAIL(c, cudaMemcpyAsync(g.scale, ones.data(), ones.size() * sizeof(double),
                                            cudaMemcpyHostToDevice, c->st));
            CUDA_OR_FAIL(c, cudaMemcpyAsync(g.scale_f, ones_f.data(), ones_f.size() * sizeof(float),
                                            cudaMemcpyHostToDevice, c->st));
            CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));   // host vectors go out of scope
        }
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_step, 0, c->n_samples * sizeof(int), c->st));

        TermArgs base;
        memset(&base, 0, sizeof(base));
        base.H = Hv;
        base.chunk_sample = c->H.chunk_sample;
        base.n_rows = c->H.n_rows;
        base.uniform = c->H.uniform;
        base.cplx = c->H.cplx;
        base.fixed_width = c->H.fixed_width;
        base.h_uniform = c->H.h_uniform;
        base.h_uniform_f = (float)c->H.h_uniform;
        base.zero_diag = c->H.zero_diag;
        base.psi0 = g.psi0;
        base.partial = c->d_partial;
        base.block_partial = c->d_block_partial;
        base.chunk_count = c->d_chunk_count;
        if (halo) {
            base.halo_ptr = c->H.halo_ptr;
            base.halo_rows = c->H.halo_rows;
            base.lcol = c->H.lcol;
            base.pslice = c->H.pslice;
            base.vpack = c->H.vpack[fp32];
            base.halo_max = c->H.halo_max;
            base.halo_ent_max = c->H.halo_ent_max;
        }
        base.num_sms = c->num_sms;                  // grid of the persistent term kernels
        ReduceArgs ra;
        ra.partial = c->d_partial;
        ra.partial2 = c->d_partial2;
        ra.sample_ticket = c->d_sample_ticket;
        ra.sample_chunk_off = c->d_sample_chunk_off;
        ra.n_samples = c->n_samples;
        ra.B = g.B;
        ra.group_state0 = g.s0;
        ra.n_states = c->n_states;
        ra.n_steps = n_steps;
        ra.step = c->d_step;
        ra.corr = c->d_corr;
        ra.norms = c->d_norms;
        ra.renorm_bound = c->renorm_fp32;
        ra.hard_bound = fp32 ? c->hard_fp32 : c->hard_fp64;
        ra.renorm_count = c->d_renorm;
        ra.error_flags = c->d_flags;
        ra.norm_ref = c->d_norm_ref;
        ra.set_ref = 0;

        // AC-conductivity observer on the state buffer `bi` (after the reduction
        // of the same step, whose counter it reads)
        auto observe = [&](int bi) -> int {
            if (c->qe_on) {
                QeArgs qa;
                qa.psi = g.buf[bi];
                qa.scale = fp32 ? g.scale : nullptr;
                qa.chunk_sample = c->H.chunk_sample;
                qa.step = c->d_step;
                qa.coef = c->d_qe_coef;
                qa.coef_f = c->d_qe_coef_f;
                qa.scale_f = fp32 ? g.scale_f : nullptr;
                qa.acc = c->d_qe_acc;
                qa.n_rows = c->H.n_rows;
                qa.B = g.B;
                qa.s0 = g.s0;
                qa.S = c->n_states;
                qa.K = c->qe_K;
                CUDA_OR_FAIL(c, launch_qe_acc(qa, fp32, c->st));
            }
            if (!c->ac_on) return TBPM_OK;
            AcArgs oa;
            oa.H = Hv;
            oa.dx = c->d_bond_dx;
            oa.dy = c->d_bond_dy;
            oa.dx32 = c->d_bond_dx32;
            oa.dy32 = c->d_bond_dy32;
            oa.scale_f = fp32 ? g.scale_f : nullptr;
            oa.psi = g.buf[bi];
            oa.scale = fp32 ? g.scale : nullptr;
            oa.chunk_sample = c->H.chunk_sample;
            oa.n_rows = c->H.n_rows;
            oa.B = g.B;
            oa.block_partial = c->d_ac_partial;
            CUDA_OR_FAIL(c, launch_ac_observe(oa, fp32, c->H.cplx, c->st));
            AcReduceArgs ar;
            ar.block_partial = c->d_ac_partial;
            ar.sample_chunk_off = c->d_sample_chunk_off;
            ar.n_samples = c->n_samples;
            ar.B = g.B;
            ar.group_state0 = g.s0;
            ar.n_states = c->n_states;
            ar.n_steps = n_steps;
            ar.step = c->d_step;
            ar.s = c->s;
            ar.corr_ac = c->d_ac_corr;
            CUDA_OR_FAIL(c, launch_ac_reduce(ar, c->st));
            return TBPM_OK;
        };

        // wavefront-fused step: item table, flags and the term tables of the
        // three buffer rotations
        FusedArgs fa;
        memset(&fa, 0, sizeof(fa));
        if (fused) {
            int R = fused_tile_rows(fp32, g.B, (c->variant[precision] >> kVariantFusedTileShift) & 3);
            while (R > kChunkRows && c->H.n_rows % R) R /= 4;   // tiles must cover the rows exactly
            const int radius = (int)((c->H.bandwidth + R - 1) / R);
            int maxB = 1;
            for (auto &g2 : c->groups) maxB = std::max(maxB, g2.B);
            rc = ensure_fused(c, M - 1, R, radius, maxB, fused_grid(fp32, g.B, c->num_sms));
            if (rc) return rc;
            std::vector<FusedTerm> tabs(3 * (size_t)kMaxTerms);
            for (int cur0 = 0; cur0 < 3; ++cur0) {
                int nx = 0;
                std::vector<Launch> sch = schedule(a, cur0, &nx);
                for (size_t k = 0; k < sch.size(); ++k) {
                    FusedTerm &ft = tabs[cur0 * kMaxTerms + k];
                    ft.x = sch[k].x;
                    ft.z = sch[k].z;
                    ft.out = sch[k].out;
                    ft.final_term = sch[k].final_term ? 1 : 0;
                    split_coeff(sch[k].c, fp32, &ft.c_hi, &ft.c_lo);
                    ft.gamma = tsign * sch[k].gamma;
                    ft.c_hi_f = (float)ft.c_hi;
                    ft.c_lo_f = (float)ft.c_lo;
                    ft.gamma_f = (float)ft.gamma;
                    one_value_table(c->H, ft);
                }
            }
            CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_fterms, tabs.data(), tabs.size() * sizeof(FusedTerm),
                                            cudaMemcpyHostToDevice, c->st));
            CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_done, 0, (size_t)(M - 1) * (c->H.n_rows / R) * sizeof(int),
                                            c->st));
            CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));    // host table goes out of scope
            fa.H = Hv;
            fa.uniform = c->H.uniform;
            fa.zero_diag = c->H.zero_diag;
            fa.diag2 = c->H.diag2_64;
            fa.psi0 = g.psi0;
            for (int k = 0; k < 3; ++k) fa.bufs[k] = g.buf[k];
            fa.items = c->d_items;
            fa.n_items = c->items_len;
            fa.n_tiles = c->H.n_rows / R;
            fa.tile_rows = R;
            fa.radius = radius;
            fa.done = c->d_done;
            fa.counter = c->d_fcounter;
            fa.epoch_ptr = c->d_step;
            fa.err = c->d_flags;
            fa.scale = g.scale;
            fa.scale_f = g.scale_f;
            fa.chunk_sample = c->H.chunk_sample;
            fa.tile_partial = c->d_tile_partial;
            fa.partial = c->d_partial;
            fa.chunk_count = c->d_chunk_count;
        }

        // C_0 = <psi0|phi(0)>
        {
            TermArgs t0 = base;
            t0.H.col = nullptr;
            t0.out = g.buf[g.cur];
            CUDA_OR_FAIL(c, launch_final(t0, fp32, g.B, threads, c->st));
            ra.scale = nullptr;
            ra.scale_f = nullptr;
            ra.set_ref = resume ? 0 : 1;
            CUDA_OR_FAIL(c, launch_reduce(ra, c->st));
            ra.set_ref = 0;
            launches += 2;
            rc = observe(g.cur);
            if (rc) return rc;
            if (c->ac_on) launches += 2;
            if (c->qe_on) launches += 1;
        }
        ra.scale = g.scale;
        ra.scale_f = g.scale_f;

        // cluster-resident stepping: every step of this one FP64 state in one launch
        const int Kc = (c->variant[precision] & kVariantCluster) && !fp32 && !fused &&
                               c->groups.size() == 1 && g.B == 1 && c->n_samples == 1 &&
                               !c->H.cplx && !c->ac_on && !c->qe_on && c->H.val64 &&
                               c->H.max_width <= kClusterMaxW && n_steps > 0 &&
                               M - 1 >= 2 && M - 1 <= kClusterMaxTerms
                           ? cluster_blocks_for(c->H.n_rows, c->H.max_width, c->H.uniform)
                           : 0;
        if (Kc > 0) {
            if (!c->d_fterms) {
                rc = dalloc(c, &c->d_fterms, 3 * (size_t)kMaxTerms);
                if (rc) return rc;
            }
            std::vector<FusedTerm> tabs(3 * (size_t)kMaxTerms);
            ClusterArgs ca;
            memset(&ca, 0, sizeof(ca));
            for (int cur0 = 0; cur0 < 3; ++cur0) {
                int nx = 0;
                std::vector<Launch> sch = schedule(a, cur0, &nx);
                ca.next_cur[cur0] = nx;
                for (size_t k = 0; k < sch.size(); ++k) {
                    FusedTerm &ft = tabs[cur0 * kMaxTerms + k];
                    ft.x = sch[k].x;
                    ft.z = sch[k].z;
                    ft.out = sch[k].out;
                    ft.final_term = sch[k].final_term ? 1 : 0;
                    split_coeff(sch[k].c, 0, &ft.c_hi, &ft.c_lo);
                    ft.gamma = tsign * sch[k].gamma;
                    one_value_table(c->H, ft);
                }
            }
            CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_fterms, tabs.data(), tabs.size() * sizeof(FusedTerm),
                                            cudaMemcpyHostToDevice, c->st));
            ca.col = c->H.col;
            ca.val = c->H.val64;
            ca.diag = c->H.diag64;
            ca.slice_ptr = c->H.slice_ptr;
            ca.fixed_width = c->H.fixed_width;
            ca.uniform = c->H.uniform;
            ca.zero_diag = c->H.zero_diag;
            ca.h_uniform = c->H.h_uniform;
            ca.max_w = std::max(1, c->H.max_width);
            ca.rows_per_cta = (int)(c->H.n_rows / Kc);
            ca.psi0 = (const double2 *)g.psi0;
            for (int k = 0; k < 3; ++k) ca.bufs[k] = (double2 *)g.buf[k];
            ca.cur0 = g.cur;
            ca.terms = c->d_fterms;
            ca.J = M - 1;
            ca.n_steps = n_steps;
            const int64_t idx0 = (int64_t)g.s0 * (n_steps + 1);
            ca.corr = c->d_corr + idx0;
            ca.norms = c->d_norms + idx0;
            ca.norm_ref = c->d_norm_ref + g.s0;
            ca.hard_bound = c->hard_fp64;
            ca.err = c->d_flags;
            size_t e0 = 0;
            if (profile) {
                e0 = ev_used;
                ev_used += ev_per_step;
                step_ev.push_back(e0);
                for (int q = 0; q < 2; ++q) CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + q], c->st));
            }
            cudaError_t e = launch_cluster_steps(ca, Kc, c->st);
            if (e != cudaSuccess)
                return fail(c, TBPM_E_CUDA, std::string("cluster steps: ") + cudaGetErrorString(e));
            if (profile)
                for (int q = 2; q < 5; ++q) CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + q], c->st));
            CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));    // host table goes out of scope
            int cur = g.cur;
            for (int n = 0; n < n_steps; ++n) cur = ca.next_cur[cur];
            g.cur = cur;
            launches += 1;
            cluster_run = true;
            continue;
        }

        int final_extra = 0;            // launches of the closing term beyond one
        auto run_step = [&](int cur, int *next_cur, bool timed) -> int {
            if (fused) {
                schedule(a, cur, next_cur);
                size_t e0 = 0;
                if (timed) {
                    e0 = ev_used;
                    ev_used += ev_per_step;
                    step_ev.push_back(e0);
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0], c->st));
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 1], c->st));
                }
                CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_fcounter, 0, sizeof(unsigned long long), c->st));
                FusedArgs f = fa;
                f.psi = g.buf[cur];
                f.terms = c->d_fterms + (size_t)cur * kMaxTerms;
                cudaError_t e = launch_step_fused(f, fp32, g.B, c->num_sms, c->st);
                if (e != cudaSuccess)
                    return fail(c, TBPM_E_CUDA, std::string("fused step: ") + cudaGetErrorString(e));
                if (timed) {
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 2], c->st));
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 3], c->st));
                }
                CUDA_OR_FAIL(c, launch_reduce(ra, c->st));
                if (timed) CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 4], c->st));
                return observe(*next_cur);
            }
            std::vector<Launch> sch = schedule(a, cur, next_cur);
            size_t e0 = 0;
            if (timed) {
                e0 = ev_used;
                ev_used += ev_per_step;
                step_ev.push_back(e0);
                CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0], c->st));
            }
            bool started_interior = false, ended_interior = false;
            for (size_t k = 0; k < sch.size(); ++k) {
                const Launch &L = sch[k];
                if (timed && L.interior && !started_interior) {
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 1], c->st));
                    started_interior = true;
                }
                if (timed && started_interior && !ended_interior && !L.interior) {
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 2], c->st));
                    ended_interior = true;
                }
                TermArgs t = base;
                t.variant = c->variant[precision];
                // complex values have the plain term kernels only (16-byte lanes)
                if (c->H.cplx) t.variant &= kVariantZigZag | kVariantStreamHints;
                if (!halo) t.variant &= ~kVariantHalo;
                t.reverse = (t.variant & kVariantZigZag) ? (int)(k & 1) : 0;
                t.x = L.x < 0 ? g.buf[cur] : g.buf[L.x];
                t.x_is_psi = L.x < 0;
                t.psi = g.buf[cur];
                t.z = L.z < 0 ? nullptr : g.buf[L.z];
                t.out = g.buf[L.out];
                split_coeff(L.c, fp32, &t.c_hi, &t.c_lo);
                t.gamma = tsign * L.gamma;
                t.c_hi_f = (float)t.c_hi;
                t.c_lo_f = (float)t.c_lo;
                t.gamma_f = (float)t.gamma;
                t.scale = g.scale;
                t.scale_f = g.scale_f;
                one_value_terms(c->H, t.gamma, &t.gh, &t.gdiag, &t.gdiag_sign);
                cudaError_t e;
                if (L.final_term) {
                    int nl = 1;
                    e = launch_final(t, fp32, g.B, threads, c->st, &nl);
                    final_extra = nl - 1;         // a term + reduction-pass closing term
                } else if (t.variant & kVariantTma)
                    e = launch_term_tma(t, fp32, g.B, c->H.max_width, c->d_flags, c->num_sms, c->st);
                else
                    e = launch_term(t, fp32, g.B, threads, c->st);
                if (e != cudaSuccess)
                    return fail(c, TBPM_E_CUDA, std::string("term kernel: ") + cudaGetErrorString(e));
            }
            if (timed) {
                if (!started_interior) {
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 1], c->st));
                }
                if (!ended_interior) {
                    CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 2], c->st));
                }
                CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 3], c->st));
            }
            CUDA_OR_FAIL(c, launch_reduce(ra, c->st));
            if (timed) CUDA_OR_FAIL(c, cudaEventRecord(c->events[e0 + 4], c->st));
            return observe(*next_cur);
        };

        for (int n = 0; n < n_steps; ++n) {
            int nxt = 0;
            if (graph) {
                if (!g.graph[g.cur]) {
                    cudaGraph_t gr;
                    CUDA_OR_FAIL(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
                    int rc2 = run_step(g.cur, &nxt, false);
                    cudaError_t e = cudaStreamEndCapture(c->st, &gr);
                    if (rc2) return rc2;
                    if (e != cudaSuccess)
                        return fail(c, TBPM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
                    e = cudaGraphInstantiate(&g.graph[g.cur], gr, 0);
                    cudaGraphDestroy(gr);
                    if (e != cudaSuccess)
                        return fail(c, TBPM_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
                } else {
                    schedule(a, g.cur, &nxt);
                }
                CUDA_OR_FAIL(c, cudaGraphLaunch(g.graph[g.cur], c->st));
            } else {
                rc = run_step(g.cur, &nxt, profile);
                if (rc) return rc;
            }
            g.cur = nxt;
            launches += fused ? 2 : M + final_extra;   // term kernels (or the fused step) + one reduction
            if (c->ac_on) launches += 2; // observer + its reduction
            if (c->qe_on) launches += 1; // quasi-eigenstate accumulation
        }
    }
    if (profile) CUDA_OR_FAIL(c, cudaEventRecord(ev_all1, c->st));

    // results and checks
    int h_flags[4];
    unsigned long long h_renorm = 0;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h_flags, c->d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, c->st));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&h_renorm, c->d_renorm, sizeof(h_renorm), cudaMemcpyDeviceToHost, c->st));
    const size_t cnt = (size_t)c->n_samples * c->n_states * (n_steps + 1);
    std::vector<double> norms(cnt);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(norms.data(), c->d_norms, cnt * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->st));
    if (corr_out)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(corr_out, c->d_corr, cnt * sizeof(double2),
                                        where_out == TBPM_HOST ? cudaMemcpyDeviceToHost
                                                               : cudaMemcpyDeviceToDevice,
                                        c->st));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));
    c->have_run = true;

    tbpm_stats &S = c->stats;
    S.n_terms = M;
    S.n_steps = n_steps;
    S.n_groups = (int)c->groups.size();
    for (int k = 0; k < 8; ++k) S.group_width[k] = k < S.n_groups ? c->groups[k].B : 0;
    S.renormalisations = (int64_t)h_renorm;
    S.kernel_launches = launches;
    // drift of each state's squared norm relative to its value at the first step
    double md = 0.0;
    for (size_t k = 0; k < cnt; ++k) {
        const double ref = norms[k - k % (n_steps + 1)];
        md = std::max(md, ref > 0.0 ? fabs(norms[k] / ref - 1.0) : norms[k]);
    }
    S.max_norm_drift = md;
    S.ms_total = S.ms_term_avg = S.ms_final_avg = S.ms_reduce_avg = 0.0;
    S.term_launches = 0;
    {
        // algorithmic bytes of one interior term launch over all groups' mean width
        double vb = 0.0;
        for (auto &g : c->groups) vb += (double)c->n_orb * 4.0 * g.B * cs;
        vb /= c->groups.size();
        // matrix: a column (and a value, unless one value serves all) per
        // stored entry, and the diagonal; the staged-gather kernel reads a
        // 16-bit halo position per entry instead of the 32-bit column, plus
        // the halo lists
        const double valb = fp32 ? 4.0 : 8.0;
        bool halo_used = halo;
        for (auto &g : c->groups)
            halo_used = halo_used && halo_launchable(fp32, g.B, false, c->H.halo_max);
        const double idxb = halo_used ? 2.0 : 4.0;
        const double entry = idxb + (c->H.uniform ? 0.0 : valb * (c->H.cplx ? 2 : 1));
        S.bytes_term = vb + (double)c->H.nnz_true * entry + (double)c->n_orb * valb;
        if (halo_used)
            S.bytes_term += 4.0 * (double)c->H.halo_total + 8.0 * (double)(c->H.n_rows / kHaloRows + 1);
        // arithmetic of the same launch (see tbpm_stats)
        double per_row = fp32 ? 8.0 : 6.0, per_entry = c->H.cplx ? 4.0 : 2.0;
        if (!fp32 && c->H.uniform && !c->H.cplx) per_row = c->H.zero_diag ? 2.0 : 4.0;
        S.ops_term = vb / (4.0 * cs * (double)c->n_orb) *
                     (per_row * (double)c->n_orb + per_entry * (double)c->H.nnz_true);
    }
    if (profile) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev_all0, ev_all1);
        S.ms_total = ms;
        double t_int = 0, t_fin = 0, t_red = 0;
        const int n_int = std::max(0, M - 4);
        for (size_t e0 : step_ev) {
            float a1 = 0, a2 = 0, a3 = 0;
            cudaEventElapsedTime(&a1, c->events[e0 + 1], c->events[e0 + 2]);
            cudaEventElapsedTime(&a2, c->events[e0 + 2], c->events[e0 + 3]);
            cudaEventElapsedTime(&a3, c->events[e0 + 3], c->events[e0 + 4]);
            t_int += a1;
            t_fin += a2;
            t_red += a3;
        }
        // fused: the whole step is one launch; report its per-term share;
        // cluster stepping: the whole run is one launch
        S.term_launches = (int64_t)step_ev.size() * (fused ? (M - 1) : n_int);
        if (cluster_run) S.term_launches = (int64_t)n_steps * (M - 1);
        if (S.term_launches) S.ms_term_avg = t_int / S.term_launches;
        if (!step_ev.empty()) {
            S.ms_final_avg = t_fin / step_ev.size();
            S.ms_reduce_avg = t_red / step_ev.size();
        }
    }
    rc = leave(c);
    if (rc) return rc;
    if (h_flags[0] & 4)
        return fail(c, TBPM_E_TIMEOUT, "a bounded wait in the TMA term kernel expired");
    if (h_flags[0] & 2) return fail(c, TBPM_E_NONFINITE, "non-finite value in a state or correlation");
    if (h_flags[0] & 1) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "norm drift %.3g above the hard bound: s = %.6g eV is likely below the "
                 "spectral radius of H (Gershgorin %.6g eV)", md, c->s, c->H.gershgorin * c->s);
        return fail(c, TBPM_E_NORM_DRIFT, buf);
    }
    c->err.clear();
    return TBPM_OK;
}

extern "C" int tbpm_correlation(tbpm_ctx *c, double *out, int where_out)
{
    if (!c || !out) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    if (where_out != TBPM_HOST && where_out != TBPM_DEVICE)
        return fail(c, TBPM_E_INVALID_ARG, "where_out must be TBPM_HOST or TBPM_DEVICE");
    if (!c->have_run) return fail(c, TBPM_E_STATE, "no propagation yet");
    const int n1 = c->corr_steps + 1;
    const size_t cnt = (size_t)c->n_samples * n1;
    int rc = enter(c);
    if (rc) return rc;
    double2 *d = nullptr;
    if (where_out == TBPM_DEVICE) {
        d = (double2 *)out;
    } else {
        rc = dalloc(c, &d, cnt);
        if (rc) return rc;
    }
    CUDA_OR_FAIL(c, launch_corr_mean(c->d_corr, c->n_samples, c->n_states, n1, d, c->st));
    if (where_out != TBPM_DEVICE) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(out, d, cnt * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));
        cudaFree(d);
    }
    c->err.clear();
    return leave(c);
}

extern "C" int tbpm_correlation_adjoint(tbpm_ctx *c, int n_steps, const double *gbar_avg,
                                        int where, double *gbar_out, int where_out)
{
    if (!c || !gbar_avg || !gbar_out) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    if (n_steps < 0) return fail(c, TBPM_E_INVALID_ARG, "n_steps < 0");
    if ((where != TBPM_HOST && where != TBPM_DEVICE) ||
        (where_out != TBPM_HOST && where_out != TBPM_DEVICE))
        return fail(c, TBPM_E_INVALID_ARG, "where must be TBPM_HOST or TBPM_DEVICE");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    const int n1 = n_steps + 1;
    const size_t cnt_in = (size_t)c->n_samples * n1;
    const size_t cnt_out = cnt_in * c->n_states;
    int rc = enter(c);
    if (rc) return rc;
    const double2 *din = nullptr;
    bool owned_in = false;
    rc = stage(c, reinterpret_cast<const double2 *>(gbar_avg), cnt_in, where,
               const_cast<double2 **>(&din), &owned_in);
    if (rc) return rc;
    double2 *dout = nullptr;
    if (where_out == TBPM_DEVICE) {
        dout = (double2 *)gbar_out;
    } else {
        rc = dalloc(c, &dout, cnt_out);
        if (rc) {
            if (owned_in) cudaFree((void *)din);
            return rc;
        }
    }
    cudaError_t e = launch_corr_mean_adjoint(din, c->n_samples, c->n_states, n1, dout, c->st);
    if (e == cudaSuccess && where_out != TBPM_DEVICE)
        e = cudaMemcpyAsync(gbar_out, dout, cnt_out * sizeof(double2), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (owned_in) cudaFree((void *)din);
    if (where_out != TBPM_DEVICE) cudaFree(dout);
    if (e != cudaSuccess)
        return fail(c, TBPM_E_CUDA, std::string("correlation adjoint: ") + cudaGetErrorString(e));
    c->err.clear();
    return leave(c);
}

extern "C" int tbpm_get_states(tbpm_ctx *c, double *phi_out, int where_out)
{
    if (!c || !phi_out) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    if (!c->have_run) return fail(c, TBPM_E_STATE, "no propagation yet");
    int rc = enter(c);
    if (rc) return rc;
    const size_t count = (size_t)c->n_states * c->n_orb;
    double2 *d = nullptr;
    if (where_out == TBPM_DEVICE) {
        d = (double2 *)phi_out;
    } else {
        rc = dalloc(c, &d, count);
        if (rc) return rc;
    }
    for (auto &g : c->groups)
        CUDA_OR_FAIL(c, launch_get_states(g.buf[g.cur], c->n_orb, c->n_states, c->H.user_to_row,
                                          g.s0, g.B, c->prec == TBPM_FP32, d, c->st));
    if (where_out != TBPM_DEVICE) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(phi_out, d, count * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->st));
        cudaFree(d);
    }
    return leave(c);
}

extern "C" int tbpm_get_norms(tbpm_ctx *c, double *out)
{
    if (!c || !out) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    if (!c->have_run) return fail(c, TBPM_E_STATE, "no propagation yet");
    const size_t cnt = (size_t)c->n_samples * c->n_states * (c->corr_steps + 1);
    CUDA_OR_FAIL(c, cudaMemcpy(out, c->d_norms, cnt * sizeof(double), cudaMemcpyDeviceToHost));
    return TBPM_OK;
}

extern "C" int tbpm_get_stats(tbpm_ctx *c, tbpm_stats *out)
{
    if (!c || !out) return fail(c, TBPM_E_INVALID_ARG, "NULL argument");
    *out = c->stats;
    return TBPM_OK;
}

// ---------------------------------------------------------------------------
// a8: adjoint propagation with checkpoints every K steps.
//
// Forward: phi_0 .. phi_{N-1} are produced step by step; phi_{jK} is kept.
// Backward, segment by segment from the last: the segment's states are
// recomputed from its checkpoint, then for each step n (descending) the
// forward polynomials T^_1 .. T^_{M-2} of phi_n are recomputed by the plain
// recurrence and the conjugate Clenshaw schedule runs with gradient
// accumulation (see adjoint_kernels.cu), ending in
// Lambda_n = gbar_n psi0 + P^dagger Lambda_{n+1}.
extern "C" int tbpm_propagate_adjoint(tbpm_ctx *c, double z, int n_steps, const double *gbar,
                                      int where, int K, double *grad_hop, double *grad_onsite,
                                      int where_out)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    if (c->H.cplx)
        return fail(c, TBPM_E_UNSUPPORTED, "the adjoint takes real hoppings only");
    if (!c->H.val64 || (c->H.n_hop > 0 && !c->H.bond_rows))
        return fail(c, TBPM_E_STATE, "the adjoint needs the FP64 Hamiltonian");
    if (n_steps < 1 || K < 1 || !gbar || !grad_hop || !grad_onsite)
        return fail(c, TBPM_E_INVALID_ARG, "bad adjoint arguments");
    if ((where != TBPM_HOST && where != TBPM_DEVICE) ||
        (where_out != TBPM_HOST && where_out != TBPM_DEVICE))
        return fail(c, TBPM_E_INVALID_ARG, "where must be TBPM_HOST or TBPM_DEVICE");
    if (K > n_steps) K = n_steps;
    std::vector<double> J(kMaxTerms);
    int M = 0;
    if (bessel_miller(z, 1e-15, kMaxTerms, J.data(), &M) != TBPM_OK || M < 2)
        return fail(c, TBPM_E_INVALID_ARG, "z out of range for the coefficient table");
    std::vector<double> a(M);
    a[0] = J[0];
    for (int m = 1; m < M; ++m) a[m] = 2.0 * J[m];

    int rc = enter(c);
    if (rc) return rc;
    rc = ensure_groups(c, TBPM_FP64);
    if (rc) return rc;
    c->have_run = false;      // the group buffers are reused as scratch below

    const size_t n_g = (size_t)c->n_samples * c->n_states * (n_steps + 1);
    double2 *d_gbar = nullptr;
    bool gbar_owned = false;
    rc = stage(c, reinterpret_cast<const double2 *>(gbar), n_g, where, &d_gbar, &gbar_owned);
    if (rc) return rc;

    int maxB = 1;
    for (auto &g : c->groups) maxB = std::max(maxB, g.B);
    const size_t vec = (size_t)c->H.n_rows * maxB * sizeof(double2);
    const int nseg = (n_steps + K - 1) / K;
    std::vector<void *> ckpt(nseg, nullptr), traj(K, nullptr), stash(M - 1, nullptr);
    double *G = nullptr, *Gd = nullptr, *d_gh = nullptr, *d_go = nullptr;
    auto release = [&]() {
        for (void *p : ckpt) cudaFree(p);
        for (void *p : traj) cudaFree(p);
        for (void *p : stash) cudaFree(p);
        cudaFree(G);
        cudaFree(Gd);
        if (where_out == TBPM_HOST) { cudaFree(d_gh); cudaFree(d_go); }
        if (gbar_owned) cudaFree(d_gbar);
    };
    for (auto &p : ckpt) if (!rc) rc = dalloc(c, (char **)&p, vec);
    for (size_t k = 1; k < traj.size() && !rc; ++k) rc = dalloc(c, (char **)&traj[k], vec);
    for (auto &p : stash) if (!rc) rc = dalloc(c, (char **)&p, vec);
    if (!rc) rc = dalloc(c, &G, (size_t)std::max<int64_t>(c->H.nnz_pad, 1));
    if (!rc) rc = dalloc(c, &Gd, (size_t)c->H.n_rows);
    if (!rc && where_out == TBPM_HOST) {
        rc = dalloc(c, &d_gh, (size_t)std::max<int64_t>(c->H.n_hop, 1));
        if (!rc) rc = dalloc(c, &d_go, (size_t)c->n_orb);
    } else if (!rc) {
        d_gh = grad_hop;
        d_go = grad_onsite;
    }
    if (rc) { release(); return rc; }
    cudaMemsetAsync(G, 0, std::max<int64_t>(c->H.nnz_pad, 1) * sizeof(double), c->st);
    cudaMemsetAsync(Gd, 0, c->H.n_rows * sizeof(double), c->st);

    SellView Hv;
    Hv.slice_ptr = c->H.slice_ptr;
    Hv.col = c->H.col;
    Hv.val = c->H.val64;
    Hv.diag = c->H.diag64;
    const int threads = c->threads[TBPM_FP64];
    int64_t launches = 0;
    int fin = 0;
    schedule(a, 0, &fin);

    for (auto &g : c->groups) {
        const int B = g.B;
        TermArgs base;
        memset(&base, 0, sizeof(base));
        base.H = Hv;
        base.chunk_sample = c->H.chunk_sample;
        base.n_rows = c->H.n_rows;
        auto term = [&](const void *x, const void *psi, const void *zz, void *out, double cc,
                        double gamma) -> int {
            TermArgs t = base;
            t.x = x;
            t.psi = psi;
            t.z = zz;
            t.out = out;
            t.c_hi = cc;
            t.gamma = gamma;
            ++launches;
            CUDA_OR_FAIL(c, launch_term(t, 0, B, threads, c->st));
            return TBPM_OK;
        };
        // one forward Clenshaw step src -> dst (tmp: scratch)
        auto step_into = [&](void *src, void *dst, void *tmp) -> int {
            void *bufs[3];
            bufs[0] = src;
            bufs[fin] = dst;
            bufs[3 - fin] = tmp;
            int nx = 0;
            for (const Launch &L : schedule(a, 0, &nx)) {
                int r2 = term(L.x < 0 ? src : bufs[L.x], src, L.z < 0 ? nullptr : bufs[L.z],
                              bufs[L.out], L.c, L.gamma);
                if (r2) return r2;
            }
            return TBPM_OK;
        };
        CUDA_OR_FAIL(c, launch_set_states(c->d_psi_user, c->n_orb, c->n_states, c->H.user_to_row,
                                          g.s0, B, 0, g.psi0, c->st));
        const size_t gvec = (size_t)c->H.n_rows * B * sizeof(double2);
        CUDA_OR_FAIL(c, cudaMemcpyAsync(ckpt[0], g.psi0, gvec, cudaMemcpyDeviceToDevice, c->st));
        // forward pass: checkpoints phi_{jK}
        void *src = ckpt[0];
        for (int n = 0; n + 1 < n_steps; ++n) {
            void *dst = g.buf[n % 2];
            if ((rc = step_into(src, dst, g.buf[2]))) { release(); return rc; }
            src = dst;
            if ((n + 1) % K == 0)
                CUDA_OR_FAIL(c, cudaMemcpyAsync(ckpt[(n + 1) / K], dst, gvec,
                                                cudaMemcpyDeviceToDevice, c->st));
        }
        // backward pass
        int lc = 0;
        CUDA_OR_FAIL(c, launch_source_init(c->H.n_rows, B, c->H.chunk_sample, d_gbar, c->n_states,
                                           g.s0, n_steps, n_steps, g.psi0, g.buf[0], c->st));
        for (int seg = nseg - 1; seg >= 0; --seg) {
            const int n0 = seg * K, n1 = std::min(n_steps, n0 + K);
            std::vector<void *> tp(n1 - n0);
            tp[0] = ckpt[seg];
            for (int k = 1; k < n1 - n0; ++k) {
                tp[k] = traj[k];
                if ((rc = step_into(tp[k - 1], tp[k], stash[0]))) { release(); return rc; }
            }
            for (int n = n1 - 1; n >= n0; --n) {
                void *phi = tp[n - n0];
                if (M - 2 >= 1 && (rc = term(phi, phi, nullptr, stash[1], 0.0, 1.0))) {
                    release(); return rc;
                }
                for (int m = 2; m <= M - 2; ++m)
                    if ((rc = term(stash[m - 1], stash[m - 1], m == 2 ? phi : stash[m - 2],
                                   stash[m], 0.0, 2.0))) {
                        release(); return rc;
                    }
                int nx = 0;
                std::vector<Launch> sch = schedule(a, lc, &nx);
                for (size_t k = 0; k < sch.size(); ++k) {
                    const Launch &L = sch[k];
                    const int m = M - 2 - (int)k;
                    AdjArgs aa;
                    memset(&aa, 0, sizeof(aa));
                    aa.H = Hv;
                    aa.x = L.x < 0 ? g.buf[lc] : g.buf[L.x];
                    aa.psi = g.buf[lc];
                    aa.z = L.z < 0 ? nullptr : g.buf[L.z];
                    aa.out = g.buf[L.out];
                    aa.T_own = m == 0 ? phi : stash[m];
                    aa.c = L.c;
                    aa.gamma = -L.gamma;
                    aa.gfac = L.gamma;
                    aa.G = G;
                    aa.Gdiag = Gd;
                    aa.gbar = m == 0 ? d_gbar : nullptr;
                    aa.psi0 = g.psi0;
                    aa.n_states = c->n_states;
                    aa.state0 = g.s0;
                    aa.n_steps = n_steps;
                    aa.step = n;
                    aa.chunk_sample = c->H.chunk_sample;
                    aa.n_rows = c->H.n_rows;
                    ++launches;
                    cudaError_t e = launch_adj_term(aa, B, threads, c->st);
                    if (e != cudaSuccess) {
                        release();
                        return fail(c, TBPM_E_CUDA, std::string("adjoint kernel: ") + cudaGetErrorString(e));
                    }
                }
                lc = nx;
            }
        }
    }
    cudaError_t e = launch_param_grads(c->H.n_hop, c->H.bond_rows, c->H.slice_ptr, c->H.col, G, Gd,
                                       c->n_orb, c->H.user_to_row, 1.0 / c->s, d_gh, d_go, c->st);
    if (e == cudaSuccess && where_out == TBPM_HOST) {
        if (c->H.n_hop > 0)
            e = cudaMemcpyAsync(grad_hop, d_gh, c->H.n_hop * sizeof(double), cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(grad_onsite, d_go, c->n_orb * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    release();
    if (e != cudaSuccess)
        return fail(c, TBPM_E_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    c->stats.kernel_launches = launches;
    c->stats.n_terms = M;
    c->stats.n_steps = n_steps;
    c->err.clear();
    return leave(c);
}

// ---------------------------------------------------------------------------
// Autotuner: times a few steps of the current Hamiltonian and states for each
// candidate (state-group width, threads per block, launch variant) and keeps
// the fastest.  The states are restored: the next propagate starts from psi0.
extern "C" int tbpm_autotune(tbpm_ctx *c, int precision, double z, int probe_steps,
                             int *best_group, int *best_threads, int *best_variant,
                             double *best_ms_per_step)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    if (precision != TBPM_FP64 && precision != TBPM_FP32)
        return fail(c, TBPM_E_INVALID_ARG, "bad precision");
    if (probe_steps < 1 || probe_steps > 64)
        return fail(c, TBPM_E_INVALID_ARG, "probe_steps must be 1..64");
    const int cap = precision == TBPM_FP64 ? 8 : 16;
    std::vector<int> widths;
    for (int B = cap; B >= 1; B /= 2)
        if (B <= c->n_states && (B >= 2 || c->n_states == 1)) widths.push_back(B);
    if (widths.empty()) widths.push_back(1);
    const int thread_opts[] = {64, 128, 256};
    const int variant_opts[] = {0, kVariantZigZag, kVariantZigZag | kVariantStreamHints,
                                kVariantZigZag | kVariantWide,
                                kVariantZigZag | kVariantSplit2, kVariantZigZag | kVariantSplit4,
                                kVariantZigZag | kVariantWide | kVariantSplit2,
                                kVariantZigZag | kVariantWide | kVariantSplit4,
                                kVariantTma, kVariantTma | kVariantZigZag, kVariantFused,
                                kVariantFused | (1 << kVariantFusedTileShift),
                                kVariantFused | (2 << kVariantFusedTileShift),
                                kVariantHalo, kVariantZigZag | kVariantHalo,
                                kVariantHalo | kVariantPipe,
                                kVariantZigZag | kVariantHalo | kVariantPipe,
                                kVariantHalo | kVariantStaged,
                                kVariantZigZag | kVariantHalo | kVariantStaged,
                                kVariantZigZag | kVariantPrefetch,
                                kVariantZigZag | kVariantWide | kVariantPrefetch,
                                kVariantZigZag | kVariantCluster};
    double best = 1e300;
    int bg = c->max_group[precision], bt = c->threads[precision], bv = c->variant[precision];
    for (int B : widths)
        for (int T : thread_opts)
            for (int V : variant_opts) {
                // the staged-gather kernel sets its own block size; it needs real
                // values and a matrix whose halo lists fit
                if ((V & kVariantHalo) && (T != thread_opts[0] || c->H.cplx ||
                                           !halo_launchable(precision == TBPM_FP32, B, false, 0)))
                    continue;
                // the fused step needs a banded row order (its dependency window
                // spans the bandwidth) and, like the TMA kernel, loses on large
                // matrices: neither is tried where it cannot win
                if ((V & kVariantFused) &&
                    (c->H.bandwidth > (1 << 16) || c->H.n_rows > (1 << 22)))
                    continue;
                if ((V & kVariantTma) && c->H.n_rows > (1 << 24)) continue;
                // the register-pipelined kernel takes real values
                if ((V & kVariantPrefetch) && c->H.cplx) continue;
                // the cluster stepping takes one FP64 state of a small real sample
                if ((V & kVariantCluster) &&
                    (T != thread_opts[0] || precision != TBPM_FP64 || B != 1 || c->H.cplx ||
                     c->n_samples != 1 ||
                     !cluster_blocks_for(c->H.n_rows, c->H.max_width, c->H.uniform)))
                    continue;
                if ((V & kVariantHalo) && !c->H.halo_ptr) {
                    std::string msg;
                    const int hr = build_halo(c->H, c->st, msg);
                    if (hr == TBPM_E_UNSUPPORTED) continue;
                    if (hr) return fail(c, hr, msg);
                }
                int rc = tbpm_set_launch_config(c, precision, B, T, V);
                if (rc) return rc;
                rc = tbpm_propagate(c, z, probe_steps, precision, nullptr, TBPM_HOST,
                                    TBPM_PROP_PROFILE);
                if (rc) return rc;
                const double ms = c->stats.ms_total / probe_steps;
                if (ms < best) { best = ms; bg = B; bt = T; bv = V; }
            }
    int rc = tbpm_set_launch_config(c, precision, bg, bt, bv);
    if (rc) return rc;
    if (best_group) *best_group = bg;
    if (best_threads) *best_threads = bt;
    if (best_variant) *best_variant = bv;
    if (best_ms_per_step) *best_ms_per_step = best;
    c->have_run = false;
    return TBPM_OK;
}

// Bond vectors d_b = r_j - r_i (nm) of the bond list, onto the stored entries.
extern "C" int tbpm_set_bond_vectors(tbpm_ctx *c, const double *dx, const double *dy, int where)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h) return fail(c, TBPM_E_STATE, "build the Hamiltonian first");
    if (c->H.n_hop > 0 && !c->H.bond_rows)
        return fail(c, TBPM_E_STATE, "the Hamiltonian was built without the bond map");
    if (c->H.n_hop > 0 && (!dx || !dy)) return fail(c, TBPM_E_INVALID_ARG, "bond vectors missing");
    if (where != TBPM_HOST && where != TBPM_DEVICE)
        return fail(c, TBPM_E_INVALID_ARG, "where must be TBPM_HOST or TBPM_DEVICE");
    int rc = enter(c);
    if (rc) return rc;
    const size_t nnz = (size_t)std::max<int64_t>(c->H.nnz_pad, 1);
    if (!c->d_bond_dx) {
        rc = dalloc(c, &c->d_bond_dx, nnz);
        if (!rc) rc = dalloc(c, &c->d_bond_dy, nnz);
        if (!rc) rc = dalloc(c, &c->d_bond_dx32, nnz);
        if (!rc) rc = dalloc(c, &c->d_bond_dy32, nnz);
        if (rc) {
            cudaFree(c->d_bond_dx);
            cudaFree(c->d_bond_dy);
            cudaFree(c->d_bond_dx32);
            c->d_bond_dx = c->d_bond_dy = nullptr;
            c->d_bond_dx32 = nullptr;
            return rc;
        }
    }
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_bond_dx, 0, nnz * sizeof(double), c->st));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_bond_dy, 0, nnz * sizeof(double), c->st));
    const double *d_x = nullptr, *d_y = nullptr;
    bool ox = false, oy = false;
    int *claim = nullptr;
    rc = stage(c, dx, (size_t)c->H.n_hop, where, const_cast<double **>(&d_x), &ox);
    if (!rc) rc = stage(c, dy, (size_t)c->H.n_hop, where, const_cast<double **>(&d_y), &oy);
    if (!rc) rc = dalloc(c, &claim, nnz);
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemsetAsync(claim, 0, nnz * sizeof(int), c->st);
    if (!rc && e == cudaSuccess) e = cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->st);
    if (!rc && e == cudaSuccess)
        e = launch_bond_vectors(c->H.n_hop, c->H.bond_rows, c->H.slice_ptr, c->H.col, d_x, d_y,
                                claim, c->d_bond_dx, c->d_bond_dy, c->d_flags, c->st);
    if (!rc && e == cudaSuccess) e = launch_vec_to_f32((int64_t)nnz, c->d_bond_dx, c->d_bond_dx32, c->st);
    if (!rc && e == cudaSuccess) e = launch_vec_to_f32((int64_t)nnz, c->d_bond_dy, c->d_bond_dy32, c->st);
    int h_err = 0;
    if (!rc && e == cudaSuccess)
        e = cudaMemcpyAsync(&h_err, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (ox) cudaFree((void *)d_x);
    if (oy) cudaFree((void *)d_y);
    cudaFree(claim);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, TBPM_E_CUDA, std::string("bond vectors: ") + cudaGetErrorString(e));
    if (h_err) {
        cudaFree(c->d_bond_dx);
        cudaFree(c->d_bond_dy);
        cudaFree(c->d_bond_dx32);
        cudaFree(c->d_bond_dy32);
        c->d_bond_dx = c->d_bond_dy = nullptr;
        c->d_bond_dx32 = c->d_bond_dy32 = nullptr;
        return fail(c, TBPM_E_INVALID_ARG, (h_err & 2) ? "non-finite bond vector"
                                                       : "bond list does not match the Hamiltonian");
    }
    c->err.clear();
    return leave(c);
}

// AC-conductivity correlation (Sec. 2.7): for each initial state psi (n_states
// per sample, at most 16), psi_2 = f(H) psi and psi_1b = [1 - f(H)] J_b psi
// (FP64, Fermi operator by Chebyshev-Clenshaw, Sec. 2.2), then psi, psi_2,
// psi_1x, psi_1y propagate as four lanes of one state group and the observer
// records <psi_2(t)|J_a|psi_1b(t)> after every step.  The caller's states are
// restored afterwards.
extern "C" int tbpm_ac_correlation(tbpm_ctx *c, double z, int n_steps, double beta, double mu,
                                   int precision, double *corr_out, int where_out, int flags)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    if (!c->d_bond_dx) return fail(c, TBPM_E_STATE, "set the bond vectors first");
    if (precision != TBPM_FP64 && precision != TBPM_FP32)
        return fail(c, TBPM_E_INVALID_ARG, "bad precision");
    if (n_steps < 0 || !corr_out || (where_out != TBPM_HOST && where_out != TBPM_DEVICE))
        return fail(c, TBPM_E_INVALID_ARG, "bad output arguments");
    if (4 * c->n_states > kMaxStates)
        return fail(c, TBPM_E_INVALID_ARG, "at most 16 initial states for the AC correlation");
    if (flags & TBPM_PROP_RESUME)
        return fail(c, TBPM_E_INVALID_ARG, "the AC correlation always starts at t = 0");
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(mu))
        return fail(c, TBPM_E_INVALID_ARG, "beta must be > 0 and mu finite");
    std::vector<double> cf;
    int rc = fermi_coefficients(beta * c->s, mu / c->s, 1e-15, 1 << 22, cf);
    if (rc) return fail(c, rc, "Fermi series too long (beta * s too large)");
    rc = enter(c);
    if (rc) return rc;

    const int S = c->n_states;
    const int64_t n_rows = c->H.n_rows, n_orb = c->n_orb;
    const size_t v4n = (size_t)n_rows * 4;
    double2 *v4 = nullptr, *f4 = nullptr, *bb[2] = {nullptr, nullptr}, *D = nullptr;
    auto release = [&]() {
        cudaFree(v4);
        cudaFree(f4);
        cudaFree(bb[0]);
        cudaFree(bb[1]);
        cudaFree(D);
    };
    rc = dalloc(c, &v4, v4n);
    if (!rc) rc = dalloc(c, &f4, v4n);
    if (!rc) rc = dalloc(c, &bb[0], v4n);
    if (!rc) rc = dalloc(c, &bb[1], v4n);
    if (!rc) rc = dalloc(c, &D, (size_t)4 * S * n_orb);
    if (rc) { release(); return rc; }

    // preparation values: FP64 when kept, else FP32 (arithmetic in FP64)
    const int fp32v = c->H.val64 ? 0 : 1;
    SellView Hp;
    Hp.slice_ptr = c->H.slice_ptr;
    Hp.col = c->H.col;
    Hp.val = fp32v ? (const void *)c->H.val32 : (const void *)c->H.val64;
    Hp.diag = fp32v ? (const void *)c->H.diag32 : (const void *)c->H.diag64;
    const int K = (int)cf.size();
    auto prep_fail = [&](cudaError_t e) {
        release();
        return fail(c, TBPM_E_CUDA, std::string("AC preparation: ") + cudaGetErrorString(e));
    };
    cudaError_t e = cudaMemsetAsync(v4, 0, v4n * sizeof(double2), c->st);
    if (e != cudaSuccess) return prep_fail(e);
    for (int p = 0; p < S; ++p) {
        e = launch_ac_load(c->d_psi_user, p, n_orb, c->H.user_to_row, v4, c->st);
        if (e == cudaSuccess)
            e = launch_current4(Hp, fp32v, c->H.cplx, n_rows, c->d_bond_dx, c->d_bond_dy, c->s, v4,
                                c->st);
        if (e != cudaSuccess) return prep_fail(e);
        // Clenshaw: b_k = c_k v + 2 H~ b_{k+1} - b_{k+2}, k = K-1 .. 1;
        // f v = c_0 v / 2 + H~ b_1 - b_2 (b_K = b_{K+1} = 0)
        int i1 = -1, i2 = -1;              // buffers of b_{k+1}, b_{k+2}
        for (int k = K - 1; k >= 1 && e == cudaSuccess; --k) {
            const int o = i2 >= 0 ? i2 : (i1 == 0 ? 1 : 0);
            e = launch_cheb_real4(Hp, fp32v, c->H.cplx, n_rows, cf[k], 2.0, -1.0, v4,
                                  i1 >= 0 ? bb[i1] : nullptr, i2 >= 0 ? bb[i2] : nullptr, bb[o],
                                  c->st);
            i2 = i1;
            i1 = o;
        }
        if (e == cudaSuccess)
            e = launch_cheb_real4(Hp, fp32v, c->H.cplx, n_rows, 0.5 * cf[0], 1.0, -1.0, v4,
                                  i1 >= 0 ? bb[i1] : nullptr, i2 >= 0 ? bb[i2] : nullptr, f4, c->st);
        if (e == cudaSuccess) e = launch_ac_store(v4, f4, p, n_orb, c->H.user_to_row, D, c->st);
        if (e != cudaSuccess) return prep_fail(e);
    }
    const size_t cnt = (size_t)c->n_samples * S * 4 * (n_steps + 1);
    rc = dalloc(c, &c->d_ac_corr, cnt);
    if (!rc) rc = dalloc(c, &c->d_ac_partial, (size_t)(n_rows / kAcRows) * 4 * 8);
    if (rc) {
        cudaFree(c->d_ac_corr);
        c->d_ac_corr = nullptr;
        release();
        return rc;
    }
    e = cudaMemsetAsync(c->d_ac_corr, 0, cnt * sizeof(double2), c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        cudaFree(c->d_ac_corr);
        c->d_ac_corr = nullptr;
        return prep_fail(e);
    }

    // the four states of each p become lanes 4p .. 4p+3 (groups of width >= 4)
    double2 *user_psi = c->d_psi_user;
    const int user_group = c->max_group[precision];
    free_groups(c);
    free_outputs(c);
    c->d_psi_user = D;
    c->n_states = 4 * S;
    if (c->max_group[precision] < 4) c->max_group[precision] = 4;
    c->ac_on = true;
    rc = tbpm_propagate(c, z, n_steps, precision, nullptr, TBPM_HOST,
                        flags & (TBPM_PROP_PROFILE | TBPM_PROP_GRAPH | TBPM_PROP_PERSISTENT));
    c->ac_on = false;
    std::string err = c->err;
    if (!rc) {
        e = cudaMemcpyAsync(corr_out, c->d_ac_corr, cnt * sizeof(double2),
                            where_out == TBPM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                            c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) {
            rc = TBPM_E_CUDA;
            err = std::string("AC correlation copy: ") + cudaGetErrorString(e);
        }
    }
    // restore the caller's states
    free_groups(c);
    free_outputs(c);
    c->d_psi_user = user_psi;
    c->n_states = S;
    c->max_group[precision] = user_group;
    cudaFree(c->d_ac_corr);
    cudaFree(c->d_ac_partial);
    c->d_ac_corr = nullptr;
    c->d_ac_partial = nullptr;
    release();                   // the derived states D included
    if (rc) return fail(c, rc, err);
    c->err.clear();
    return leave(c);
}

// Quasi-eigenstates (Sec. 2.6): forward and backward runs with the
// accumulation hook, then the caller's layout and the normalisation.
extern "C" int tbpm_quasi_eigenstates(tbpm_ctx *c, double z, int n_steps, int n_energies,
                                      const double *energies, int precision, double *out,
                                      double *norms_out, int where_out, int flags)
{
    if (!c) return fail(nullptr, TBPM_E_INVALID_ARG, "ctx is NULL");
    if (!c->have_h || c->n_states < 1)
        return fail(c, TBPM_E_STATE, "build the Hamiltonian and set states first");
    if (n_steps < 1 || n_energies < 1 || n_energies > 16 || !energies || !out ||
        (where_out != TBPM_HOST && where_out != TBPM_DEVICE))
        return fail(c, TBPM_E_INVALID_ARG, "bad quasi-eigenstate arguments");
    if (flags & (TBPM_PROP_RESUME | TBPM_PROP_BACKWARD))
        return fail(c, TBPM_E_INVALID_ARG, "the quasi-eigenstates run both directions from t = 0");
    for (int k = 0; k < n_energies; ++k)
        if (!std::isfinite(energies[k])) return fail(c, TBPM_E_INVALID_ARG, "non-finite energy");
    if (!(z > 0.0)) return fail(c, TBPM_E_INVALID_ARG, "z must be > 0");
    const int K = n_energies, S = c->n_states;
    const int64_t n_rows = c->H.n_rows, n_orb = c->n_orb;
    const double tau = z / c->s;
    // coefficient tables, forward then backward (the n = 0 term once)
    std::vector<double2> tab(2 * (size_t)(n_steps + 1) * K);
    for (int dir = 0; dir < 2; ++dir)
        for (int n = 0; n <= n_steps; ++n) {
            const double w = 0.5 * (1.0 + cos(M_PI * (double)n / (double)n_steps));
            const double t = (dir ? -1.0 : 1.0) * n * tau;
            for (int k = 0; k < K; ++k) {
                const double f = (dir && n == 0) ? 0.0 : tau / (2.0 * M_PI) * w;
                tab[((size_t)dir * (n_steps + 1) + n) * K + k] =
                    make_double2(f * cos(energies[k] * t), f * sin(energies[k] * t));
            }
        }
    std::vector<float2> tab_f(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) tab_f[i] = make_float2((float)tab[i].x, (float)tab[i].y);
    int rc = enter(c);
    if (rc) return rc;
    double2 *d_tab = nullptr, *d_out = nullptr;
    float2 *d_tab_f = nullptr;
    double *d_norms = nullptr;
    int64_t *d_off = nullptr;
    auto release = [&]() {
        cudaFree(c->d_qe_acc);
        c->d_qe_acc = nullptr;
        c->d_qe_coef = nullptr;
        c->d_qe_coef_f = nullptr;
        c->qe_on = false;
        cudaFree(d_tab);
        cudaFree(d_tab_f);
        cudaFree(d_norms);
        cudaFree(d_off);
        if (where_out == TBPM_HOST) cudaFree(d_out);
    };
    rc = dalloc(c, &c->d_qe_acc, (size_t)K * n_rows * S);
    if (!rc) rc = dalloc(c, &d_tab, tab.size());
    if (!rc) rc = dalloc(c, &d_tab_f, tab_f.size());
    if (!rc) rc = dalloc(c, &d_norms, (size_t)K * S * c->n_samples);
    if (!rc) rc = dalloc(c, &d_off, (size_t)c->n_samples + 1);
    if (!rc && where_out == TBPM_HOST) rc = dalloc(c, &d_out, (size_t)K * S * n_orb);
    if (rc) { release(); return rc; }
    if (where_out == TBPM_DEVICE) d_out = reinterpret_cast<double2 *>(out);
    cudaError_t e = cudaMemsetAsync(c->d_qe_acc, 0, (size_t)K * n_rows * S * sizeof(double2), c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice,
                            c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tab_f, tab_f.data(), tab_f.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, c->sample_off.data(), (c->n_samples + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);      // host tables go out of scope
    if (e != cudaSuccess) {
        release();
        return fail(c, TBPM_E_CUDA, std::string("quasi-eigenstates: ") + cudaGetErrorString(e));
    }
    c->qe_on = true;
    c->qe_K = K;
    const int pf = flags & (TBPM_PROP_PROFILE | TBPM_PROP_GRAPH | TBPM_PROP_PERSISTENT);
    c->d_qe_coef = d_tab;
    c->d_qe_coef_f = d_tab_f;
    rc = tbpm_propagate(c, z, n_steps, precision, nullptr, TBPM_HOST, pf);
    if (!rc) {
        c->d_qe_coef = d_tab + (size_t)(n_steps + 1) * K;
        c->d_qe_coef_f = d_tab_f + (size_t)(n_steps + 1) * K;
        rc = tbpm_propagate(c, z, n_steps, precision, nullptr, TBPM_HOST, pf | TBPM_PROP_BACKWARD);
    }
    c->qe_on = false;
    if (rc) {
        std::string m = c->err;
        release();
        return fail(c, rc, m);
    }
    e = launch_qe_finish(c->d_qe_acc, precision == TBPM_FP32, K, S, n_rows, n_orb, c->n_samples,
                         c->H.user_to_row,
                         c->H.orb_sample, d_off, d_out, d_norms, c->st);
    if (e == cudaSuccess && where_out == TBPM_HOST)
        e = cudaMemcpyAsync(out, d_out, (size_t)K * S * n_orb * sizeof(double2),
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && norms_out)
        e = cudaMemcpyAsync(norms_out, d_norms, (size_t)K * S * c->n_samples * sizeof(double),
                            cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    release();
    if (e != cudaSuccess)
        return fail(c, TBPM_E_CUDA, std::string("quasi-eigenstates: ") + cudaGetErrorString(e));
    c->err.clear();
    return leave(c);
}
