// dual.cu -- packing of the inputs, the dual lower bound (Sec. 3, eq.
// LP-lower-bound), sequential primal rounding (Sec. 4, Primal Rounding) and
// the energy (eq. energy-min) on sm_103a.
#include <cfloat>
#include <climits>
#include <cstdint>

#include "kernels.h"

namespace mplpp {

namespace {

constexpr int kThreads = 256;

// Copies the caller's row-major tables into the padded layout (row stride ld,
// pad +inf) and the unaries into un0 (FP32) and agg (double-float entries,
// version 0), pad 0.
// Flags non-finite costs.
__global__ void pack_tables_kernel(const EdgeDesc *edges, int n_edges, const float *src, float *tab, int *err)
{
    for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        const long long n = static_cast<long long>(ed.Lu) * ed.ld;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = static_cast<int>(i / ed.ld);
            const int t = static_cast<int>(i - static_cast<long long>(s) * ed.ld);
            float v = INFINITY;
            if (t < ed.Lv) {
                v = src[ed.poff + static_cast<long long>(s) * ed.Lv + t];
                if (!isfinite(v)) atomicCAS(err, 0, ERR_NONFINITE);
            }
            tab[ed.toff + i] = v;
        }
    }
}

__global__ void pack_unary_kernel(const NodeDesc *nodes, int n_nodes, const float *src, float *un0, ulonglong2 *agg,
                                  int *err)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = warp; u < n_nodes; u += nw) {
        const NodeDesc nd = nodes[u];
        const int Lp = (nd.L + 3) & ~3;
        for (int s = lane; s < Lp; s += 32) {
            float v = 0.f;
            if (s < nd.L) {
                v = src[nd.uoff + s];
                if (!isfinite(v)) atomicCAS(err, 0, ERR_NONFINITE);
            }
            un0[nd.aoff + s] = v;
            agg[nd.aoff + s] = se_make(make_float2(v, 0.f), 0u);
        }
    }
}

template <int T>
__device__ __forceinline__ double block_min(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < T / 32 ? red[l] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;  // valid in thread 0
}

// emin[e] = min_{s,t} (theta_uv(s,t) - phi_{v->u}(s)) - phi_{u->v}(t)   (FP64)
__global__ void __launch_bounds__(kThreads) bound_edges_kernel(const EdgeDesc *edges, int n_edges,
                                                               const float *tab, const ulonglong2 *msg, double *emin)
{
    __shared__ double red[32];
    for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        double m = INFINITY;
        const long long n = static_cast<long long>(ed.Lu) * ed.Lv;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = static_cast<int>(i / ed.Lv);
            const int t = static_cast<int>(i - static_cast<long long>(s) * ed.Lv);
            const double r =
                (static_cast<double>(tab[ed.toff + static_cast<long long>(s) * ed.ld + t]) - se_d(msg[ed.mu + s])) -
                se_d(msg[ed.mv + t]);
            m = fmin(m, r);
        }
        m = block_min<kThreads>(m, red);
        if (threadIdx.x == 0) emin[e] = m;
    }
}

// nmin[u] = min_s theta^phi_u(s)   (FP64)
__global__ void bound_nodes_kernel(const NodeDesc *nodes, int n_nodes, const ulonglong2 *agg, double *nmin)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = warp; u < n_nodes; u += nw) {
        const NodeDesc nd = nodes[u];
        double m = INFINITY;
        for (int s = lane; s < nd.L; s += 32) m = fmin(m, se_d(agg[nd.aoff + s]));
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) nmin[u] = m;
    }
}

// Fixed-order FP64 sum (deterministic): thread i adds elements i, i+T, ...,
// then a fixed tree.
template <int T>
__device__ double block_sum_fixed(double v, double *red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) bound_sum_kernel(const int *model_node_off, const int *model_edge_off,
                                                             const double *nmin, const double *emin, int exact,
                                                             double *out)
{
    __shared__ double red[kThreads];
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int u = model_node_off[m] + threadIdx.x; u < model_node_off[m + 1]; u += kThreads)
        acc += nmin[u];
    if (exact)
        for (int e = model_edge_off[m] + threadIdx.x; e < model_edge_off[m + 1]; e += kThreads)
            acc += emin[e];
    const double D = block_sum_fixed<kThreads>(acc, red);
    if (threadIdx.x == 0) out[m] = D;
}

// Sequential rounding of one model per CTA: node u's objective over its
// labels is its reparametrized unary plus, for every earlier neighbour v in
// increasing order, theta^phi_vu(x_v, s) = (theta_vu(x_v,s) - phi_{u->v}(x_v))
// - phi_{v->u}(s); FP64 sums in that order, argmin with the lowest index.
__global__ void __launch_bounds__(kThreads) round_kernel(const EdgeDesc *edges, const NodeDesc *nodes,
                                                         const int *in_off, const int *in_edge,
                                                         const int *model_node_off, const float *tab,
                                                         const ulonglong2 *agg, const ulonglong2 *msg, int *labels,
                                                         int *err)
{
    __shared__ double rv[32];
    __shared__ int ri[32];
    const int m = blockIdx.x;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int u = model_node_off[m]; u < model_node_off[m + 1]; ++u) {
        const NodeDesc nd = nodes[u];
        double best = INFINITY;
        int bi = INT_MAX;
        for (int s = threadIdx.x; s < nd.L; s += kThreads) {
            double acc = se_d(agg[nd.aoff + s]);
            for (int k = in_off[u]; k < in_off[u + 1]; ++k) {
                const EdgeDesc ed = edges[in_edge[k]];
                const int xv = labels[ed.gu];
                const double term =
                    (static_cast<double>(tab[ed.toff + static_cast<long long>(xv) * ed.ld + s]) -
                     se_d(msg[ed.mu + xv])) -
                    se_d(msg[ed.mv + s]);
                acc = acc + term;
            }
            if (acc < best) {
                best = acc;
                bi = s;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (l == 0) {
            rv[w] = best;
            ri[w] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = rv[0];
            int i = ri[0];
            for (int j = 1; j < kThreads / 32; ++j)
                if (rv[j] < b || (rv[j] == b && ri[j] < i)) {
                    b = rv[j];
                    i = ri[j];
                }
            if (i == INT_MAX) {  // every objective value was NaN
                i = 0;
                atomicCAS(err, 0, ERR_NONFINITE);
            }
            labels[u] = i;
        }
        __syncthreads();
    }
}

// E(x | original costs) in FP64 (eq. energy-min), fixed-order sums.
__global__ void __launch_bounds__(kThreads) energy_kernel(const EdgeDesc *edges, const NodeDesc *nodes,
                                                          const int *model_node_off, const int *model_edge_off,
                                                          const float *tab, const float *un0, const int *labels,
                                                          double *energy)
{
    __shared__ double red[kThreads];
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int u = model_node_off[m] + threadIdx.x; u < model_node_off[m + 1]; u += kThreads)
        acc += static_cast<double>(un0[nodes[u].aoff + labels[u]]);
    for (int e = model_edge_off[m] + threadIdx.x; e < model_edge_off[m + 1]; e += kThreads) {
        const EdgeDesc ed = edges[e];
        acc += static_cast<double>(tab[ed.toff + static_cast<long long>(labels[ed.gu]) * ed.ld + labels[ed.gv]]);
    }
    const double En = block_sum_fixed<kThreads>(acc, red);
    if (threadIdx.x == 0) energy[m] = En;
}

// agg := (un0, 0), msg := 0: the state phi = 0 (version 0)
__global__ void init_state_kernel(const float *un0, ulonglong2 *agg, long long n_agg, ulonglong2 *msg,
                                  long long n_msg)
{
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_agg; i += stride)
        agg[i] = se_make(make_float2(un0[i], 0.f), 0u);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_msg; i += stride)
        msg[i] = se_make(make_float2(0.f, 0.f), 0u);
}

// version := 0 in both words of every entry
__global__ void restamp_kernel(ulonglong2 *agg, long long n_agg, ulonglong2 *msg, long long n_msg)
{
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    const unsigned long long keep = 0xffffffffull;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_agg; i += stride) {
        const ulonglong2 e = agg[i];
        agg[i] = make_ulonglong2(e.x & keep, e.y & keep);
    }
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_msg; i += stride) {
        const ulonglong2 e = msg[i];
        msg[i] = make_ulonglong2(e.x & keep, e.y & keep);
    }
}

int grid_for(long long work, int per_block_items)
{
    long long g = (work + per_block_items - 1) / per_block_items;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_pack(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                        const float *unary_src, const float *pair_src, float *tab, float *un0, ulonglong2 *agg, int *err,
                        cudaStream_t st)
{
    if (n_edges > 0) {
        pack_tables_kernel<<<grid_for(n_edges, 1), kThreads, 0, st>>>(edges, n_edges, pair_src, tab, err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_nodes > 0) {
        pack_unary_kernel<<<grid_for(n_nodes, kThreads / 32), kThreads, 0, st>>>(nodes, n_nodes, unary_src, un0,
                                                                                 agg, err);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_init_state(const float *un0, ulonglong2 *agg, long long n_agg, ulonglong2 *msg, long long n_msg,
                              cudaStream_t st)
{
    init_state_kernel<<<grid_for(n_agg > n_msg ? n_agg : n_msg, kThreads), kThreads, 0, st>>>(un0, agg, n_agg, msg,
                                                                                           n_msg);
    return cudaGetLastError();
}

cudaError_t launch_restamp(ulonglong2 *agg, long long n_agg, ulonglong2 *msg, long long n_msg, cudaStream_t st)
{
    restamp_kernel<<<grid_for(n_agg > n_msg ? n_agg : n_msg, kThreads), kThreads, 0, st>>>(agg, n_agg, msg, n_msg);
    return cudaGetLastError();
}

cudaError_t launch_bound(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes, const float *tab,
                         const ulonglong2 *agg, const ulonglong2 *msg, double *emin, double *nmin, const int *model_node_off,
                         const int *model_edge_off, int n_models, int exact, double *out, cudaStream_t st)
{
    if (exact && n_edges > 0) {
        bound_edges_kernel<<<grid_for(n_edges, 1), kThreads, 0, st>>>(edges, n_edges, tab, msg, emin);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_nodes > 0) {
        bound_nodes_kernel<<<grid_for(n_nodes, kThreads / 32), kThreads, 0, st>>>(nodes, n_nodes, agg, nmin);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    bound_sum_kernel<<<n_models, kThreads, 0, st>>>(model_node_off, model_edge_off, nmin, emin, exact, out);
    return cudaGetLastError();
}

cudaError_t launch_round(const EdgeDesc *edges, const NodeDesc *nodes, const int *in_off, const int *in_edge,
                         const int *model_node_off, const int *model_edge_off, int n_models, const float *tab,
                         const ulonglong2 *agg, const ulonglong2 *msg, const float *un0, int *labels, double *energy, int *err,
                         cudaStream_t st)
{
    round_kernel<<<n_models, kThreads, 0, st>>>(edges, nodes, in_off, in_edge, model_node_off, tab, agg, msg, labels,
                                               err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_kernel<<<n_models, kThreads, 0, st>>>(edges, nodes, model_node_off, model_edge_off, tab, un0, labels,
                                                energy);
    return cudaGetLastError();
}

}  // namespace mplpp
