// noalloc.cu -- dual bound of a reparametrized model without any device
// allocation: mplpp_bound_noalloc (include/mplpp.h).
//
// Some callers cannot call cudaMalloc: code that owns a fixed device arena and
// forbids allocations after start-up, real-time loops that cannot afford an
// allocation's latency or its implicit synchronization, and plugins hosted by
// another runtime whose allocator must see every byte.  They pass their own
// device buffers for every input and output; the working memory this
// computation needs (table and message offsets, per-node and per-edge minima)
// lives in one file-scope device array of fixed size instead.
//
// The array is reached from host code only through its device address,
// obtained with cudaGetSymbolAddress once per device context (the first call
// on a device, and again after that device's context was destroyed and
// recreated, e.g. by cudaDeviceReset: the cache is keyed by the context's
// unique id); the name itself, in host code, is not a device address.  Every
// call shares the array: calls that overlap on the GPU (other streams, other
// host threads) race on it.  Every word a call reads is written earlier by the
// same call, so nothing needs clearing between calls.
#include <climits>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>

#include "mplpp.h"

namespace {

constexpr long long kMaxNodes = MPLPP_NOALLOC_MAX_NODES;
constexpr long long kMaxEdges = MPLPP_NOALLOC_MAX_EDGES;
constexpr long long align256(long long x) { return (x + 255) & ~255LL; }
// layout of the scratch array (bytes)
constexpr long long kOffStatus = 0;                                       // int: input check result
constexpr long long kOffNode = 256;                                       // int64 [n + 1]: node vector offsets
constexpr long long kOffPair = kOffNode + align256(8 * (kMaxNodes + 1));  // int64 [E + 1]: table offsets
constexpr long long kOffMsg = kOffPair + align256(8 * (kMaxEdges + 1));   // int64 [E + 1]: message offsets
constexpr long long kOffNmin = kOffMsg + align256(8 * (kMaxEdges + 1));   // float [n]: node minima
constexpr long long kOffEmin = kOffNmin + align256(4 * kMaxNodes);        // float [E]: edge minima
constexpr long long kScratchBytes = kOffEmin + align256(4 * kMaxEdges);
static_assert(kScratchBytes == MPLPP_NOALLOC_SCRATCH_BYTES, "scratch size in mplpp.h is out of date");

static __device__ __align__(256) unsigned char g_bound_scratch[kScratchBytes];

constexpr int kScanThreads = 1024;
constexpr int kThreads = 256;

struct Scratch {
    int *status;
    long long *node_off, *pair_off, *msg_off;
    float *nmin, *emin;
};

__host__ __device__ inline Scratch carve(unsigned char *base)
{
    Scratch s;
    s.status = reinterpret_cast<int *>(base + kOffStatus);
    s.node_off = reinterpret_cast<long long *>(base + kOffNode);
    s.pair_off = reinterpret_cast<long long *>(base + kOffPair);
    s.msg_off = reinterpret_cast<long long *>(base + kOffMsg);
    s.nmin = reinterpret_cast<float *>(base + kOffNmin);
    s.emin = reinterpret_cast<float *>(base + kOffEmin);
    return s;
}

// Exclusive prefix sums of a per-item size, one CTA: every thread sums a
// contiguous chunk, the chunk totals are scanned in shared memory, then every
// chunk is written out.
template <typename F>
__device__ void block_scan(int count, long long *out, F size_of, long long *part)
{
    const int T = blockDim.x, tid = threadIdx.x;
    const int chunk = (count + T - 1) / T;
    const int b = tid * chunk, e = min(count, b + chunk);
    long long sum = 0;
    for (int i = b; i < e; ++i) sum += size_of(i);
    part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        long long acc = 0;
        for (int i = 0; i < T; ++i) {
            const long long v = part[i];
            part[i] = acc;
            acc += v;
        }
        out[count] = acc;
    }
    __syncthreads();
    long long acc = part[tid];
    for (int i = b; i < e; ++i) {
        out[i] = acc;
        acc += size_of(i);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kScanThreads) offsets_kernel(unsigned char *scratch, int n, int E, const int *labels,
                                                               const int *eu, const int *ev)
{
    __shared__ long long part[kScanThreads];
    const Scratch s = carve(scratch);
    if (threadIdx.x == 0) *s.status = 0;
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += blockDim.x)
        if (labels[u] < 1 || labels[u] > 65535) atomicOr(s.status, 1);
    for (int e = threadIdx.x; e < E; e += blockDim.x)
        if (eu[e] < 0 || ev[e] >= n || eu[e] >= ev[e]) atomicOr(s.status, 2);
    __syncthreads();
    if (*reinterpret_cast<volatile int *>(s.status) != 0) return;
    block_scan(n, s.node_off, [&](int u) { return static_cast<long long>(labels[u]); }, part);
    block_scan(E, s.pair_off, [&](int e) { return static_cast<long long>(labels[eu[e]]) * labels[ev[e]]; }, part);
    block_scan(E, s.msg_off, [&](int e) { return static_cast<long long>(labels[eu[e]]) + labels[ev[e]]; }, part);
}

// min_s theta^phi_u(s) per node (one warp per node)
__global__ void node_min_kernel(const unsigned char *scratch, int n, const int *labels, const float *agg)
{
    const Scratch s = carve(const_cast<unsigned char *>(scratch));
    if (*s.status) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = warp; u < n; u += nw) {
        float m = INFINITY;
        for (int i = lane; i < labels[u]; i += 32) m = fminf(m, agg[s.node_off[u] + i]);
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s.nmin[u] = m;
    }
}

// min_{s,t} (theta_uv(s,t) - phi_{v->u}(s)) - phi_{u->v}(t) per edge (one CTA
// per edge): rows by warp, columns by lane, 32-bit indices within a table
// (L_u, L_v <= 65,535 as for the solver, so a row offset a * L_v fits).
__global__ void __launch_bounds__(kThreads) edge_min_kernel(const unsigned char *scratch, int E, const int *labels,
                                                            const int *eu, const int *ev, const float *pairwise,
                                                            const float *msg)
{
    __shared__ float red[kThreads / 32];
    const Scratch s = carve(const_cast<unsigned char *>(scratch));
    if (*s.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        const int Lu = labels[eu[e]], Lv = labels[ev[e]];
        const float *th = pairwise + s.pair_off[e];
        const float *pu = msg + s.msg_off[e];
        const float *pv = pu + Lu;
        float m = INFINITY;
        for (int a = warp; a < Lu; a += kThreads / 32) {
            const float *row = th + static_cast<unsigned>(a) * static_cast<unsigned>(Lv);
            const float pa = pu[a];
            for (int b = lane; b < Lv; b += 32) m = fminf(m, (row[b] - pa) - pv[b]);
        }
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float r = red[0];
            for (int j = 1; j < kThreads / 32; ++j) r = fminf(r, red[j]);
            s.emin[e] = r;
        }
        __syncthreads();
    }
}

// D = sum of node minima + sum of edge minima in FP64, fixed order.
__global__ void __launch_bounds__(kThreads) sum_kernel(const unsigned char *scratch, int n, int E, double *out)
{
    __shared__ double red[kThreads];
    const Scratch s = carve(const_cast<unsigned char *>(scratch));
    if (*s.status) return;
    double acc = 0.0;
    for (int u = threadIdx.x; u < n; u += kThreads) acc += static_cast<double>(s.nmin[u]);
    for (int e = threadIdx.x; e < E; e += kThreads) acc += static_cast<double>(s.emin[e]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

std::mutex g_mu;
struct ScratchAddr {
    unsigned long long ctx_id;  // unique id of the context the address belongs to
    void *addr;
};
ScratchAddr g_addr[64] = {};
thread_local std::string g_error;

mplpp_status fail(mplpp_status st, const std::string &m)
{
    g_error = m;
    return st;
}

// Unique id of the current context (cuCtxGetCurrent + cuCtxGetId through the
// runtime's driver entry points, so the library does not link libcuda);
// false where the driver does not offer them.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

}  // namespace

extern "C" const char *mplpp_noalloc_last_error(void)
{
    return g_error.c_str();
}

extern "C" mplpp_status mplpp_bound_noalloc(int32_t n_nodes, int32_t n_edges, const int32_t *labels,
                                            const int32_t *edge_u, const int32_t *edge_v, const float *pairwise,
                                            const float *agg, const float *msg, double *out, void *stream)
{
    g_error.clear();
    if (n_nodes < 1 || n_edges < 0) return fail(MPLPP_E_INVALID, "need n_nodes >= 1 and n_edges >= 0");
    if (n_nodes > kMaxNodes || n_edges > kMaxEdges)
        return fail(MPLPP_E_UNSUPPORTED, "mplpp_bound_noalloc handles at most " + std::to_string(kMaxNodes) +
                                             " nodes and " + std::to_string(kMaxEdges) + " edges; got " +
                                             std::to_string(n_nodes) + " and " + std::to_string(n_edges));
    if (!labels || !agg || !msg || !out || (n_edges > 0 && (!edge_u || !edge_v || !pairwise)))
        return fail(MPLPP_E_INVALID, "NULL array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MPLPP_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(MPLPP_E_UNSUPPORTED, "device index above 63");
    // the current device's primary context must exist before its id is read
    // (cudaSetDevice initializes it; no allocation)
    if ((e = cudaSetDevice(dev)) != cudaSuccess)
        return fail(MPLPP_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        unsigned long long ctx = 0;
        const bool have_id = current_context_id(&ctx);
        if (!have_id || !g_addr[dev].addr || g_addr[dev].ctx_id != ctx) {
            // set-up: once per device context, with that device current
            void *a = nullptr;
            e = cudaGetSymbolAddress(&a, g_bound_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = ScratchAddr{0, nullptr};
                return fail(MPLPP_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_addr[dev] = ScratchAddr{have_id ? ctx : 0, a};
        }
        base = g_addr[dev].addr;
    }
    unsigned char *scratch = static_cast<unsigned char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    offsets_kernel<<<1, kScanThreads, 0, st>>>(scratch, n_nodes, n_edges, labels, edge_u, edge_v);
    node_min_kernel<<<(n_nodes + 7) / 8, 256, 0, st>>>(scratch, n_nodes, labels, agg);
    if (n_edges > 0)
        edge_min_kernel<<<n_edges < 65535 ? n_edges : 65535, kThreads, 0, st>>>(scratch, n_edges, labels, edge_u,
                                                                              edge_v, pairwise, msg);
    sum_kernel<<<1, kThreads, 0, st>>>(scratch, n_nodes, n_edges, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(MPLPP_E_CUDA, cudaGetErrorString(e));
    int status = 0;
    e = cudaMemcpyAsync(&status, scratch + kOffStatus, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MPLPP_E_CUDA, cudaGetErrorString(e));
    if (status & 1) return fail(MPLPP_E_INVALID, "labels must be in 1..65535");
    if (status & 2) return fail(MPLPP_E_INVALID, "edges must satisfy 0 <= u < v < n_nodes");
    return MPLPP_OK;
}
