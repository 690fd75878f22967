// record.cu -- the Handshake update in FP64, optionally recording argmins, for
// the backward pass.
//
// The gradient of D_T is the gradient of one linear piece of a piecewise
// linear function, selected by the argmins of the forward.  A binary32
// trajectory drifts from the exact one by ~1e-6 relative over many
// iterations, enough to select different pieces at near-ties; the backward
// therefore replays the iterations in binary64 (same message-form arithmetic
// and association as handshake.cu, on a double copy of the state), so that its
// argmins are those of the exact-arithmetic trajectory up to binary64 rounding.
// One CTA per edge of a matching; one launch per matching.
#include <cfloat>
#include <climits>

#include "backward.h"
#include "kernels.h"

namespace mplpp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void amin_d(double &m, int &i, double v, int j)
{
    if (v < m || (v == m && j < i)) {
        m = v;
        i = j;
    }
}

__device__ __forceinline__ void warp_amin_d(double &m, int &i)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, m, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        amin_d(m, i, om, oi);
    }
}

template <bool REC>
__global__ void __launch_bounds__(kThreads) rec64_phase_kernel(const EdgeDesc *edges, const int *items,
                                                               const float *tab, double *agg, double *msg,
                                                               unsigned char *rec, const long long *rec_off, int lmax)
{
    extern __shared__ __align__(16) double shd[];
    double *uh = shd;           // [Lu]
    double *alpha = uh + lmax;  // [Lu]
    double *vh = alpha + lmax;  // [Lv]
    double *bv = vh + lmax;     // [Lv]
    double *beta = bv + lmax;   // [Lv]
    const int e = items[blockIdx.x];
    const EdgeDesc ed = edges[e];
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const float *th = tab + ed.toff;
    unsigned short *t1 = nullptr, *s2 = nullptr, *t3 = nullptr;
    if (REC) {
        t1 = reinterpret_cast<unsigned short *>(rec + rec_off[e]);
        s2 = t1 + Lu;
        t3 = s2 + Lv;
    }
    for (int s = tid; s < Lu; s += blockDim.x) uh[s] = agg[ed.au + s] - msg[ed.mu + s];
    for (int t = tid; t < Lv; t += blockDim.x) vh[t] = agg[ed.av + t] - msg[ed.mv + t];
    __syncthreads();
    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + vh(t)] + uh(s)),  alpha = uh - a
    for (int s = warp; s < Lu; s += nw) {
        double m = INFINITY;
        int mi = INT_MAX;
        for (int t = lane; t < Lv; t += 32) {
            const double v = static_cast<double>(th[static_cast<long long>(s) * ld + t]) + vh[t];
            if (v < m) {
                m = v;
                mi = t;
            }
        }
        warp_amin_d(m, mi);
        if (lane == 0) {
            const double a = 0.5 * (m + uh[s]);
            alpha[s] = uh[s] - a;
            if (REC) t1[s] = static_cast<unsigned short>(mi);
        }
    }
    __syncthreads();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t),  beta = vh - b
    for (int t = tid; t < Lv; t += blockDim.x) {
        double m = INFINITY;
        int mi = 0;
        for (int s = 0; s < Lu; ++s) {
            const double v = static_cast<double>(th[static_cast<long long>(s) * ld + t]) + alpha[s];
            if (v < m) {
                m = v;
                mi = s;
            }
        }
        const double b = m + vh[t];
        bv[t] = b;
        beta[t] = vh[t] - b;
        if (REC) s2[t] = static_cast<unsigned short>(mi);
    }
    __syncthreads();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s)
    for (int s = warp; s < Lu; s += nw) {
        double m = INFINITY;
        int mi = INT_MAX;
        for (int t = lane; t < Lv; t += 32) {
            const double v = static_cast<double>(th[static_cast<long long>(s) * ld + t]) + beta[t];
            if (v < m) {
                m = v;
                mi = t;
            }
        }
        warp_amin_d(m, mi);
        if (lane == 0) {
            const double c = m + uh[s];
            agg[ed.au + s] = c;
            msg[ed.mu + s] = c - uh[s];
            if (REC) t3[s] = static_cast<unsigned short>(mi);
        }
    }
    for (int t = tid; t < Lv; t += blockDim.x) {
        agg[ed.av + t] = bv[t];
        msg[ed.mv + t] = bv[t] - vh[t];
    }
}

__global__ void widen_kernel(const float *src, double *dst, long long n)
{
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[i] = static_cast<double>(src[i]);
}

}  // namespace

size_t rec64_smem_bytes(int lmax)
{
    return static_cast<size_t>(lmax) * 5 * sizeof(double);
}

cudaError_t launch_rec64_phase(const EdgeDesc *edges, const int *items, int n_items, const float *tab, double *agg,
                               double *msg, unsigned char *rec, const long long *rec_off, int lmax, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = rec64_smem_bytes(lmax);
    if (rec) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(rec64_phase_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        rec64_phase_kernel<true><<<n_items, kThreads, smem, st>>>(edges, items, tab, agg, msg, rec, rec_off, lmax);
    } else {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(rec64_phase_kernel<false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        rec64_phase_kernel<false><<<n_items, kThreads, smem, st>>>(edges, items, tab, agg, msg, nullptr, nullptr, lmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_widen(const float *src, double *dst, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 65535LL * 8);
    widen_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace mplpp
