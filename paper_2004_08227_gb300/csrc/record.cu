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
#include <algorithm>
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

// ---------------------------------------------------------------------------
// The same update with FP64 work only where it can decide a minimum.  GB300
// runs FP64 at a small fraction of its FP32 rate, so every minimization is
// first screened in FP32 and only its surviving candidates are evaluated in
// FP64, with exactly the FP64 expression of rec64_phase_kernel above; the
// minima and argmins are therefore bit for bit those of the all-FP64 kernel.
//
// Screen of min_j V(j), V(j) = theta(j) + x(j) (x the FP64 vector of the
// minimization, theta the FP32 table entries along a row or a column):
//   w(j) = fl32(x(j) - x(0)) (the difference taken in FP64),
//   c(j) = fl32(theta(j) + w(j)).
// With D = max_j |w(j)| and h = max_j |theta(j)| over the row / column,
//   |c(j) - (theta(j) + w(j))| <= 2^-24 (h + D),
//   |w(j) - (x(j) - x(0))|     <= 2^-24 D (1 + 2^-24) + 2^-53 |x(j) - x(0)|,
// so |c(j) - (V(j) - x(0))| <= 2^-22 (h + D) = e1 (a factor 2 to spare); and
// the FP64 value v(j) = fl64(theta(j) + x(j)) errs from V(j) by at most
// 2^-53 (h + D + |x(0)|)(1 + 2^-22) <= 2^-50 (h + D + |x(0)|) = e2.  If j* is
// the FP64 argmin and c(jc) the FP32 minimum, then
//   c(j*) <= V(j*) - x(0) + e1 <= v(j*) - x(0) + e1 + e2
//         <= v(jc) - x(0) + e1 + e2 <= c(jc) + 2 e1 + 2 e2,
// so every j with c(j) <= c(jc) + 2 e1 + 2 e2 (threshold rounded upwards) is a
// candidate, and the FP64 argmin (the lowest index among equal FP64 minima)
// is among the candidates.  The candidates of a pass go to a per-CTA list;
// each is evaluated in FP64 by one thread and merged into its row's / column's
// minimum with 64-bit shared-memory atomics on an order-preserving key (value
// first, then the lowest index among equal values), so the order of the list
// does not matter.  A pass whose candidates overflow the list takes the
// all-FP64 scan instead.  The table is staged in shared memory with an odd row
// stride (conflict-free row and column access).
namespace {

constexpr int kScrThreads = 256;
constexpr int kCandMax = 2048;  // candidates per pass

__device__ __forceinline__ unsigned long long order_key(double v)
{
    v = v + 0.0;  // -0 -> +0: equal values get equal keys
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

struct ScreenSmem {
    float *tab;                 // [Lu][ldp] staged table, ldp odd
    double *uh, *vh, *al, *be;  // FP64 vectors (uh, alpha: Lu; vh, beta: Lv)
    double *bv;                 // b(t) [Lv]
    float *w;                   // FP32 shifted vector of the current pass [lmax]
    float *pmin, *pmax;         // partial FP32 minima and |theta| maxima [G][n]
    float *thr;                 // per row / column threshold [lmax]
    unsigned long long *key;    // per row / column FP64 minimum key [lmax]
    int *arg;                   // per row / column argmin [lmax]
    int2 *cand;                 // [kCandMax] (row or column, index along it)
    int *count;                 // [2] candidate count, scratch
    float *red;                 // [kScrThreads / 32]
};

__device__ __forceinline__ float block_max_f(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
    __syncthreads();
    return r;
}

// One minimization family: for every line i < n (rows of the table when
// ROWS, else columns), m(i) = min_j [theta(i, j) + x(j)] over j < len with
// its lowest argmin, where x is the FP64 vector xv (x(0) = xv[0]) and w its
// FP32 shifted copy (in sm.w, max |w| = D).  Results in sm.key / sm.arg.
template <bool ROWS>
__device__ void screened_min(const ScreenSmem &sm, int ldp, int n, int len, const double *xv, float D)
{
    const int T = blockDim.x, tid = threadIdx.x;
    const int G = max(1, T / max(n, 1));  // threads per line
    const int span = (len + G - 1) / G;   // elements per thread
    auto th = [&](int i, int j) { return ROWS ? sm.tab[i * ldp + j] : sm.tab[j * ldp + i]; };
    const double x0 = xv[0];
    // scan 1: partial FP32 minima and |theta| maxima
    for (int q = tid; q < G * n; q += T) {
        const int i = q % n, g = q / n;
        const int j0 = g * span, j1 = min(len, j0 + span);
        float mn = INFINITY, mx = 0.f;
        for (int j = j0; j < j1; ++j) {
            const float t = th(i, j);
            mn = fminf(mn, t + sm.w[j]);
            mx = fmaxf(mx, fabsf(t));
        }
        sm.pmin[g * n + i] = mn;
        sm.pmax[g * n + i] = mx;
    }
    if (tid == 0) sm.count[0] = 0;
    __syncthreads();
    const float ax0 = __double2float_ru(fabs(x0));
    for (int i = tid; i < n; i += T) {
        float mn = INFINITY, h = 0.f;
        for (int g = 0; g < G; ++g) {
            mn = fminf(mn, sm.pmin[g * n + i]);
            h = fmaxf(h, sm.pmax[g * n + i]);
        }
        const float e1 = __fmul_ru(0x1p-22f, __fadd_ru(h, D));
        const float e2 = __fmul_ru(0x1p-50f, __fadd_ru(__fadd_ru(h, D), ax0));
        sm.thr[i] = __fadd_ru(__fadd_ru(mn, __fmul_ru(2.f, e1)), __fadd_ru(__fmul_ru(2.f, e2), 0x1p-126f));
        sm.key[i] = ~0ull;
        sm.arg[i] = INT_MAX;
    }
    __syncthreads();
    // scan 2: candidates
    for (int q = tid; q < G * n; q += T) {
        const int i = q % n, g = q / n;
        const int j0 = g * span, j1 = min(len, j0 + span);
        const float tr = sm.thr[i];
        for (int j = j0; j < j1; ++j)
            if (th(i, j) + sm.w[j] <= tr) {
                const int k = atomicAdd(&sm.count[0], 1);
                if (k < kCandMax) sm.cand[k] = make_int2(i, j);
            }
    }
    __syncthreads();
    const int nc = sm.count[0];
    if (nc <= kCandMax) {
        // FP64 values of the candidates, merged per line: value, then index
        for (int k = tid; k < nc; k += T) {
            const int2 c = sm.cand[k];
            const double v = static_cast<double>(th(c.x, c.y)) + xv[c.y];
            atomicMin(&sm.key[c.x], order_key(v));
        }
        __syncthreads();
        for (int k = tid; k < nc; k += T) {
            const int2 c = sm.cand[k];
            const double v = static_cast<double>(th(c.x, c.y)) + xv[c.y];
            if (order_key(v) == sm.key[c.x]) atomicMin(&sm.arg[c.x], c.y);
        }
    } else {
        // too many near-ties: every element in FP64 (the all-FP64 scan)
        for (int i = tid; i < n; i += T) {
            double m = INFINITY;
            int mi = 0;
            for (int j = 0; j < len; ++j) {
                const double v = static_cast<double>(th(i, j)) + xv[j];
                if (v < m) {
                    m = v;
                    mi = j;
                }
            }
            sm.key[i] = order_key(m);
            sm.arg[i] = mi;
        }
    }
    __syncthreads();
}

// w = fl32(x - x(0)) for j < len (0 beyond, up to pad), returns max |w|
__device__ __forceinline__ float shifted(const double *x, int len, int pad, float *w, float *red)
{
    const double x0 = x[0];
    float m = 0.f;
    for (int j = threadIdx.x; j < pad; j += blockDim.x) {
        const float v = j < len ? static_cast<float>(x[j] - x0) : 0.f;
        w[j] = v;
        m = fmaxf(m, fabsf(v));
    }
    return block_max_f(m, red);
}

template <bool REC>
__global__ void __launch_bounds__(kScrThreads) rec_screen_kernel(const EdgeDesc *edges, const int *items,
                                                                 const float *tab, double *agg, double *msg,
                                                                 unsigned char *rec, const long long *rec_off,
                                                                 int lmax)
{
    extern __shared__ __align__(16) double shd[];
    const int e = items[blockIdx.x];
    const EdgeDesc ed = edges[e];
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld, ldp = ld | 1;
    const int T = blockDim.x, tid = threadIdx.x;
    const int PM = max(T, lmax);  // partials: G groups x n lines <= max(T, n)
    ScreenSmem sm;
    sm.uh = shd;
    sm.vh = sm.uh + lmax;
    sm.al = sm.vh + lmax;
    sm.be = sm.al + lmax;
    sm.bv = sm.be + lmax;
    sm.key = reinterpret_cast<unsigned long long *>(sm.bv + lmax);
    sm.cand = reinterpret_cast<int2 *>(sm.key + lmax);
    sm.w = reinterpret_cast<float *>(sm.cand + kCandMax);
    sm.thr = sm.w + lmax;
    sm.arg = reinterpret_cast<int *>(sm.thr + lmax);
    sm.count = sm.arg + lmax;
    sm.red = reinterpret_cast<float *>(sm.count + 4);
    sm.pmin = sm.red + kScrThreads / 32;
    sm.pmax = sm.pmin + PM;
    sm.tab = sm.pmax + PM;
    unsigned short *t1 = nullptr, *s2 = nullptr, *t3 = nullptr;
    if (REC) {
        t1 = reinterpret_cast<unsigned short *>(rec + rec_off[e]);
        s2 = t1 + Lu;
        t3 = s2 + Lv;
    }
    const float *th = tab + ed.toff;
    for (int i = tid; i < Lu * ld; i += T) {
        const int s = i / ld, t = i - s * ld;
        sm.tab[s * ldp + t] = th[i];
    }
    for (int s = tid; s < Lu; s += T) sm.uh[s] = agg[ed.au + s] - msg[ed.mu + s];
    for (int t = tid; t < Lv; t += T) sm.vh[t] = agg[ed.av + t] - msg[ed.mv + t];
    __syncthreads();
    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + vh(t)] + uh(s)),  alpha = uh - a
    float D = shifted(sm.vh, Lv, Lv, sm.w, sm.red);
    screened_min<true>(sm, ldp, Lu, Lv, sm.vh, D);
    for (int s = tid; s < Lu; s += T) {
        const double a = 0.5 * (key_value(sm.key[s]) + sm.uh[s]);
        sm.al[s] = sm.uh[s] - a;
        if (REC) t1[s] = static_cast<unsigned short>(sm.arg[s]);
    }
    __syncthreads();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t),  beta = vh - b
    D = shifted(sm.al, Lu, Lu, sm.w, sm.red);
    screened_min<false>(sm, ldp, Lv, Lu, sm.al, D);
    for (int t = tid; t < Lv; t += T) {
        const double b = key_value(sm.key[t]) + sm.vh[t];
        sm.bv[t] = b;
        sm.be[t] = sm.vh[t] - b;
        if (REC) s2[t] = static_cast<unsigned short>(sm.arg[t]);
    }
    __syncthreads();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s)
    D = shifted(sm.be, Lv, Lv, sm.w, sm.red);
    screened_min<true>(sm, ldp, Lu, Lv, sm.be, D);
    for (int s = tid; s < Lu; s += T) {
        const double c = key_value(sm.key[s]) + sm.uh[s];
        agg[ed.au + s] = c;
        msg[ed.mu + s] = c - sm.uh[s];
        if (REC) t3[s] = static_cast<unsigned short>(sm.arg[s]);
    }
    for (int t = tid; t < Lv; t += T) {
        agg[ed.av + t] = sm.bv[t];
        msg[ed.mv + t] = sm.bv[t] - sm.vh[t];
    }
}

}  // namespace

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

size_t rec_screen_smem_bytes(int lmax, long long tab_floats)
{
    // uh, vh, alpha, beta, b (FP64), keys; candidates; w, thr (FP32), arg; count; red;
    // pmin, pmax; the staged table
    const size_t PM = static_cast<size_t>(std::max(kScrThreads, lmax));
    return static_cast<size_t>(lmax) * (6 * 8 + 2 * 4 + 4) + kCandMax * sizeof(int2) + 4 * 4 + 4 * (kScrThreads / 32) +
           2 * 4 * PM + 4 * static_cast<size_t>(tab_floats);
}

cudaError_t launch_rec_screen_phase(const EdgeDesc *edges, const int *items, int n_items, const float *tab,
                                    double *agg, double *msg, unsigned char *rec, const long long *rec_off, int lmax,
                                    long long tab_floats, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = rec_screen_smem_bytes(lmax, tab_floats);
    if (rec) {
        cudaError_t e = cudaFuncSetAttribute(rec_screen_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        rec_screen_kernel<true><<<n_items, kScrThreads, smem, st>>>(edges, items, tab, agg, msg, rec, rec_off, lmax);
    } else {
        cudaError_t e = cudaFuncSetAttribute(rec_screen_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        rec_screen_kernel<false><<<n_items, kScrThreads, smem, st>>>(edges, items, tab, agg, msg, nullptr, nullptr,
                                                                     lmax);
    }
    return cudaGetLastError();
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
