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
// is among the candidates.  One group of G threads (a power of two, G lines
// per block of threads; the groups of a warp hold consecutive lines) handles
// a line: both FP32 scans and the bound from the line's own h and
// max |w(j)|.  The warp's candidates are appended to a per-warp list and
// evaluated in FP64 32 at a time (one candidate per lane: GB300 issues an FP64
// instruction at the cost of a full warp however few lanes are active), and
// merged into their line's minimum with 64-bit shared-memory atomics on an
// order-preserving key (value first, then the lowest index among equal
// values), so neither the order of the list nor of the lanes matters.  A warp
// whose list overflows scans its lines in FP64 entirely.  One block barrier
// per pass.  The table is staged in shared memory with an odd row stride.
namespace {

constexpr int kScrThreads = 256;
constexpr int kWarpCands = 128;  // candidates per warp and pass
constexpr int kSpanReg = 16;     // a thread's sums of a line kept in registers (up to this many)

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

// m(i) = min_j [theta(i, j) + x(j)], j < len, for every line i < n (rows of the
// staged table when ROWS, else columns), with its lowest argmin; w(j) =
// fl32(x(j) - x(0)).  key / arg: [n] per-line scratch; cand: this warp's list
// [kWarpCands].  emit(i, m, argmin) runs on the line group's first thread.
template <bool ROWS, typename F>
__device__ __forceinline__ void screened_lines(const float *tab, int ldp, int n, int len, const double *xv,
                                               const float *w, unsigned long long *key, int *arg, int2 *cand, F emit)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    int G = 32;
    while (G > 1 && G * n > T) G >>= 1;
    const int k = tid & (G - 1), g0 = tid / G, ng = T / G;
    const float ax0 = __double2float_ru(fabs(xv[0]));
    auto th = [&](int i, int j) { return ROWS ? tab[i * ldp + j] : tab[j * ldp + i]; };
    const int span = (len + G - 1) / G;  // elements of a line per thread
    const bool reg = span <= kSpanReg;
    for (int base = 0; base < n; base += ng) {  // the same trip count in every thread
        const int i = base + g0;
        const bool on = i < n;
        float mn = INFINITY, h = 0.f, d = 0.f;
        float sv[kSpanReg];  // the FP32 sums, for the candidate test
#pragma unroll
        for (int r = 0; r < kSpanReg; ++r) {
            const int j = k + r * G;
            sv[r] = INFINITY;
            if (on && j < len) {
                const float t = th(i, j);
                const float wj = w[j];
                sv[r] = t + wj;
                mn = fminf(mn, sv[r]);
                h = fmaxf(h, fabsf(t));
                d = fmaxf(d, fabsf(wj));
            }
        }
        if (on)
            for (int j = k + kSpanReg * G; j < len; j += G) {
                const float t = th(i, j);
                const float wj = w[j];
                mn = fminf(mn, t + wj);
                h = fmaxf(h, fabsf(t));
                d = fmaxf(d, fabsf(wj));
            }
        for (int o = G >> 1; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
            d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
        }
        // c(jc) + 2 e1 + 2 e2, every operation rounded upwards (d bounds |w| on the line)
        const float e1 = __fmul_ru(0x1p-22f, __fadd_ru(h, d));
        const float e2 = __fmul_ru(0x1p-50f, __fadd_ru(__fadd_ru(h, d), ax0));
        const float thr = __fadd_ru(__fadd_ru(mn, __fmul_ru(2.f, e1)), __fadd_ru(__fmul_ru(2.f, e2), 0x1p-126f));
        if (on && k == 0) {
            key[i] = ~0ull;
            arg[i] = INT_MAX;
        }
        // the warp's candidates into its list (warp-uniform trip count; the
        // list's order does not matter)
        int nc = 0;
        bool over = false;
        if (reg) {
            // a mask of the thread's candidates, a prefix sum of the counts over the warp
            unsigned m = 0u;
#pragma unroll
            for (int r = 0; r < kSpanReg; ++r)
                if (sv[r] <= thr) m |= 1u << r;  // +inf beyond the line (thr is finite)
            const int cnt = __popc(m);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            nc = __shfl_sync(0xffffffffu, incl, 31);
            for (int slot = incl - cnt; m; m &= m - 1u, ++slot)
                if (slot < kWarpCands) cand[slot] = make_int2(i, k + (__ffs(m) - 1) * G);
        } else {
            for (int r = 0; r < span; ++r) {
                const int j = k + r * G;
                const bool c = on && j < len && th(i, j) + w[j] <= thr;
                const unsigned mask = __ballot_sync(0xffffffffu, c);
                const int slot = nc + __popc(mask & ((1u << lane) - 1u));
                if (c && slot < kWarpCands) cand[slot] = make_int2(i, j);
                nc += __popc(mask);
            }
        }
        if (nc > kWarpCands) {
            over = true;
            nc = 0;
        }
        __syncwarp();
        if (!over) {
            // FP64 values, 32 candidates per instruction, merged per line; the
            // keys stay in registers for the argmin step (FP64 is computed once)
            unsigned long long kv[kWarpCands / 32];
#pragma unroll
            for (int r = 0; r < kWarpCands / 32; ++r) {
                const int c = lane + 32 * r;
                if (c < nc) {
                    const int2 q = cand[c];
                    kv[r] = order_key(static_cast<double>(th(q.x, q.y)) + xv[q.y]);
                    atomicMin(&key[q.x], kv[r]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < kWarpCands / 32; ++r) {
                const int c = lane + 32 * r;
                if (c < nc) {
                    const int2 q = cand[c];
                    if (kv[r] == key[q.x]) atomicMin(&arg[q.x], q.y);
                }
            }
            __syncwarp();
        } else if (on && k == 0) {
            // too many near-ties in this warp's lines: every element in FP64
            double m = INFINITY;
            int mi = 0;
            for (int j = 0; j < len; ++j) {
                const double v = static_cast<double>(th(i, j)) + xv[j];
                if (v < m) {
                    m = v;
                    mi = j;
                }
            }
            key[i] = order_key(m);
            arg[i] = mi;
        }
        __syncwarp();
        if (on && k == 0) emit(i, key_value(key[i]), arg[i]);
    }
}

template <bool REC>
// descs, rec_off: the matching's edges and their record offsets, in schedule
// order (one independent load each per block)
__global__ void __launch_bounds__(kScrThreads, 4) rec_screen_kernel(const EdgeDesc *descs, const float *tab,
                                                                 double *agg, double *msg, unsigned char *rec,
                                                                 const long long *rec_off, int lmax)
{
    extern __shared__ __align__(16) double shd[];
    const EdgeDesc ed = descs[blockIdx.x];
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld, ldp = ld | 1;
    const int T = blockDim.x, tid = threadIdx.x, warp = tid >> 5;
    double *uh = shd, *vh = uh + lmax, *al = vh + lmax, *be = al + lmax, *bv = be + lmax;
    unsigned long long *key = reinterpret_cast<unsigned long long *>(bv + lmax);  // [lmax] per-line minima
    int2 *cand = reinterpret_cast<int2 *>(key + lmax) + warp * kWarpCands;      // this warp's list
    int *arg = reinterpret_cast<int *>(reinterpret_cast<int2 *>(key + lmax) + (kScrThreads / 32) * kWarpCands);
    float *w = reinterpret_cast<float *>(arg + lmax);  // [lmax] the current pass's shifted vector
    float *st = w + lmax;                              // [Lu][ldp] staged table
    unsigned short *t1 = nullptr, *s2 = nullptr, *t3 = nullptr;
    if (REC) {
        t1 = reinterpret_cast<unsigned short *>(rec + rec_off[blockIdx.x]);
        s2 = t1 + Lu;
        t3 = s2 + Lv;
    }
    // the node vectors (requested first), the table (16-byte chunks, a
    // thread's next eight requested before any is stored, so the loads
    // overlap), shifted vh
    const double vh0 = agg[ed.av] - msg[ed.mv];
    for (int s = tid; s < Lu; s += T) uh[s] = agg[ed.au + s] - msg[ed.mu + s];
    for (int t = tid; t < Lv; t += T) vh[t] = agg[ed.av + t] - msg[ed.mv + t];
    const float4 *th4 = reinterpret_cast<const float4 *>(tab + ed.toff);
    const int Q = ld >> 2, nq = Lu * Q;
    for (int base = tid; base < nq; base += 8 * T) {
        float4 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (base + r * T < nq) v[r] = th4[base + r * T];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int c = base + r * T;
            if (c < nq) {
                const int s = c / Q;
                float *d = st + s * ldp + 4 * (c - s * Q);
                d[0] = v[r].x;
                d[1] = v[r].y;
                d[2] = v[r].z;
                d[3] = v[r].w;
            }
        }
    }
    for (int t = tid; t < Lv; t += T) w[t] = static_cast<float>(vh[t] - vh0);
    __syncthreads();
    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + vh(t)] + uh(s)),  alpha = uh - a
    screened_lines<true>(st, ldp, Lu, Lv, vh, w, key, arg, cand, [&](int s, double m, int mi) {
        const double a = 0.5 * (m + uh[s]);
        al[s] = uh[s] - a;
        if (REC) t1[s] = static_cast<unsigned short>(mi);
    });
    __syncthreads();
    for (int s = tid; s < Lu; s += T) w[s] = static_cast<float>(al[s] - al[0]);
    __syncthreads();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t),  beta = vh - b
    screened_lines<false>(st, ldp, Lv, Lu, al, w, key, arg, cand, [&](int t, double m, int mi) {
        const double b = m + vh[t];
        bv[t] = b;
        be[t] = vh[t] - b;
        if (REC) s2[t] = static_cast<unsigned short>(mi);
    });
    __syncthreads();
    for (int t = tid; t < Lv; t += T) {
        w[t] = static_cast<float>(be[t] - be[0]);
        agg[ed.av + t] = bv[t];
        msg[ed.mv + t] = bv[t] - vh[t];
    }
    __syncthreads();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s)
    screened_lines<true>(st, ldp, Lu, Lv, be, w, key, arg, cand, [&](int s, double m, int mi) {
        const double c = m + uh[s];
        agg[ed.au + s] = c;
        msg[ed.mu + s] = c - uh[s];
        if (REC) t3[s] = static_cast<unsigned short>(mi);
    });
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
    // uh, vh, alpha, beta, b (FP64), keys; the warps' candidate lists; args; w (FP32); the staged table
    return static_cast<size_t>(lmax) * (6 * 8 + 4 + 4) + sizeof(int2) * (kScrThreads / 32) * kWarpCands +
           4 * static_cast<size_t>(tab_floats);
}

cudaError_t launch_rec_screen_phase(const EdgeDesc *descs, int n_items, const float *tab,
                                    double *agg, double *msg, unsigned char *rec, const long long *rec_off, int lmax,
                                    long long tab_floats, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = rec_screen_smem_bytes(lmax, tab_floats);
    if (rec) {
        cudaError_t e = raise_smem_limit(rec_screen_kernel<true>, smem);
        if (e != cudaSuccess) return e;
        rec_screen_kernel<true><<<n_items, kScrThreads, smem, st>>>(descs, tab, agg, msg, rec, rec_off, lmax);
    } else {
        cudaError_t e = raise_smem_limit(rec_screen_kernel<false>, smem);
        if (e != cudaSuccess) return e;
        rec_screen_kernel<false><<<n_items, kScrThreads, smem, st>>>(descs, tab, agg, msg, nullptr, nullptr, lmax);
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
            cudaError_t e = raise_smem_limit(rec64_phase_kernel<true>, smem);
            if (e != cudaSuccess) return e;
        }
        rec64_phase_kernel<true><<<n_items, kThreads, smem, st>>>(edges, items, tab, agg, msg, rec, rec_off, lmax);
    } else {
        if (smem > 48 * 1024) {
            cudaError_t e = raise_smem_limit(rec64_phase_kernel<false>, smem);
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
