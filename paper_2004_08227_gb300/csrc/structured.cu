// structured.cu -- the Handshake update (Sec. 4, eq. (H), three-minimization
// form) without reading the pairwise tables, for truncated-linear costs
// theta_uv(s,t) = w_uv min(|s - t|, tau_uv) (Potts: tau = 1) and
// truncated-quadratic costs w_uv min((s - t)^2, tau_uv).  The paper notes the
// speed-up that lower envelopes give in message passing for such costs
// (Sec. 1 and Sec. 4).
//
// Each of the three minimizations has the form
//   m(s) = min_t [theta(s,t) + h(t)],   t < Lh, s < Ls.
// Window: only t within distance R of s can cost less than w tau (R the
// largest distance with |s - t| < tau, or (s - t)^2 < tau), so the window
// plus the global minimizer of h hold the minimum; used for quadratic costs
// up to R = 16 and for linear truncation up to R = 7 (Potts included), it
// reproduces the dense kernel's minimum of the same rounded values bit for
// bit.  Envelope, for quadratic costs with R > 16: the lower envelope of the
// untruncated parabolas and the global minimizer (dt_envelope).
// Scans, for longer linear truncation (w, tau >= 0): the minimum splits into
//   min_{t <= s} (h(t) - w t) + w s,   min_{t >= s} (h(t) + w t) - w s,
//   min_t h(t) + w tau,
// a prefix minimum, a suffix minimum and the global minimum of h, found by
// warp scans.  The scans only choose a minimizer in each part; the three are
// then evaluated as the dense path evaluates an entry (theta rounded to FP32
// once, as in the materialized table, then h added) and the smallest is
// taken, so a minimum differs from the dense kernel's only where rounding
// decides between candidates of equal exact value (common: reparametrized
// vectors form linear ramps along which w |s - t| + h(t) is constant).
// The vectors h, the O(L) double-float arithmetic and the write-back are
// those of the dense kernel (uh, vh; w1 = vh - vh(0), alpha, beta).
//
// One warp per edge: looped (one launch per matching) or persistent (every
// warp taking edges from one global queue, versioned waits); the tables are
// not read at all, so an update moves O(L) bytes.
#include "kernels.h"

namespace mplpp {

namespace {

constexpr int kStructThreads = 256;
constexpr int kStructWarps = kStructThreads / 32;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kWindowMax = 7;       // linear truncation radius up to which the direct window beats the scans
constexpr int kQuadWindowMax = 16;  // quadratic truncation radius up to which the window beats the envelope

struct VI {
    float v;
    int i;
};

// smaller value, then smaller index
__device__ __forceinline__ VI vi_min(VI a, VI b)
{
    return (b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

__device__ __forceinline__ VI vi_shfl_up(VI a, int o)
{
    return {__shfl_up_sync(kAll, a.v, o), __shfl_up_sync(kAll, a.i, o)};
}

__device__ __forceinline__ VI vi_shfl_down(VI a, int o)
{
    return {__shfl_down_sync(kAll, a.v, o), __shfl_down_sync(kAll, a.i, o)};
}

__device__ __forceinline__ VI vi_shfl_xor(VI a, int o)
{
    return {__shfl_xor_sync(kAll, a.v, o), __shfl_xor_sync(kAll, a.i, o)};
}

// the dense table's entry theta(s,t) in FP32: the product rounded on its own
// (never fused with a following addition, as a table entry is not)
__device__ __forceinline__ float theta_tl(int s, int t, float w, float tau, bool quad)
{
    const float d = fabsf(static_cast<float>(s - t));
    return __fmul_rn(w, fminf(quad ? __fmul_rn(d, d) : d, tau));
}

// The largest distance R with theta below w tau: |s - t| < tau (linear),
// (s - t)^2 < tau (quadratic); -1 if none.  At most 1024 (beyond any label
// count the kernel takes).
__device__ __forceinline__ int trunc_radius(float tau, bool quad)
{
    if (!(tau > 0.f)) return -1;
    if (!quad) return static_cast<int>(fminf(ceilf(tau), 1025.f)) - 1;
    float r = fminf(floorf(sqrtf(tau)), 1024.f);  // distances squared are exact up to 4096
    if (r * r >= tau) r -= 1.f;
    if (r < 1024.f && (r + 1.f) * (r + 1.f) < tau) r += 1.f;
    return static_cast<int>(r);
}

// out[s] = min over t in [s - R, s + R] and t_g of theta(s,t) + h[t]
template <bool QUAD>
__device__ __forceinline__ void dt_window(const float *h, int Lh, int Ls, float w, float tau, int R, VI g, float *out,
                                          int lane)
{
    for (int s = lane; s < Ls; s += 32) {
        float best = theta_tl(s, g.i, w, tau, QUAD) + g.v;
        const int lo = s - R > 0 ? s - R : 0, hi = s + R < Lh - 1 ? s + R : Lh - 1;
        for (int t = lo; t <= hi; ++t) best = fminf(best, theta_tl(s, t, w, tau, QUAD) + h[t]);
        out[s] = best;
    }
}

// Truncated quadratic costs with a wide truncation radius: min_t [w min((s-t)^2,
// tau) + h(t)] = min(min_t [w (s-t)^2 + h(t)], w tau + min_t h(t)), and the
// first part is the lower envelope of the parabolas w (s - t)^2 + h(t) (the
// distance transform of sampled functions, Felzenszwalb and Huttenlocher):
// lane 0 builds it in one pass over t (parabola t replaces those it covers;
// env[k] = {left end of parabola k's interval, t}), then every lane finds the
// parabola over each of its s by binary search.  The envelope only chooses
// candidates: that parabola, its two neighbours on the envelope (against the
// rounding of the breakpoints) and the global minimizer of h are evaluated as
// the dense path evaluates an entry, and the smallest is taken, so a minimum
// differs from the dense kernel's only where rounding decides between
// candidates of nearly equal value.  O(L) per minimization plus O(log L) per
// label, instead of a window of O(L) labels per label.
__device__ void dt_envelope(const float *h, int Lh, int Ls, float w, float tau, VI g, float *out, VI *env, int lane)
{
    if (lane == 0) {
        int K = 1;
        env[0] = VI{-INFINITY, 0};
        for (int q = 1; q < Lh; ++q) {
            const float fq = h[q] + w * static_cast<float>(q) * static_cast<float>(q);
            float z;
            for (;;) {
                const int p0 = env[K - 1].i;
                const float fp = h[p0] + w * static_cast<float>(p0) * static_cast<float>(p0);
                z = (fq - fp) / (2.f * w * static_cast<float>(q - p0));
                if (K > 1 && z <= env[K - 1].v) {
                    --K;  // parabola p0 lies above the envelope everywhere
                } else {
                    break;
                }
            }
            env[K++] = VI{z, q};
        }
        env[Lh] = VI{static_cast<float>(K), -1};  // the envelope's length, after its last entry
    }
    __syncwarp();
    const int K = static_cast<int>(env[Lh].v);
    for (int s = lane; s < Ls; s += 32) {
        const float x = static_cast<float>(s);
        int lo = 0, hi = K - 1;  // the last k with env[k].v <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (env[mid].v <= x) lo = mid;
            else hi = mid - 1;
        }
        float best = theta_tl(s, g.i, w, tau, true) + g.v;
        for (int k = lo > 0 ? lo - 1 : 0; k <= lo + 1 && k < K; ++k) {
            const int t = env[k].i;
            best = fminf(best, theta_tl(s, t, w, tau, true) + h[t]);
        }
        out[s] = best;
    }
    __syncwarp();
}

// out[s] = min_t [theta(s,t) + h[t]] for s < Ls, t < Lh (1 <= Lh, Ls <= 32 k);
// lane owns t in [lane k, lane k + k).  pre / suf: [Lh] scratch of the warp.
__device__ void dt_trunc(const float *h, int Lh, int Ls, float w, float tau, bool quad, float *out, VI *pre,
                         VI *suf, int lane, int k)
{
    const VI none = {INFINITY, 0x7fffffff};
    const int t0 = lane * k;
    // global minimum of h (lowest index on ties)
    VI g = none;
    for (int t = lane; t < Lh; t += 32) g = vi_min(g, VI{h[t], t});
    for (int o = 16; o > 0; o >>= 1) g = vi_min(g, vi_shfl_xor(g, o));
    // Short truncation (Potts included) and every quadratic cost: only t
    // within distance R of s can cost less than w tau, so that window plus the
    // global minimizer hold the minimum.  Every t outside the window costs
    // w tau + h(t) >= w tau + h(t_g) >= theta(s, t_g) + h(t_g) after rounding
    // (rounding is monotone), so the result is the dense kernel's minimum of
    // the same rounded values, bit for bit.
    const int R = trunc_radius(tau, quad);
    if (quad && R > kQuadWindowMax && w > 0.f) {
        dt_envelope(h, Lh, Ls, w, tau, g, out, pre, lane);
        return;
    }
    if (quad || R <= kWindowMax) {
        if (quad)
            dt_window<true>(h, Lh, Ls, w, tau, R, g, out, lane);
        else
            dt_window<false>(h, Lh, Ls, w, tau, R, g, out, lane);
        __syncwarp();
        return;
    }
    // prefix minima of h(t) - w t: this lane's run, the warp's exclusive scan
    VI run = none;
    for (int j = 0; j < k; ++j) {
        const int t = t0 + j;
        if (t < Lh) {
            run = vi_min(run, VI{h[t] - w * static_cast<float>(t), t});
            pre[t] = run;
        }
    }
    VI inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const VI x = vi_shfl_up(inc, o);
        if (lane >= o) inc = vi_min(x, inc);  // the earlier lanes' (lower t) minimum first
    }
    VI exc = vi_shfl_up(inc, 1);
    if (lane == 0) exc = none;
    for (int j = 0; j < k; ++j) {
        const int t = t0 + j;
        if (t < Lh) pre[t] = vi_min(exc, pre[t]);
    }
    // suffix minima of h(t) + w t
    run = none;
    for (int j = k - 1; j >= 0; --j) {
        const int t = t0 + j;
        if (t < Lh) {
            run = vi_min(run, VI{h[t] + w * static_cast<float>(t), t});
            suf[t] = run;
        }
    }
    inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const VI x = vi_shfl_down(inc, o);
        if (lane + o < 32) inc = vi_min(inc, x);
    }
    exc = vi_shfl_down(inc, 1);
    if (lane == 31) exc = none;
    for (int j = 0; j < k; ++j) {
        const int t = t0 + j;
        if (t < Lh) suf[t] = vi_min(suf[t], exc);
    }
    __syncwarp();
    // the three parts' minimizers, each evaluated exactly as the dense path
    // evaluates an entry (the scans' keys h(t) -+ w t round at the scale of
    // w t, so they only choose within each part)
    for (int s = lane; s < Ls; s += 32) {
        const int tp = pre[min(s, Lh - 1)].i;
        VI best = {theta_tl(s, tp, w, tau, false) + h[tp], tp};
        if (s < Lh) {
            const int ts = suf[s].i;
            best = vi_min(best, VI{theta_tl(s, ts, w, tau, false) + h[ts], ts});
        }
        best = vi_min(best, VI{theta_tl(s, g.i, w, tau, false) + g.v, g.i});
        out[s] = best.v;
    }
    __syncwarp();
}

// One structured Handshake update of edge e by one warp.  SIGNAL (persistent
// form): the node entries are polled until they carry the versions in ver, and
// the new entries carry ver + 1; otherwise versions are not checked and the
// new entries carry 1 (the looped driver orders the matchings by launches).
template <bool SIGNAL>
__device__ void struct_item(const StructParams &p, int e, const EdgeDesc &ed, Versions ver, char *base, int lane)
{
    const int lmax = p.lmax;
    // per warp: uh, vh (double-float), h and m (FP32), pre and suf (value, index)
    float2 *uh = reinterpret_cast<float2 *>(base);
    float2 *vh = uh + lmax;
    float *h = reinterpret_cast<float *>(vh + lmax);
    float *m = h + lmax;
    VI *pre = reinterpret_cast<VI *>(m + lmax);
    VI *suf = pre + lmax;

    const float2 wt = p.param[e];
    const float w = wt.x, tau = wt.y;
    const bool quad = p.kind[e] == kPairQuad;
    const int Lu = ed.Lu, Lv = ed.Lv;
    ulonglong2 *agg = p.agg;
    ulonglong2 *msg = p.msg;
    const unsigned va = ver.u + ver.bump;

    // unaries without this edge's messages: up to kB entries of each node per
    // lane requested before any is used (one round trip per 32 kB labels; the
    // polling form holds them across its waits, so it takes 2 per lane to keep
    // its registers -- and co-resident warps -- at the looped form's count)
    constexpr int kB = SIGNAL ? 2 : 4;
    const int Lm = Lu > Lv ? Lu : Lv;
    for (int base0 = 0; base0 < Lm; base0 += 32 * kB) {
        ulonglong2 xu[kB], mu[kB], xv[kB], mv[kB];
#pragma unroll
        for (int j = 0; j < kB; ++j) {
            const int i = base0 + lane + 32 * j;
            if (i < Lu) {
                xu[j] = ld_se(agg + ed.au + i);
                mu[j] = ld_se(msg + ed.mu + i);
            }
            if (i < Lv) {
                xv[j] = ld_se(agg + ed.av + i);
                mv[j] = ld_se(msg + ed.mv + i);
            }
        }
        if (SIGNAL) {  // bounded wait for the expected versions; only stale words are requested again
            for (long long spins = 1;; ++spins) {
                bool ok = true;
#pragma unroll
                for (int j = 0; j < kB; ++j) {
                    const int i = base0 + lane + 32 * j;
                    if (i < Lu) ok = ok && se_ok(xu[j], va) && se_ok(mu[j], ver.e);
                    if (i < Lv) ok = ok && se_ok(xv[j], ver.v) && se_ok(mv[j], ver.e);
                }
                if (ok) break;
                if ((spins & 63) == 0 && *reinterpret_cast<volatile int *>(p.err) != 0) break;  // draining
                if (spins > p.spin_limit) {
                    atomicCAS(p.err, 0, ERR_TIMEOUT);
                    break;
                }
                if (spins > 64) __nanosleep(64);
#pragma unroll
                for (int j = 0; j < kB; ++j) {
                    const int i = base0 + lane + 32 * j;
                    if (i < Lu) {
                        if (!se_ok(xu[j], va)) xu[j] = ld_se(agg + ed.au + i);
                        if (!se_ok(mu[j], ver.e)) mu[j] = ld_se(msg + ed.mu + i);
                    }
                    if (i < Lv) {
                        if (!se_ok(xv[j], ver.v)) xv[j] = ld_se(agg + ed.av + i);
                        if (!se_ok(mv[j], ver.e)) mv[j] = ld_se(msg + ed.mv + i);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kB; ++j) {
            const int i = base0 + lane + 32 * j;
            if (i < Lu) uh[i] = df_sub(se_df(xu[j]), se_df(mu[j]));
            if (i < Lv) vh[i] = df_sub(se_df(xv[j]), se_df(mv[j]));
        }
    }
    __syncwarp();
    const float2 vref = vh[0];
    for (int t = lane; t < Lv; t += 32) h[t] = df_to_f(df_sub(vh[t], vref));
    __syncwarp();
    const int ku = (Lu + 31) >> 5, kv = (Lv + 31) >> 5;
    const unsigned nu = SIGNAL ? ver.u + 1u : 1u, nv = SIGNAL ? ver.v + 1u : 1u, ne = SIGNAL ? ver.e + 1u : 1u;

    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + w1(t)] + vh(0) + uh(s)); alpha = uh - a
    dt_trunc(h, Lv, Lu, w, tau, quad, m, pre, suf, lane, kv);
    for (int s = lane; s < Lu; s += 32) {
        // alpha = uh - a = 1/2 (uh - vh(0) - m), its value in exact arithmetic
        h[s] = df_to_f(df_half(df_add_f(df_sub(uh[s], vref), -m[s])));
    }
    __syncwarp();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t); beta = vh - b; node v's new vector
    dt_trunc(h, Lu, Lv, w, tau, quad, m, pre, suf, lane, ku);
    for (int t = lane; t < Lv; t += 32) {
        const float2 b = df_add_f(vh[t], m[t]);
        h[t] = -m[t];  // beta = vh - b, in exact arithmetic
        st_se(agg + ed.av + t, se_make(b, nv));
        st_se(msg + ed.mv + t, se_make(df_sub(b, vh[t]), ne));
    }
    __syncwarp();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s); node u's new vector
    dt_trunc(h, Lv, Lu, w, tau, quad, m, pre, suf, lane, kv);
    for (int s = lane; s < Lu; s += 32) {
        const float2 c = df_add_f(uh[s], m[s]);
        st_se(agg + ed.au + s, se_make(c, nu));
        st_se(msg + ed.mu + s, se_make(df_sub(c, uh[s]), ne));
    }
    __syncwarp();  // the warp's vectors are rewritten by its next item
}

__global__ void __launch_bounds__(kStructThreads) struct_kernel(StructParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int item = blockIdx.x * kStructWarps + wib;
    if (item >= p.n_items) return;
    const int e = p.items[item];
    struct_item<false>(p, e, p.edges[e], Versions{0u, 0u, 0u, 0u},
                       smem_raw + static_cast<size_t>(wib) * struct_bytes_per_warp(p.lmax), lane);
}

// Persistent form: every warp takes the next item of one global queue (the
// list of the queue driver, handshake.cu: each model's updates in schedule
// order, the models interleaved by progress) until the iterations are done.
// Every wait is on an earlier item, held by a co-resident warp, so the waits
// end; no block barrier.
__global__ void __launch_bounds__(kStructThreads, 4) struct_queue_kernel(StructParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    char *base = smem_raw + static_cast<size_t>(wib) * struct_bytes_per_warp(p.lmax);
    const long long EE = p.queue_items, total = EE * static_cast<long long>(p.iterations);
    for (long long k = 0;; ++k) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(p.queue, 1ull);
        g = __shfl_sync(kAll, g, 0);
        if (static_cast<long long>(g) >= total) break;
        const WorkItem *w = p.work + static_cast<long long>(g) % EE;
        const long long it = static_cast<long long>(g) / EE;
        const int e = __ldg(&w->edge);
        const Versions ver = {static_cast<unsigned>(it) * static_cast<unsigned>(__ldg(&w->deg_u)) +
                                  static_cast<unsigned>(__ldg(&w->pos_u)),
                              static_cast<unsigned>(it) * static_cast<unsigned>(__ldg(&w->deg_v)) +
                                  static_cast<unsigned>(__ldg(&w->pos_v)),
                              static_cast<unsigned>(it),
                              (p.test_wait && k == 0 && blockIdx.x == 0 && wib == 0) ? 1u : 0u};
        struct_item<true>(p, e, p.edges[e], ver, base, lane);
    }
}

// tables of structured edges from their parameters, as the caller would have
// given them densely (rows padded to ld with +inf)
__global__ void materialize_kernel(const EdgeDesc *edges, const float2 *param, const int *kind, int n, float *tab,
                                   int *err)
{
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        const float2 wt = param[e];
        const bool quad = kind[e] == kPairQuad;
        if (!(isfinite(wt.x) && isfinite(wt.y) && wt.x >= 0.f && wt.y >= 0.f)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, ERR_NONFINITE);
            continue;
        }
        const long long n_ent = static_cast<long long>(ed.Lu) * ed.ld;
        for (long long i = threadIdx.x; i < n_ent; i += blockDim.x) {
            const int s = static_cast<int>(i / ed.ld);
            const int t = static_cast<int>(i - static_cast<long long>(s) * ed.ld);
            tab[ed.toff + i] = t < ed.Lv ? theta_tl(s, t, wt.x, wt.y, quad) : INFINITY;
        }
    }
}

}  // namespace

cudaError_t struct_prepare(int lmax)
{
    return raise_smem_limit(struct_kernel, kStructWarps * struct_bytes_per_warp(lmax));
}

cudaError_t launch_struct(const StructParams &p, cudaStream_t st)
{
    if (p.n_items <= 0) return cudaSuccess;
    const int blocks = (p.n_items + kStructWarps - 1) / kStructWarps;
    struct_kernel<<<blocks, kStructThreads, kStructWarps * struct_bytes_per_warp(p.lmax), st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_struct_queue(const StructParams &p, int blocks, cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;  // (shared memory attribute set by struct_queue_max_blocks)
    struct_queue_kernel<<<blocks, kStructThreads, kStructWarps * struct_bytes_per_warp(p.lmax), st>>>(p);
    return cudaGetLastError();
}

int struct_queue_max_blocks(int lmax)
{
    const size_t smem = kStructWarps * struct_bytes_per_warp(lmax);
    if (raise_smem_limit(struct_queue_kernel, smem) != cudaSuccess) return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, struct_queue_kernel, kStructThreads, smem) !=
        cudaSuccess)
        return 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

cudaError_t launch_materialize(const EdgeDesc *edges, const float2 *param, const int *kind, int n, float *tab,
                               int *err, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    materialize_kernel<<<n < 4096 ? n : 4096, 256, 0, st>>>(edges, param, kind, n, tab, err);
    return cudaGetLastError();
}

}  // namespace mplpp
