// resident.cu -- the MPLP++ Handshake update with a whole model resident in one
// CTA (resident driver), for many small models (label counts <= 32).
//
// The update is the one of handshake.cu (Sec. 4, eq. (H), three-minimization
// form, message-form state, double-float O(L) arithmetic, FP32 minimizations
// on shifted operands) with the same operations per element and the same
// double-float steps, so it gives the same state bit for bit as every other
// driver.  What differs is where the state lives: one CTA owns one model for
// all iterations, keeps its reparametrized unaries and messages in shared
// memory, and separates the matchings by a block barrier -- the barrier
// between matchings of the paper's GPU implementation (Sec. 6) at the scope
// of a CTA.  Nothing waits on another CTA and no state crosses L2 between
// updates; the tables are read from L2 once the first iteration has touched
// them (the kernel can stage a model's tables in shared memory too, which
// the host does not select: fewer models then share an SM).  One warp updates one edge of a matching: lane s holds row s
// of the table and lane t column t (loaded together, in registers), so every
// minimization is a sequential loop in one lane, with no shuffles.
#include <cfloat>
#include <cstdint>

#include "kernels.h"

namespace mplpp {

namespace {

// Per-warp vectors of the edge being updated.
struct ResWarp {
    float2 *uh, *vh;           // [32] double-float unaries without this edge's messages
    float *w1, *alpha, *beta;  // [32] FP32 shifted operands of passes 1, 2 and 3
};

__device__ __forceinline__ ResWarp res_warp(char *base, int warp)
{
    char *b = base + static_cast<size_t>(warp) * kResWarpBytes;
    ResWarp r;
    r.uh = reinterpret_cast<float2 *>(b);
    r.vh = r.uh + kResMaxL;
    r.w1 = reinterpret_cast<float *>(r.vh + kResMaxL);
    r.alpha = r.w1 + kResMaxL;
    r.beta = r.alpha + kResMaxL;
    return r;
}

// One Handshake update of edge ed (L_u, L_v <= LM <= 32) by one warp, on the
// model's shared-memory state: agg and msg hold the model's entries (offsets
// relative to the model's first node and first edge).
template <int LM>
__device__ __forceinline__ void res_update(const EdgeDesc &ed, const float *tab, long long tbase, float2 *agg,
                                           float2 *msg, long long abase, long long mbase, const ResWarp &w, int lane)
{
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld;
    float2 *au = agg + (ed.au - abase), *av = agg + (ed.av - abase);
    float2 *mu = msg + (ed.mu - mbase), *mv = msg + (ed.mv - mbase);
    // row `lane` and column `lane` of the table (FP32, +inf beyond the labels)
    float row[LM], col[LM];
    const float *th = tab + (ed.toff - tbase);
#pragma unroll
    for (int t = 0; t < LM; ++t) row[t] = (lane < Lu && t < Lv) ? th[lane * ld + t] : INFINITY;
#pragma unroll
    for (int s = 0; s < LM; ++s) col[s] = (lane < Lv && s < Lu) ? th[s * ld + lane] : INFINITY;
    if (lane < Lu) w.uh[lane] = df_sub(au[lane], mu[lane]);
    if (lane < Lv) w.vh[lane] = df_sub(av[lane], mv[lane]);
    __syncwarp();
    const float2 vref = w.vh[0];
    if (lane < Lv) w.w1[lane] = df_to_f(df_sub(w.vh[lane], vref));
    __syncwarp();
    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + w1(t)] + vh(0) + uh(s));  alpha = uh - a
    if (lane < Lu) {
        float m = INFINITY;
#pragma unroll
        for (int t = 0; t < LM; ++t)
            if (t < Lv) m = fminf(m, row[t] + w.w1[t]);
        const float2 u = w.uh[lane];
        const float2 a = df_half(df_add(df_add_f(vref, m), u));
        w.alpha[lane] = df_to_f(df_sub(u, a));
    }
    __syncwarp();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t),  beta = vh - b
    if (lane < Lv) {
        float m = INFINITY;
#pragma unroll
        for (int s = 0; s < LM; ++s)
            if (s < Lu) m = fminf(m, col[s] + w.alpha[s]);
        const float2 vh = w.vh[lane];
        const float2 b = df_add_f(vh, m);
        w.beta[lane] = df_to_f(df_sub(vh, b));
        av[lane] = b;
        mv[lane] = df_sub(b, vh);
    }
    __syncwarp();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s)
    if (lane < Lu) {
        float m = INFINITY;
#pragma unroll
        for (int t = 0; t < LM; ++t)
            if (t < Lv) m = fminf(m, row[t] + w.beta[t]);
        const float2 u = w.uh[lane];
        const float2 c = df_add_f(u, m);
        au[lane] = c;
        mu[lane] = df_sub(c, u);
    }
    __syncwarp();  // the warp's vectors are rewritten by its next update
}

template <int LM>
__global__ void __launch_bounds__(512) hs_resident_kernel(ResParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int m = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const ResModel md = p.models[m];
    float2 *agg = reinterpret_cast<float2 *>(smem_raw);
    float2 *msg = agg + md.agg_n;
    char *wbase = reinterpret_cast<char *>(msg + md.msg_n);
    const ResWarp w = res_warp(wbase, warp);
    // the model's state from the solver's versioned entries, and its tables
    for (long long i = tid; i < md.agg_n; i += blockDim.x) agg[i] = se_df(p.agg[md.agg_base + i]);
    for (long long i = tid; i < md.msg_n; i += blockDim.x) msg[i] = se_df(p.msg[md.msg_base + i]);
    const float *tab = p.tab;
    long long tbase = 0;
    if (p.stage_tables) {  // 16-byte aligned: the warp vectors are a multiple of 16 bytes
        float4 *st = reinterpret_cast<float4 *>(wbase + static_cast<size_t>(W) * kResWarpBytes);
        const float4 *src = reinterpret_cast<const float4 *>(p.tab + md.tab_base);
        for (long long i = tid; i < md.tab_n / 4; i += blockDim.x) st[i] = src[i];
        tab = reinterpret_cast<const float *>(st);
        tbase = md.tab_base;
    }
    __syncthreads();
    const int *off = p.sched_off + md.sched;  // [P + 1] matchings of this model
    for (int it = 0; it < p.iterations; ++it)
        for (int k = 0; k < md.P; ++k) {
            for (int j = off[k] + warp; j < off[k + 1]; j += W) {
                const EdgeDesc ed = p.edges[p.sched_edges[j]];
                res_update<LM>(ed, tab, tbase, agg, msg, md.agg_base, md.msg_base, w, lane);
            }
            __syncthreads();  // the barrier between matchings
        }
    for (long long i = tid; i < md.agg_n; i += blockDim.x) p.agg[md.agg_base + i] = se_make(agg[i], 0u);
    for (long long i = tid; i < md.msg_n; i += blockDim.x) p.msg[md.msg_base + i] = se_make(msg[i], 0u);
}

}  // namespace

cudaError_t res_prepare(size_t smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(hs_resident_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(hs_resident_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(hs_resident_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
}

// lmax: the largest label count of the solver (<= kResMaxL): the register
// arrays of a lane's row and column are sized 8, 16 or 32.
cudaError_t launch_resident(const ResParams &p, int n_models, int threads, size_t smem, int lmax, cudaStream_t st)
{
    if (n_models <= 0) return cudaSuccess;
    if (lmax <= 8)
        hs_resident_kernel<8><<<n_models, threads, smem, st>>>(p);
    else if (lmax <= 16)
        hs_resident_kernel<16><<<n_models, threads, smem, st>>>(p);
    else
        hs_resident_kernel<32><<<n_models, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace mplpp
