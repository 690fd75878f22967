// rules.cu -- the MPLP update (Sec. 4, eq. (M)) and the uniform update
// (Sec. 4, eq. (U)) on the solver's message-form state, as alternatives to the
// Handshake update for the paper's dominance comparison (Prop. 2: H >= M >= U
// after one update; Thm. 2: the same for one iteration from equal states).
//
// With uh(s) = agg_u(s) - phi_{v->u}(s), vh(t) = agg_v(t) - phi_{u->v}(t) and
// g(s,t) = theta_uv(s,t) + uh(s) + vh(t) (the pairwise table is never written):
//   M:  agg_u(s) := 1/2 min_t g(s,t),        agg_v(t) := 1/2 min_s g(s,t)
//   U:  agg_u(s) := agg_v(t) := 1/2 min_{s,t} g(s,t)
// and phi_{v->u} := agg_u - uh, phi_{u->v} := agg_v - vh, so that the
// reparametrized table g - agg_u - agg_v stays implicit.
//
// Precision as in the Handshake kernel: the O(L^2) minimizations run in FP32
// on the table plus a shifted copy of the other node's vector rounded once to
// FP32 (w1(t) = vh(t) - vh(0) for row minima, w2(s) = uh(s) - uh(0) for column
// minima); the O(L) arithmetic is double-float.  The row minimum feeds the
// same expression as the Handshake kernel's first pass, so M's node-u result
// equals the Handshake a(s) bit for bit.
//
// One CTA per edge of a matching (one launch per matching, the launch boundary
// is the barrier).  Row minima: one warp per row, coalesced float4 reads of
// the row and a hardware warp reduction.  Column minima (M): one thread per
// float4 column chunk, walking the rows (coalesced across the threads); the
// table is read twice, the second time mostly from L2 for tables up to a few
// MB per matching.  U needs the row pass only.
#include "kernels.h"

namespace mplpp {

namespace {

constexpr int kRuleThreads = 256;

__device__ __forceinline__ float warp_min(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// a < b for normalized double-float values
__device__ __forceinline__ bool df_less(float2 a, float2 b)
{
    return a.x < b.x || (a.x == b.x && a.y < b.y);
}

__device__ __forceinline__ float2 df_min(float2 a, float2 b)
{
    return df_less(b, a) ? b : a;
}

__device__ __forceinline__ float2 df_shfl_xor(float2 v, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ void put(ulonglong2 *agg_e, ulonglong2 *msg_e, float2 val, float2 base)
{
    // looped updates: entries carry version 1 (the persistent drivers restamp)
    st_se(agg_e, se_make(val, 1u));
    st_se(msg_e, se_make(df_sub(val, base), 1u));
}

template <int RULE>
__global__ void __launch_bounds__(kRuleThreads) rule_kernel(RuleParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const EdgeDesc ed = p.edges[p.items[blockIdx.x]];
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld, Q = ld >> 2;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, W = T >> 5;
    const int lu4 = (Lu + 3) & ~3;
    float2 *uh = reinterpret_cast<float2 *>(smem_raw);  // [lu4]
    float2 *vh = uh + lu4;                               // [ld]
    float2 *red = vh + ld;                               // [32] (U)
    float *w1 = reinterpret_cast<float *>(red + 32);     // [ld]   16-byte aligned: every array above is
    float *w2 = w1 + ld;                                 // [lu4]  a multiple of 16 bytes
    ulonglong2 *agg = p.agg;
    ulonglong2 *msg = p.msg;

    for (int s = tid; s < Lu; s += T)
        uh[s] = df_sub(se_df(ld_se(agg + ed.au + s)), se_df(ld_se(msg + ed.mu + s)));
    for (int t = tid; t < ld; t += T)
        vh[t] = t < Lv ? df_sub(se_df(ld_se(agg + ed.av + t)), se_df(ld_se(msg + ed.mv + t))) : make_float2(0.f, 0.f);
    __syncthreads();
    const float2 vref = vh[0], uref = uh[0];
    for (int t = tid; t < ld; t += T) w1[t] = t < Lv ? df_to_f(df_sub(vh[t], vref)) : 0.f;
    if (RULE == kRuleM)
        for (int s = tid; s < Lu; s += T) w2[s] = df_to_f(df_sub(uh[s], uref));
    __syncthreads();

    const float4 *t4 = reinterpret_cast<const float4 *>(p.tab + ed.toff);
    const float4 *w14 = reinterpret_cast<const float4 *>(w1);
    // rows: G(s) = min_t g(s,t) = min_t [theta(s,t) + w1(t)] + vh(0) + uh(s)
    float2 gmin = make_float2(INFINITY, 0.f);
    for (int s = warp; s < Lu; s += W) {
        const float4 *row = t4 + static_cast<size_t>(s) * Q;
        float m = INFINITY;
        for (int q = lane; q < Q; q += 32) m = min_add4(m, row[q], w14[q]);
        m = warp_min(m);
        const float2 g = df_add(df_add_f(vref, m), uh[s]);
        if (RULE == kRuleM) {
            if (lane == 0) put(agg + ed.au + s, msg + ed.mu + s, df_half(g), uh[s]);
        } else {
            gmin = df_min(gmin, g);
        }
    }
    if (RULE == kRuleM) {
        // columns: min_s g(s,t) = min_s [theta(s,t) + w2(s)] + uh(0) + vh(t)
        for (int q = tid; q < Q; q += T) {
            float4 m = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
            for (int s = 0; s < Lu; ++s) m = min4(m, add4s(t4[static_cast<size_t>(s) * Q + q], w2[s]));
            const float mc[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = 4 * q + j;
                if (t < Lv) put(agg + ed.av + t, msg + ed.mv + t, df_half(df_add(df_add_f(uref, mc[j]), vh[t])), vh[t]);
            }
        }
    } else {
        // min over the CTA's rows (every lane of a warp holds its warp's minimum)
        if (lane == 0) red[warp] = gmin;
        __syncthreads();
        if (warp == 0) {
            float2 v = lane < W ? red[lane] : make_float2(INFINITY, 0.f);
            for (int o = 16; o > 0; o >>= 1) v = df_min(v, df_shfl_xor(v, o));
            if (lane == 0) red[0] = v;
        }
        __syncthreads();
        const float2 half = df_half(red[0]);
        for (int s = tid; s < Lu; s += T) put(agg + ed.au + s, msg + ed.mu + s, half, uh[s]);
        for (int t = tid; t < Lv; t += T) put(agg + ed.av + t, msg + ed.mv + t, half, vh[t]);
    }
}

}  // namespace

size_t rule_smem_bytes(int lumax, int ldmax)
{
    const size_t lu4 = (static_cast<size_t>(lumax) + 3) & ~static_cast<size_t>(3);
    return (lu4 + ldmax + 32) * sizeof(float2) + (static_cast<size_t>(ldmax) + lu4) * sizeof(float);
}

cudaError_t rule_prepare(size_t smem)
{
    cudaError_t e = raise_smem_limit(rule_kernel<kRuleM>, smem);
    if (e != cudaSuccess) return e;
    return raise_smem_limit(rule_kernel<kRuleU>, smem);
}

cudaError_t launch_rule(const RuleParams &p, int rule, int n_items, size_t smem, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    if (rule == kRuleM)
        rule_kernel<kRuleM><<<n_items, kRuleThreads, smem, st>>>(p);
    else
        rule_kernel<kRuleU><<<n_items, kRuleThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace mplpp
