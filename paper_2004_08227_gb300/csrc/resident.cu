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
// updates.
//
// One group of LM lanes (LM = 8, 16 or 32: the label bound rounded up) updates
// one edge: lane s of the group holds row s of the table and lane t column t
// (in registers), so every minimization is a sequential loop in one lane,
// with no shuffles, and a warp updates 32 / LM edges at once.  The tables are
// read from memory (they are read-only); for LM <= 16 a group loads the table
// of the next edge it will update while it updates the current one, so the
// load latency is hidden behind an update.
#include <cfloat>
#include <cstdint>

#include "kernels.h"

namespace mplpp {

namespace {

// Per-group vectors of the edge being updated (7 LM words per group, so a
// warp's groups fill kResWarpBytes).
struct ResVec {
    float2 *uh, *vh;           // [LM] double-float unaries without this edge's messages
    float *w1, *alpha, *beta;  // [LM] FP32 shifted operands of passes 1, 2 and 3
};

template <int LM>
__device__ __forceinline__ ResVec res_vec(char *base, int slot)
{
    char *b = base + static_cast<size_t>(slot) * (28 * LM);
    ResVec r;
    r.uh = reinterpret_cast<float2 *>(b);
    r.vh = r.uh + LM;
    r.w1 = reinterpret_cast<float *>(r.vh + LM);
    r.alpha = r.w1 + LM;
    r.beta = r.alpha + LM;
    return r;
}

// Fields of a scheduled edge (ResParams::sched_desc).
struct ResEdge {
    int toff, au, av, mu, mv, Lu, Lv, ld;
};

__device__ __forceinline__ ResEdge res_edge(int4 d)
{
    return ResEdge{d.x,      d.y & 0xffff, (d.y >> 16) & 0xffff, d.z & 0xffff, (d.z >> 16) & 0xffff,
                   d.w & 0xff, (d.w >> 8) & 0xff, (d.w >> 16) & 0xff};
}

// Row l and column l of edge ed's table (FP32, +inf beyond the labels; tab:
// the model's first table).  The row is read in 16-byte chunks up to the
// padded stride ld, whose padding columns hold +inf.
template <int LM>
__device__ __forceinline__ void res_load(const ResEdge &ed, const float *tab, int l, float (&row)[LM],
                                         float (&col)[LM])
{
    const float *th = tab + ed.toff;
    const float4 *r4 = reinterpret_cast<const float4 *>(th + l * ed.ld);
    const float4 inf4 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
#pragma unroll
    for (int j = 0; j < LM / 4; ++j) {
        const float4 v = (l < ed.Lu && 4 * j < ed.ld) ? __ldg(r4 + j) : inf4;
        row[4 * j] = v.x;
        row[4 * j + 1] = v.y;
        row[4 * j + 2] = v.z;
        row[4 * j + 3] = v.w;
    }
#pragma unroll
    for (int s = 0; s < LM; ++s) col[s] = (l < ed.Lv && s < ed.Lu) ? __ldg(th + s * ed.ld + l) : INFINITY;
}

// min_t [x(t) + y(t)] over t < n in order, y read from shared memory (16-byte
// aligned).  LM <= 16: four at a time over all LM entries -- entries of x
// beyond the labels are +inf, so they never win (fminf ignores the NaN that
// inf + -inf would give); LM = 32: one at a time up to n (its registers are
// taken by the row and the column).
template <int LM>
__device__ __forceinline__ float res_min_add(const float (&x)[LM], const float *y, int n)
{
    float m = INFINITY;
    if constexpr (LM <= 16) {
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
#pragma unroll
        for (int j = 0; j < LM / 4; ++j) {
            const float4 v = y4[j];
            m = fminf(m, x[4 * j] + v.x);
            m = fminf(m, x[4 * j + 1] + v.y);
            m = fminf(m, x[4 * j + 2] + v.z);
            m = fminf(m, x[4 * j + 3] + v.w);
        }
    } else {
#pragma unroll
        for (int t = 0; t < LM; ++t)
            if (t < n) m = fminf(m, x[t] + y[t]);
    }
    return m;
}

// One Handshake update of edge ed (L_u, L_v <= LM) by a group of LM lanes (l:
// the lane's index in the group) on the model's shared-memory state: agg and
// msg hold the model's entries (offsets relative to the model's first node
// and first edge).  Every lane of the warp calls it (act false: a group
// without an edge this round), for the warp-wide synchronizations.
template <int LM>
__device__ __forceinline__ void res_update(bool act, const ResEdge &ed, const float (&row)[LM],
                                           const float (&col)[LM], float2 *agg, float2 *msg, const ResVec &w, int l)
{
    const int Lu = act ? ed.Lu : 0, Lv = act ? ed.Lv : 0;
    float2 *au = agg + (act ? ed.au : 0), *av = agg + (act ? ed.av : 0);
    float2 *mu = msg + (act ? ed.mu : 0), *mv = msg + (act ? ed.mv : 0);
    if (l < Lu) w.uh[l] = df_sub(au[l], mu[l]);
    if (l < Lv) w.vh[l] = df_sub(av[l], mv[l]);
    __syncwarp();
    const float2 vref = w.vh[0];
    if (l < Lv) w.w1[l] = df_to_f(df_sub(w.vh[l], vref));
    __syncwarp();
    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + w1(t)] + vh(0) + uh(s));  alpha = uh - a
    if (l < Lu) {
        const float m = res_min_add<LM>(row, w.w1, Lv);
        // alpha = uh - a = 1/2 (uh - vh(0) - m), its value in exact arithmetic
        w.alpha[l] = df_to_f(df_half(df_add_f(df_sub(w.uh[l], vref), -m)));
    }
    __syncwarp();
    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t),  beta = vh - b
    if (l < Lv) {
        const float m = res_min_add<LM>(col, w.alpha, Lu);
        const float2 vh = w.vh[l];
        const float2 b = df_add_f(vh, m);
        w.beta[l] = -m;  // vh - b in exact arithmetic
        av[l] = b;
        mv[l] = df_sub(b, vh);
    }
    __syncwarp();
    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s)
    if (l < Lu) {
        const float m = res_min_add<LM>(row, w.beta, Lv);
        const float2 u = w.uh[l];
        const float2 c = df_add_f(u, m);
        au[l] = c;
        mu[l] = df_sub(c, u);
    }
    __syncwarp();  // the group's vectors are rewritten by its next update
}

// The walk of one group through a model's schedule: matching k, round r (the
// group's edge of round r is the model's scheduled edge off[k] + r * slots +
// slot, if below off[k + 1]), iteration it.  Every group of the CTA takes the
// same steps.
struct ResPos {
    int it, k, r;
};

__device__ __forceinline__ bool res_next(ResPos &q, const int *off, int P, int slots, int iterations)
{
    if ((q.r + 1) * slots < off[q.k + 1] - off[q.k]) {
        ++q.r;
        return true;
    }
    q.r = 0;
    if (++q.k < P) return true;
    q.k = 0;
    return ++q.it < iterations;
}

template <int LM>
__global__ void __launch_bounds__(512) hs_resident_kernel(ResParams p)
{
    constexpr int G = LM, EPW = 32 / LM;  // lanes per edge, edges per warp
    constexpr bool kPrefetch = LM <= 16;  // registers for a second row and column
    extern __shared__ __align__(16) char smem_raw[];
    const int m = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int l = lane % G, slot = warp * EPW + lane / G, slots = W * EPW;
    const ResModel md = p.models[m];
    // shared memory: the state, the groups' vectors, the matching offsets
    float2 *agg = reinterpret_cast<float2 *>(smem_raw);
    float2 *msg = agg + md.agg_n;
    // the groups' vectors start on a 16-byte boundary (they are read four
    // floats at a time; every vector is a multiple of 16 bytes long)
    char *vec = smem_raw + ((static_cast<size_t>(md.agg_n + md.msg_n) * sizeof(float2) + 15) & ~size_t{15});
    const ResVec w = res_vec<LM>(vec, slot);
    int *off = reinterpret_cast<int *>(vec + static_cast<size_t>(W) * kResWarpBytes);  // [P + 1] from 0
    const int *goff = p.sched_off + md.sched;
    const int e0 = goff[0];
    const int4 *desc = p.sched_desc + e0;  // the model's scheduled edges
    const float *mtab = p.tab + md.tab_base;
    for (int i = tid; i <= md.P; i += blockDim.x) off[i] = goff[i] - e0;
    for (long long i = tid; i < md.agg_n; i += blockDim.x) agg[i] = se_df(p.agg[md.agg_base + i]);
    for (long long i = tid; i < md.msg_n; i += blockDim.x) msg[i] = se_df(p.msg[md.msg_base + i]);
    __syncthreads();
    auto edge_at = [&](const ResPos &q, bool more, ResEdge &ed) {
        const int j = off[q.k] + q.r * slots + slot;
        const bool a = more && j < off[q.k + 1];
        if (a) ed = res_edge(__ldg(desc + j));
        return a;
    };
    if (p.iterations > 0 && md.P > 0) {
        // three steps in flight: the edge being updated (its table in row,
        // col), the next one (its table loading), the one after (its
        // descriptor loading)
        ResPos q = {0, 0, 0};
        ResEdge ed{}, ed1{};
        bool act = edge_at(q, true, ed);
        float row[LM], col[LM];
        if (act) res_load<LM>(ed, mtab, l, row, col);
        ResPos q1 = q;
        bool more1 = res_next(q1, off, md.P, slots, p.iterations);
        bool act1 = edge_at(q1, more1, ed1);
        for (;;) {
            float rown[LM], coln[LM];
            if (kPrefetch && act1) res_load<LM>(ed1, mtab, l, rown, coln);
            ResPos q2 = q1;
            const bool more2 = more1 && res_next(q2, off, md.P, slots, p.iterations);
            ResEdge ed2{};
            const bool act2 = edge_at(q2, more2, ed2);
            res_update<LM>(act, ed, row, col, agg, msg, w, l);
            if (!more1) break;
            if (q1.k != q.k || q1.it != q.it) __syncthreads();  // the barrier between matchings
            q = q1;
            act = act1;
            ed = ed1;
            if (kPrefetch) {
#pragma unroll
                for (int t = 0; t < LM; ++t) {
                    row[t] = rown[t];
                    col[t] = coln[t];
                }
            } else if (act) {
                res_load<LM>(ed, mtab, l, row, col);
            }
            q1 = q2;
            more1 = more2;
            act1 = act2;
            ed1 = ed2;
        }
    }
    __syncthreads();
    for (long long i = tid; i < md.agg_n; i += blockDim.x) p.agg[md.agg_base + i] = se_make(agg[i], 0u);
    for (long long i = tid; i < md.msg_n; i += blockDim.x) p.msg[md.msg_base + i] = se_make(msg[i], 0u);
}

}  // namespace

cudaError_t res_prepare(size_t smem)
{
    cudaError_t e;
    if ((e = raise_smem_limit(hs_resident_kernel<8>, smem)) != cudaSuccess)
        return e;
    if ((e = raise_smem_limit(hs_resident_kernel<16>, smem)) != cudaSuccess)
        return e;
    return raise_smem_limit(hs_resident_kernel<32>, smem);
}

// lmax: the largest label count of the solver (<= kResMaxL): lanes per edge
// res_lanes(lmax) = 8, 16 or 32.
cudaError_t launch_resident(const ResParams &p, int n_models, int threads, size_t smem, int lmax, cudaStream_t st)
{
    if (n_models <= 0) return cudaSuccess;
    switch (res_lanes(lmax)) {
    case 8: hs_resident_kernel<8><<<n_models, threads, smem, st>>>(p); break;
    case 16: hs_resident_kernel<16><<<n_models, threads, smem, st>>>(p); break;
    default: hs_resident_kernel<32><<<n_models, threads, smem, st>>>(p); break;
    }
    return cudaGetLastError();
}

}  // namespace mplpp
