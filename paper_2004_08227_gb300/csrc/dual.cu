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

// emin[e] = min_{s,t} (theta_uv(s,t) - phi_{v->u}(s)) - phi_{u->v}(t), the
// FP64 value of that expression minimized over all (s,t), computed with FP64
// arithmetic only where it can decide the minimum (GB300's FP64 rate is far
// below its FP32 rate).  Per row s, an FP32 screen first:
//   e(t) = fl32(theta(s,t) - d(t)),  d(t) = fl32(phi_{u->v}(t) - phi_{u->v}(0)).
// With D = max_t |d(t)| and Th = max_t |theta(s,t)|, every e(t) is within
//   eps1 = 2^-22 (D + Th)
// of the exact theta(s,t) - phi_{u->v}(t) + phi_{u->v}(0)  (d(t): two
// roundings, <= 2^-23 |d|(1 + 2^-23); the FP32 difference: <= 2^-24 (Th + D)),
// and the FP64 evaluation of an entry is within
//   eps2 = 2^-50 (Th + |phi_{v->u}(s)| + |phi_{u->v}(0)| + 2 D)
// of its exact value.  An entry with e(t) > min_t e + 4 eps1 + 2 eps2 is then
// strictly above the row's minimizer in exact arithmetic by more than 2 eps2,
// so its FP64 value cannot be the row's (hence the table's) FP64 minimum.  The
// threshold is formed in FP32 with upward rounding (a superset of the
// candidates); each warp appends its rows' candidates (usually one or two per
// row) to a list in shared memory and evaluates them in FP64 32 at a time, one
// per lane, so FP64 instructions run with full warps; the table's minimum is
// the minimum over all candidates.  Messages are decoded to FP64 once per
// edge.  The result equals the FP64 minimum over every entry, bit for bit.
constexpr int kCandCap = 64;  // candidate list entries per warp

__global__ void __launch_bounds__(kThreads) bound_edges_kernel(const EdgeDesc *edges, int n_edges,
                                                               const float *tab, const ulonglong2 *msg, int lmax,
                                                               double *emin)
{
    extern __shared__ double dyn[];
    double *p1 = dyn;                                       // [lmax] phi_{v->u}(s)
    double *p2 = dyn + lmax;                                // [lmax] phi_{u->v}(t)
    float *a1 = reinterpret_cast<float *>(dyn + 2 * lmax);  // [lmax] |phi_{v->u}(s)| rounded up
    float *dsh = a1 + lmax;                                 // [lmax] d(t)
    __shared__ double red[32];
    __shared__ float redf[32];
    __shared__ int2 cands[kThreads / 32][kCandCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kThreads / 32;
    int2 *cl = cands[warp];
    for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        const double ref = se_d(msg[ed.mv]);
        const float aref = __double2float_ru(fabs(ref));
        float dmax = 0.f;
        for (int t = threadIdx.x; t < ed.Lv; t += kThreads) {
            const double v = se_d(msg[ed.mv + t]);
            const float d = static_cast<float>(v - ref);
            p2[t] = v;
            dsh[t] = d;
            dmax = fmaxf(dmax, fabsf(d));
        }
        for (int s = threadIdx.x; s < ed.Lu; s += kThreads) {
            const double v = se_d(msg[ed.mu + s]);
            p1[s] = v;
            a1[s] = __double2float_ru(fabs(v));
        }
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0) redf[warp] = dmax;
        __syncthreads();
        float D = 0.f;
        for (int w = 0; w < nw; ++w) D = fmaxf(D, redf[w]);
        const float *trow = tab + ed.toff;
        double m = INFINITY;  // this lane's minimum over the candidates it evaluated
        int ncl = 0;          // list length (the same in every lane)
        auto flush = [&]() {
            __syncwarp();
            for (int i = lane; i < ncl; i += 32) {
                const int2 c = cl[i];
                m = fmin(m, (static_cast<double>(trow[static_cast<long long>(c.x) * ed.ld + c.y]) - p1[c.x]) - p2[c.y]);
            }
            __syncwarp();
            ncl = 0;
        };
        for (int s = warp; s < ed.Lu; s += nw) {
            const float *row = trow + static_cast<long long>(s) * ed.ld;
            float me = INFINITY, th = 0.f;
            for (int t = lane; t < ed.Lv; t += 32) {
                const float x = row[t];
                me = fminf(me, x - dsh[t]);
                th = fmaxf(th, fabsf(x));
            }
            for (int o = 16; o > 0; o >>= 1) {
                me = fminf(me, __shfl_xor_sync(0xffffffffu, me, o));
                th = fmaxf(th, __shfl_xor_sync(0xffffffffu, th, o));
            }
            // me + 4 eps1 + 2 eps2, every operation rounded upwards
            const float eps1 = __fmul_ru(0x1p-22f, __fadd_ru(D, th));
            const float eps2 = __fmul_ru(0x1p-50f, __fadd_ru(__fadd_ru(th, a1[s]), __fadd_ru(aref, __fmul_ru(2.f, D))));
            const float thr = __fadd_ru(__fadd_ru(me, __fmul_ru(4.f, eps1)), __fadd_ru(__fmul_ru(2.f, eps2), 0x1p-126f));
            for (int t0 = 0; t0 < ed.Lv; t0 += 32) {  // warp-uniform trip count
                const int t = t0 + lane;
                const bool c = t < ed.Lv && row[t] - dsh[t] <= thr;
                const unsigned mask = __ballot_sync(0xffffffffu, c);
                if (mask) {
                    if (ncl + __popc(mask) > kCandCap) flush();
                    if (c) cl[ncl + __popc(mask & ((1u << lane) - 1u))] = make_int2(s, t);
                    ncl += __popc(mask);
                }
            }
        }
        flush();
        m = block_min<kThreads>(m, red);
        if (threadIdx.x == 0) emin[e] = m;
        __syncthreads();  // p1, p2, a1, dsh, redf and the lists are rewritten for the next edge
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
// GB300's FP64 rate is far below its FP32 rate, so every label's objective
// is first evaluated in double-float (FP32 operations), O(s), with
//   |O(s) - exact| and |FP64 value - exact| <= B(s) = (K + 8) 2^-43 S(s),
// S(s) = |agg_u(s)| + sum_k (|theta| + |phi_{u->v}| + |phi_{v->u}(s)|), K
// earlier neighbours (each double-float addition errs by at most
// 3 * 2^-48 (|a| + |b|), and a label's terms are summed by up to 16 threads
// whose partial sums are then added in a tree: at most K + 4 additions per
// label plus two per term; B carries a factor of more than 10 of margin).  With O(s)
// bracketed in FP32 (upward / downward rounding) as [lo(s), hi(s)], a label
// with lo(s) > H = min_s hi(s) can neither attain the FP64 minimum nor tie
// with it.  A single remaining candidate is therefore the FP64 argmin without
// any FP64 work; several (ties, near-ties) are summed in FP64 in neighbour
// order and compared, so the decision always equals the all-FP64 one.
// Latency: the in-edges of node u + 1 whose neighbour is already decided are
// staged (table row offset, messages) and their table rows prefetched into
// L2 by the threads without labels while node u is decided.
constexpr int kRoundThreads = 512;

// Block b decides the nodes of model b in order, or (level_nodes given) the
// single node level_nodes[b]: a node whose earlier neighbours were all decided
// by earlier launches, so the nodes of one level are decided in parallel.
__global__ void __launch_bounds__(kRoundThreads) round_kernel(const NodeDesc *nodes, const int *in_off,
                                                              const InRec *in_rec, const int *model_node_off,
                                                              const int *level_nodes, const float *tab,
                                                              const ulonglong2 *agg, const ulonglong2 *msg,
                                                              int *labels, int *err)
{
    constexpr int T = kRoundThreads;
    __shared__ double rv[T / 32];
    __shared__ int ri[T / 32];
    __shared__ float rh[T / 32];
    // staged earlier neighbours (up to T per chunk), two sets: node u's and,
    // prepared meanwhile, node u + 1's
    __shared__ long long k_row[2][T], k_mv[2][T];
    __shared__ float2 k_phf[2][T];
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    const int w = tid >> 5, l = tid & 31;
    constexpr int kBatch = 16;  // rows of different tables miss in L2: loads in flight
    const int u0 = level_nodes ? level_nodes[m] : model_node_off[m];
    const int u1 = level_nodes ? u0 + 1 : model_node_off[m + 1];
    auto stage_one = [&](int set, int slot, const InRec &r, int xv) {
        k_row[set][slot] = r.toff + static_cast<long long>(xv) * r.ld;
        k_mv[set][slot] = r.mv;
        const double ph = se_d(msg[r.mu + xv]);
        const float hi = static_cast<float>(ph);
        k_phf[set][slot] = make_float2(hi, static_cast<float>(ph - static_cast<double>(hi)));
    };
    bool pre = false;  // node u's set was staged (except a neighbour u - 1) during node u - 1
    for (int u = u0; u < u1; ++u) {
        const int set = (u - u0) & 1;
        const NodeDesc nd = nodes[u];
        const int L = nd.L;
        const int k0 = in_off[u], k1 = in_off[u + 1], K = k1 - k0;
        const bool chunked = K > T;
        // threads per label: the largest power of two (<= 16) leaving half the
        // block free to prepare the next node; labels beyond T / P loop (P = 1)
        int P = 1;
        while (P < 16 && 2 * P * L <= T / 2) P *= 2;
        const int s_of = tid / P, part = tid % P;
        const int nlab = T / P;  // labels per sweep
        // node u's staged neighbours: complete the set (the neighbour u - 1 was
        // still undecided) or stage it now
        if (!chunked) {
            if (pre) {
                if (K > 0 && tid == K - 1) {
                    const InRec r = in_rec[k0 + tid];
                    if (r.gu == u - 1) stage_one(set, tid, r, labels[r.gu]);
                }
            } else if (tid < K) {
                const InRec r = in_rec[k0 + tid];
                stage_one(set, tid, r, labels[r.gu]);
            }
            __syncthreads();
        }
        // the next node's neighbours decided by now, by threads without labels
        const int busy = ((L < nlab ? L : nlab) * P + 31) & ~31;
        const bool prep = u + 1 < u1 && in_off[u + 2] - in_off[u + 1] <= T && T - busy >= 32;
        if (prep && tid >= busy) {
            const int Ln = nodes[u + 1].L;
            for (int k = in_off[u + 1] + tid - busy; k < in_off[u + 2]; k += T - busy) {
                const InRec r = in_rec[k];
                if (r.gu < u) {
                    const int xv = labels[r.gu];
                    stage_one(set ^ 1, k - in_off[u + 1], r, xv);
                    const float *pr = tab + r.toff + static_cast<long long>(xv) * r.ld;
                    for (int q = 0; q < Ln; q += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + q));
                }
            }
        }
        // double-float screen; thread (s, part) sums neighbours k = part, part + P, ...
        float hsel = INFINITY;
        float lo_own = INFINITY;
        float2 o = make_float2(0.f, 0.f);
        float sa = 0.f;
        const int s = s_of;
        const bool mine = s < L && s < nlab;
        if (mine && part == 0) {
            o = se_df(agg[nd.aoff + s]);
            sa = fabsf(o.x);
        }
        for (int c0 = k0; c0 < k1; c0 += T) {
            const int nc = min(T, k1 - c0);
            if (chunked) {  // long neighbour lists: staged chunk by chunk
                __syncthreads();
                if (tid < nc) {
                    const InRec r = in_rec[c0 + tid];
                    stage_one(set, tid, r, labels[r.gu]);
                }
                __syncthreads();
            }
            if (mine)
                for (int kb = part; kb < nc; kb += kBatch * P) {
                    float tv[kBatch];
                    ulonglong2 mv[kBatch];
#pragma unroll
                    for (int q = 0; q < kBatch; ++q) {
                        const int k = kb + q * P;
                        if (k < nc) {
                            tv[q] = tab[k_row[set][k] + s];
                            mv[q] = msg[k_mv[set][k] + s];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kBatch; ++q) {
                        const int k = kb + q * P;
                        if (k < nc) {
                            const float2 f1 = k_phf[set][k], f2 = se_df(mv[q]);
                            o = df_add(o, df_sub(df_sub(make_float2(tv[q], 0.f), f1), f2));
                            sa += fabsf(tv[q]) + fabsf(f1.x) + fabsf(f2.x);
                        }
                    }
                }
        }
        // the P partial sums of a label (consecutive lanes), added in a tree
        for (int q = 1; q < P; q <<= 1) {
            const float ox = __shfl_xor_sync(0xffffffffu, o.x, q), oy = __shfl_xor_sync(0xffffffffu, o.y, q);
            o = df_add(o, make_float2(ox, oy));
            sa += __shfl_xor_sync(0xffffffffu, sa, q);
        }
        if (mine) {
            const float cK = static_cast<float>(K + 8);
            const float b = __fadd_ru(__fmul_ru(cK, __fadd_ru(__fmul_ru(0x1.1p-43f, sa), 0x1p-120f)), fabsf(o.y));
            lo_own = __fsub_rd(o.x, b);
            hsel = __fadd_ru(o.x, b);
        }
        for (int q = 16; q > 0; q >>= 1) hsel = fminf(hsel, __shfl_xor_sync(0xffffffffu, hsel, q));
        if (l == 0) rh[w] = hsel;
        __syncthreads();
        float H = rh[0];
        for (int q = 1; q < T / 32; ++q) H = fminf(H, rh[q]);
        bool cand = mine && part == 0 && lo_own <= H;
        // labels beyond one sweep (L > T, P = 1) are never screened: decided the
        // exact way below
        const bool extra = L > nlab;
        const int ncand = __syncthreads_count(cand);
        if (ncand == 1 && !extra) {
            // the only label that can attain the FP64 minimum
            if (cand) labels[u] = s;
            __syncthreads();
        } else {
            // several candidates (ties or near-ties), none (NaN objectives), or
            // labels beyond one sweep: FP64 sums in neighbour order
            double best = INFINITY;
            int bi = INT_MAX;
            if (cand) {
                double a = se_d(agg[nd.aoff + s]);
                for (int k = k0; k < k1; ++k) {
                    const InRec r = in_rec[k];
                    const int xv = labels[r.gu];
                    a = a + ((static_cast<double>(tab[r.toff + static_cast<long long>(xv) * r.ld + s]) -
                              se_d(msg[r.mu + xv])) -
                             se_d(msg[r.mv + s]));
                }
                best = a;
                bi = s;
            }
            if (extra && part == 0)
                for (int s2 = nlab + s_of; s2 < L; s2 += nlab) {
                    double a = se_d(agg[nd.aoff + s2]);
                    for (int k = k0; k < k1; ++k) {
                        const InRec r = in_rec[k];
                        const int xv = labels[r.gu];
                        a = a + ((static_cast<double>(tab[r.toff + static_cast<long long>(xv) * r.ld + s2]) -
                                  se_d(msg[r.mu + xv])) -
                                 se_d(msg[r.mv + s2]));
                    }
                    if (a < best || (a == best && s2 < bi)) {
                        best = a;
                        bi = s2;
                    }
                }
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o2);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o2);
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
            if (tid == 0) {
                double bb = INFINITY;
                int i = INT_MAX;
                for (int q = 0; q < T / 32; ++q)
                    if (ri[q] != INT_MAX && (rv[q] < bb || (rv[q] == bb && ri[q] < i))) {
                        bb = rv[q];
                        i = ri[q];
                    }
                if (i == INT_MAX) {  // no candidate: every objective value was NaN
                    i = 0;
                    atomicCAS(err, 0, ERR_NONFINITE);
                }
                labels[u] = i;
            }
            __syncthreads();
        }
        pre = prep;
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
                         const int *model_edge_off, int n_models, int exact, int lmax, double *out, cudaStream_t st)
{
    if (exact && n_edges > 0) {
        const int lm = lmax > 0 ? lmax : 1;
        const size_t smem = (2 * sizeof(double) + 2 * sizeof(float)) * static_cast<size_t>(lm);
        if (smem > 48 * 1024) {
            cudaError_t e = raise_smem_limit(bound_edges_kernel, smem);
            if (e != cudaSuccess) return e;
        }
        bound_edges_kernel<<<grid_for(n_edges, 1), kThreads, smem, st>>>(edges, n_edges, tab, msg, lm, emin);
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

cudaError_t launch_round(const EdgeDesc *edges, const NodeDesc *nodes, const int *in_off, const InRec *in_rec,
                         const int *model_node_off, const int *model_edge_off, int n_models, const float *tab,
                         const ulonglong2 *agg, const ulonglong2 *msg, const float *un0, int *labels, double *energy, int *err,
                         const int *level_nodes, const int *level_off, int n_levels, cudaStream_t st)
{
    if (n_levels > 0) {  // one launch per level, one block per node of the level
        for (int lv = 0; lv < n_levels; ++lv) {
            const int nb = level_off[lv + 1] - level_off[lv];
            round_kernel<<<nb, kRoundThreads, 0, st>>>(nodes, in_off, in_rec, model_node_off,
                                                       level_nodes + level_off[lv], tab, agg, msg, labels, err);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    } else {
        round_kernel<<<n_models, kRoundThreads, 0, st>>>(nodes, in_off, in_rec, model_node_off, nullptr, tab, agg, msg,
                                                         labels, err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    energy_kernel<<<n_models, kThreads, 0, st>>>(edges, nodes, model_node_off, model_edge_off, tab, un0, labels,
                                                energy);
    return cudaGetLastError();
}

}  // namespace mplpp
