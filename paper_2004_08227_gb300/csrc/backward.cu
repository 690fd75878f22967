// backward.cu -- gradient of the dual bound after T Handshake iterations with
// respect to the original unary and pairwise costs, by reverse-mode
// differentiation of the message-form iteration (handshake.cu).
//
// D is piecewise linear in the costs; inside one linear piece every minimum is
// attained at a fixed argument, so D is a sum of selected entries.  The
// iterations are replayed in FP64 (record.cu) from phi = 0, keeping a state
// checkpoint every k iterations; then, segment by segment from the last, the
// segment is recomputed while the argmins of the three minimizations of every
// update are recorded:
//   t1(s) = argmin_t [theta(s,t) + vh(t)],  s2(t) = argmin_s [theta(s,t) + alpha(s)],
//   t3(s) = argmin_t [theta(s,t) + beta(t)]          (lowest index on ties)
// and the updates are replayed in reverse schedule order.  With the adjoints
// Au, Phu (of agg_u and phi_{v->u} after the update) and Av, Phv:
//   cbar = Au + Phu;  uhbar = Au;  bbar = Av + Phv;  vhbar = -Phv
//   betabar(t) = sum_{s: t3(s)=t} cbar(s);  thetabar(s, t3(s)) += cbar(s)
//   vhbar += betabar;  bbar -= betabar;  vhbar += bbar
//   alphabar(s) = sum_{t: s2(t)=s} bbar(t); thetabar(s2(t), t) += bbar(t)
//   uhbar += alphabar / 2   (alpha = uh - a, a = (m1 + uh) / 2)
//   m1bar = -alphabar / 2;  thetabar(s, t1(s)) += m1bar(s);
//   vhbar(t) += sum_{s: t1(s)=t} m1bar(s)
// and the adjoints before the update are Au = uhbar, Phu = -uhbar,
// Av = vhbar, Phv = -vhbar.  The sums over argmin preimages are gathers in a
// fixed order, so the result is deterministic.  Edges of one matching touch
// disjoint nodes, so a matching's edges run in parallel as in the forward.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "backward.h"
#include "kernels.h"
#include "solver.h"

namespace mplpp {

namespace {

constexpr int kThreads = 256;

// Adjoint of D = sum_u min agg_u + sum_e min residual_e at the final state.
__global__ void bw_init_nodes_kernel(const NodeDesc *nodes, int n_nodes, const double *agg, const float *dD,
                                     double *adj_agg)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = warp; u < n_nodes; u += nw) {
        const NodeDesc nd = nodes[u];
        double m = INFINITY;
        int mi = INT_MAX;
        for (int s = lane; s < nd.L; s += 32) {
            const double v = agg[nd.aoff + s];
            if (v < m) {
                m = v;
                mi = s;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double om = __shfl_xor_sync(0xffffffffu, m, o);
            const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
            if (om < m || (om == m && oi < mi)) {
                m = om;
                mi = oi;
            }
        }
        if (lane == 0 && mi != INT_MAX) adj_agg[nd.aoff + mi] += static_cast<double>(dD[nd.model]);
    }
}

__global__ void __launch_bounds__(kThreads) bw_init_edges_kernel(const EdgeDesc *edges, int n_edges, const float *tab,
                                                                 const double *msg, const float *dD, double *adj_msg,
                                                                 double *gtab)
{
    __shared__ double rv[kThreads / 32];
    __shared__ long long ri[kThreads / 32];
    for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        double m = INFINITY;
        long long mi = LLONG_MAX;
        const long long n = static_cast<long long>(ed.Lu) * ed.Lv;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = static_cast<int>(i / ed.Lv);
            const int t = static_cast<int>(i - static_cast<long long>(s) * ed.Lv);
            const double r =
                (static_cast<double>(tab[ed.toff + static_cast<long long>(s) * ed.ld + t]) - msg[ed.mu + s]) -
                msg[ed.mv + t];
            if (r < m) {
                m = r;
                mi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double om = __shfl_xor_sync(0xffffffffu, m, o);
            const long long oi = __shfl_xor_sync(0xffffffffu, mi, o);
            if (om < m || (om == m && oi < mi)) {
                m = om;
                mi = oi;
            }
        }
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            rv[w] = m;
            ri[w] = mi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 1; j < kThreads / 32; ++j)
                if (rv[j] < rv[0] || (rv[j] == rv[0] && ri[j] < ri[0])) {
                    rv[0] = rv[j];
                    ri[0] = ri[j];
                }
            if (ri[0] != LLONG_MAX) {
                const int s = static_cast<int>(ri[0] / ed.Lv);
                const int t = static_cast<int>(ri[0] - static_cast<long long>(s) * ed.Lv);
                const double d = static_cast<double>(dD[ed.model]);
                gtab[ed.toff + static_cast<long long>(s) * ed.ld + t] += d;
                adj_msg[ed.mu + s] -= d;
                adj_msg[ed.mv + t] -= d;
            }
        }
        __syncthreads();
    }
}

// Sums of values over the preimages of an index map, deterministic: every
// element k < n holds key[k] (< m) and value val[k]; per warp, the lanes with
// equal keys (__match_any_sync) are summed in lane order by the lowest of them
// into that warp's partial part[warp][key]; afterwards (after a barrier) the
// caller adds the warps' partials in warp order.  part[w][*] must be zero for
// keys a warp does not hold; zero_part restores that after use.
__device__ __forceinline__ void warp_preimage_sums(int n, const int *key, const double *val, double *part, int m)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int base = 0; base < n; base += T) {  // the same trip count in every thread
        const int k = base + tid;
        const bool on = k < n;
        const int kk = on ? key[k] : -1 - lane;  // idle lanes never match an active one
        const unsigned grp = __match_any_sync(0xffffffffu, kk);
        if (on && (grp & ((1u << lane) - 1u)) == 0) {  // the group's lowest lane
            double acc = 0.0;
            const int b0 = k - lane;
            for (unsigned g = grp; g; g &= g - 1) acc += val[b0 + (__ffs(g) - 1)];
            part[((base / T) * (T >> 5) + warp) * m + kk] = acc;
        }
    }
}

// Reverse of one Handshake update per CTA (one matching per launch).
__global__ void __launch_bounds__(kThreads) bw_phase_kernel(BwParams p, int first)
{
    extern __shared__ __align__(16) double sh[];
    const int j = first + static_cast<int>(blockIdx.x);  // schedule position: descriptor and record offset at once
    const EdgeDesc ed = p.descs[j];
    const int Lu = ed.Lu, Lv = ed.Lv, T = blockDim.x, tid = threadIdx.x;
    const int lm = p.lmax;
    const int nw = ((lm + T - 1) / T) * (T >> 5);  // warp partial rows (a warp per 32 keys of a pass)
    double *cb = sh;         // cbar = m3bar            [Lu]
    double *uhb = cb + lm;   // uhbar                   [Lu]
    double *alb = uhb + lm;  // alphabar                [Lu]
    double *m1b = alb + lm;  // m1bar                   [Lu]
    double *bb = m1b + lm;   // bbar = m2bar            [Lv]
    double *vhb = bb + lm;   // vhbar                   [Lv]
    double *beb = vhb + lm;  // betabar                 [Lv]
    double *part = beb + lm;  // [nw][lm] warp partial sums
    int *t1 = reinterpret_cast<int *>(part + static_cast<size_t>(nw) * lm);
    int *s2 = t1 + lm;
    int *t3 = s2 + lm;
    const unsigned short *rec = reinterpret_cast<const unsigned short *>(p.rec + p.rec_off[j]);
    double *g = p.gtab + ed.toff;
    for (int i = tid; i < nw * lm; i += T) part[i] = 0.0;
    for (int s = tid; s < Lu; s += T) {
        const double Au = p.adj_agg[ed.au + s];
        const double Pu = p.adj_msg[ed.mu + s];
        cb[s] = Au + Pu;
        uhb[s] = Au;
        // recorded indices are < L for finite values; clamp so that no record
        // can address outside the table
        t1[s] = min(static_cast<int>(rec[s]), Lv - 1);
        t3[s] = min(static_cast<int>(rec[Lu + Lv + s]), Lv - 1);
    }
    for (int t = tid; t < Lv; t += T) {
        const double Av = p.adj_agg[ed.av + t];
        const double Pv = p.adj_msg[ed.mv + t];
        bb[t] = Av + Pv;
        vhb[t] = -Pv;
        s2[t] = min(static_cast<int>(rec[Lu + t]), Lu - 1);
    }
    __syncthreads();
    // pass 3 reversed: c(s) = theta(s, t3(s)) + beta(t3(s)) + uh(s)
    warp_preimage_sums(Lu, t3, cb, part, lm);
    for (int s = tid; s < Lu; s += T) g[static_cast<long long>(s) * ed.ld + t3[s]] += cb[s];
    __syncthreads();
    // beta = vh - b;  b = m2 + vh
    for (int t = tid; t < Lv; t += T) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) {
            acc += part[w * lm + t];
            part[w * lm + t] = 0.0;
        }
        const double v = vhb[t] + acc;
        const double b = bb[t] - acc;
        bb[t] = b;
        vhb[t] = v + b;
    }
    __syncthreads();
    // pass 2 reversed: m2(t) = theta(s2(t), t) + alpha(s2(t))
    for (int t = tid; t < Lv; t += T) g[static_cast<long long>(s2[t]) * ed.ld + t] += bb[t];
    warp_preimage_sums(Lv, s2, bb, part, lm);
    __syncthreads();
    // alpha = uh - a;  a = (m1 + uh) / 2
    for (int s = tid; s < Lu; s += T) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) {
            acc += part[w * lm + s];
            part[w * lm + s] = 0.0;
        }
        alb[s] = acc;
        const double ab = -acc;
        uhb[s] = (uhb[s] + acc) + 0.5 * ab;
        m1b[s] = 0.5 * ab;
    }
    __syncthreads();
    // pass 1 reversed: m1(s) = theta(s, t1(s)) + vh(t1(s))
    for (int s = tid; s < Lu; s += T) g[static_cast<long long>(s) * ed.ld + t1[s]] += m1b[s];
    warp_preimage_sums(Lu, t1, m1b, part, lm);
    __syncthreads();
    for (int t = tid; t < Lv; t += T) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += part[w * lm + t];
        vhb[t] += acc;
    }
    // uh = agg_u - phi_{v->u}, vh = agg_v - phi_{u->v} (values before the update)
    for (int s = tid; s < Lu; s += T) {
        p.adj_agg[ed.au + s] = uhb[s];
        p.adj_msg[ed.mu + s] = -uhb[s];
    }
    for (int t = tid; t < Lv; t += T) {
        p.adj_agg[ed.av + t] = vhb[t];
        p.adj_msg[ed.mv + t] = -vhb[t];
    }
}

__global__ void unpack_grad_kernel(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                                   const long long *pair_base, const long long *unary_base, const double *gtab,
                                   const double *adj_agg, float *grad_pair, float *grad_un)
{
    for (int e = blockIdx.x; e < n_edges; e += gridDim.x) {
        const EdgeDesc ed = edges[e];
        const long long dst = pair_base[ed.model] + ed.poff;
        const long long n = static_cast<long long>(ed.Lu) * ed.Lv;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = static_cast<int>(i / ed.Lv);
            const int t = static_cast<int>(i - static_cast<long long>(s) * ed.Lv);
            grad_pair[dst + i] = static_cast<float>(gtab[ed.toff + static_cast<long long>(s) * ed.ld + t]);
        }
    }
    for (int u = blockIdx.x; u < n_nodes; u += gridDim.x) {
        const NodeDesc nd = nodes[u];
        for (int s = threadIdx.x; s < nd.L; s += blockDim.x)
            grad_un[unary_base[nd.model] + nd.uoff + s] = static_cast<float>(adj_agg[nd.aoff + s]);
    }
}

}  // namespace

cudaError_t launch_bw_init(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes, const float *tab,
                           const double *agg, const double *msg, const float *dD, double *adj_agg, double *adj_msg,
                           double *gtab, cudaStream_t st)
{
    if (n_nodes > 0) {
        bw_init_nodes_kernel<<<std::max(1, std::min(65535, (n_nodes + 7) / 8)), kThreads, 0, st>>>(nodes, n_nodes, agg,
                                                                                                  dD, adj_agg);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_edges > 0) {
        bw_init_edges_kernel<<<std::min(n_edges, 1 << 20), kThreads, 0, st>>>(edges, n_edges, tab, msg, dD, adj_msg,
                                                                             gtab);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

size_t bw_phase_smem_bytes(int lmax)
{
    const size_t nw = static_cast<size_t>((lmax + kThreads - 1) / kThreads) * (kThreads / 32);
    return static_cast<size_t>(lmax) * ((7 + nw) * sizeof(double) + 3 * sizeof(int));
}

cudaError_t launch_bw_phase(const BwParams &p, int first, int n_items, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = bw_phase_smem_bytes(p.lmax);
    if (smem > 48 * 1024) {
        cudaError_t e = raise_smem_limit(bw_phase_kernel, smem);
        if (e != cudaSuccess) return e;
    }
    bw_phase_kernel<<<n_items, kThreads, smem, st>>>(p, first);
    return cudaGetLastError();
}

cudaError_t launch_unpack_grad(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                               const long long *pair_base, const long long *unary_base, const double *gtab,
                               const double *adj_agg, float *grad_pair, float *grad_un, cudaStream_t st)
{
    const int grid = std::max(1, std::min(std::max(n_edges, n_nodes), 1 << 20));
    unpack_grad_kernel<<<grid, kThreads, 0, st>>>(edges, n_edges, nodes, n_nodes, pair_base, unary_base, gtab, adj_agg,
                                                  grad_pair, grad_un);
    return cudaGetLastError();
}

}  // namespace mplpp

using namespace mplpp;

namespace {

mplpp_status bfail(mplpp_solver *s, mplpp_status st, const std::string &m)
{
    s->err = m;
    return st;
}

#define BCK(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return bfail(s, MPLPP_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr long long kRecordAllBytes = 1LL << 30;  // argmin records kept for a one-replay backward

template <typename T>
cudaError_t ensure(mplpp_solver *s, T **p, size_t count)
{
    if (*p) return cudaSuccess;
    return s->alloc(p, count);
}

// One FP64 iteration: every matching in schedule order (screened kernel when
// the largest table fits shared memory, tab_floats > 0; else all-FP64 scans).
cudaError_t rec64_iteration(mplpp_solver *s, unsigned char *rec, int lmax, long long tab_floats, cudaStream_t st)
{
    for (int ph = 0; ph < s->P; ++ph) {
        const int *items = s->d_phase_edges + s->phase_off[ph];
        const int n = s->phase_off[ph + 1] - s->phase_off[ph];
        const int f = s->phase_off[ph];
        cudaError_t e = tab_floats > 0 ? launch_rec_screen_phase(s->d_sched_desc + f, n, s->d_tab, s->d_agg64,
                                                                 s->d_msg64, rec, s->d_sched_rec_off + f, lmax,
                                                                 tab_floats, st)
                                       : launch_rec64_phase(s->d_edges, items, n, s->d_tab, s->d_agg64, s->d_msg64, rec,
                                                            s->d_rec_off, lmax, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" mplpp_status mplpp_backward(mplpp_solver *s, const float *dD, float *grad_unary, float *grad_pairwise)
{
    if (!s || !dD || !grad_unary || (s->sum_pair > 0 && !grad_pairwise)) return MPLPP_E_INVALID;
    s->err.clear();
    const int k = s->opt.record_every;
    if (k <= 0) return bfail(s, MPLPP_E_STATE, "backward needs options.record_every > 0");
    if (!s->history_valid)
        return bfail(s, MPLPP_E_STATE, "the state was loaded: the iterations since phi = 0 are unknown");
    const long long Ttot = s->iterations;
    const int nm = static_cast<int>(s->models.size());
    cudaStream_t st = s->stream;
    int lmax = 1;
    for (auto &nd : s->h_nodes) lmax = std::max(lmax, nd.L);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (rec64_smem_bytes(lmax) > static_cast<size_t>(optin) || bw_phase_smem_bytes(lmax) > static_cast<size_t>(optin))
        return bfail(s, MPLPP_E_UNSUPPORTED, "backward supports at most ~1400 labels per node");
    long long tab_floats = 0;  // the screened replay stages the largest table in shared memory
    for (auto &ed : s->h_edges) tab_floats = std::max(tab_floats, 1LL * ed.Lu * (ed.ld | 1));
    if ((s->opt.test_backward & 1) || rec_screen_smem_bytes(lmax, tab_floats) > static_cast<size_t>(optin))
        tab_floats = 0;

    // buffers
    if (!s->d_rec_off) {
        std::vector<long long> off(s->EE);
        long long acc = 0;
        for (int e = 0; e < s->EE; ++e) {
            off[e] = acc;
            acc += 2LL * (2LL * s->h_edges[e].Lu + s->h_edges[e].Lv);
            acc = (acc + 3) & ~3LL;
        }
        s->rec_stride = std::max(4LL, acc);
        // the same in schedule order, with the edges' descriptors: a block of
        // the replay or the reverse sweep reads both at once
        std::vector<EdgeDesc> sd(s->EE);
        std::vector<long long> so(s->EE);
        for (int j = 0; j < s->EE; ++j) {
            sd[j] = s->h_edges[s->phase_edges[j]];
            so[j] = off[s->phase_edges[j]];
        }
        BCK(s->alloc(&s->d_rec_off, std::max(1, s->EE)));
        BCK(s->alloc(&s->d_sched_desc, std::max(1, s->EE)));
        BCK(s->alloc(&s->d_sched_rec_off, std::max(1, s->EE)));
        BCK(cudaMemcpyAsync(s->d_rec_off, off.data(), sizeof(long long) * s->EE, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(s->d_sched_desc, sd.data(), sizeof(EdgeDesc) * s->EE, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(s->d_sched_rec_off, so.data(), sizeof(long long) * s->EE, cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));
    }
    if (!s->d_pbase) {
        std::vector<long long> pb(nm), ub(nm);
        long long a = 0, b = 0;
        for (int m = 0; m < nm; ++m) {
            pb[m] = a;
            ub[m] = b;
            a += s->models[m].pair_size;
            b += s->models[m].unary_size;
        }
        BCK(s->alloc(&s->d_pbase, nm));
        BCK(s->alloc(&s->d_ubase, nm));
        BCK(cudaMemcpyAsync(s->d_pbase, pb.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(s->d_ubase, ub.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));
    }
    BCK(ensure(s, &s->d_agg64, s->aggN));
    BCK(ensure(s, &s->d_msg64, s->msgN));
    BCK(ensure(s, &s->d_adj_agg, s->aggN));
    BCK(ensure(s, &s->d_adj_msg, s->msgN));
    BCK(ensure(s, &s->d_gtab, s->tabN));
    // When the argmin records of every iteration fit kRecordAllBytes, the one
    // replay records them all (no checkpoints, no second replay); otherwise a
    // state checkpoint every k iterations and each segment replayed again,
    // recording, before its reverse sweep.
    const bool record_all = Ttot > 0 && s->rec_stride * Ttot <= kRecordAllBytes && !(s->opt.test_backward & 2);
    const long long rec_slots = record_all ? Ttot : k;
    if (s->rec_slots < rec_slots) {
        BCK(s->release(s->d_rec));
        s->d_rec = nullptr;
        BCK(s->alloc(&s->d_rec, static_cast<size_t>(s->rec_stride) * rec_slots));
        s->rec_slots = rec_slots;
    }
    BCK(ensure(s, &s->d_dD, nm));
    const long long nseg = record_all ? 0 : (Ttot + k - 1) / k;
    while (static_cast<long long>(s->ckpt64.size()) < nseg) {
        double *c = nullptr;
        BCK(s->alloc(&c, static_cast<size_t>(s->aggN + s->msgN)));
        s->ckpt64.push_back(c);
    }

    // FP64 replay from phi = 0: recording every iteration, or a checkpoint every k
    BCK(launch_widen(s->d_un0, s->d_agg64, s->aggN, st));
    BCK(cudaMemsetAsync(s->d_msg64, 0, sizeof(double) * s->msgN, st));
    for (long long it = 0; it < Ttot; ++it) {
        if (!record_all && it % k == 0) {
            double *c = s->ckpt64[it / k];
            BCK(cudaMemcpyAsync(c, s->d_agg64, sizeof(double) * s->aggN, cudaMemcpyDeviceToDevice, st));
            BCK(cudaMemcpyAsync(c + s->aggN, s->d_msg64, sizeof(double) * s->msgN, cudaMemcpyDeviceToDevice, st));
        }
        BCK(rec64_iteration(s, record_all ? s->d_rec + it * s->rec_stride : nullptr, lmax, tab_floats, st));
    }
    BCK(cudaMemcpyAsync(s->d_dD, dD, sizeof(float) * nm, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(s->d_adj_agg, 0, sizeof(double) * s->aggN, st));
    BCK(cudaMemsetAsync(s->d_adj_msg, 0, sizeof(double) * s->msgN, st));
    BCK(cudaMemsetAsync(s->d_gtab, 0, sizeof(double) * s->tabN, st));
    BCK(launch_bw_init(s->d_edges, s->EE, s->d_nodes, s->N, s->d_tab, s->d_agg64, s->d_msg64, s->d_dD, s->d_adj_agg,
                       s->d_adj_msg, s->d_gtab, st));

    BwParams bp = {};
    bp.descs = s->d_sched_desc;
    bp.rec_off = s->d_sched_rec_off;
    bp.adj_agg = s->d_adj_agg;
    bp.adj_msg = s->d_adj_msg;
    bp.gtab = s->d_gtab;
    bp.lmax = lmax;
    for (long long it = record_all ? Ttot - 1 : -1; it >= 0; --it) {
        bp.rec = s->d_rec + it * s->rec_stride;
        for (int ph = s->P - 1; ph >= 0; --ph)
            BCK(launch_bw_phase(bp, s->phase_off[ph], s->phase_off[ph + 1] - s->phase_off[ph], st));
    }
    for (long long j = nseg - 1; j >= 0; --j) {
        const int len = static_cast<int>(std::min<long long>(k, Ttot - j * k));
        BCK(cudaMemcpyAsync(s->d_agg64, s->ckpt64[j], sizeof(double) * s->aggN, cudaMemcpyDeviceToDevice, st));
        BCK(cudaMemcpyAsync(s->d_msg64, s->ckpt64[j] + s->aggN, sizeof(double) * s->msgN, cudaMemcpyDeviceToDevice,
                            st));
        for (int i = 0; i < len; ++i)
            BCK(rec64_iteration(s, s->d_rec + static_cast<long long>(i) * s->rec_stride, lmax, tab_floats, st));
        for (int i = len - 1; i >= 0; --i) {
            bp.rec = s->d_rec + static_cast<long long>(i) * s->rec_stride;
            for (int ph = s->P - 1; ph >= 0; --ph)
                BCK(launch_bw_phase(bp, s->phase_off[ph], s->phase_off[ph + 1] - s->phase_off[ph], st));
        }
    }
    float *d_gu = nullptr, *d_gp = nullptr;
    float *gu = grad_unary, *gp = grad_pairwise;
    if (!s->opt.inputs_on_device) {
        BCK(cudaMalloc(&d_gu, sizeof(float) * std::max(1LL, s->sum_unary)));
        cudaError_t e = cudaMalloc(&d_gp, sizeof(float) * std::max(1LL, s->sum_pair));
        if (e != cudaSuccess) {
            cudaFree(d_gu);
            return bfail(s, MPLPP_E_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        gu = d_gu;
        gp = d_gp;
    }
    cudaError_t e = launch_unpack_grad(s->d_edges, s->EE, s->d_nodes, s->N, s->d_pbase, s->d_ubase, s->d_gtab,
                                       s->d_adj_agg, gp, gu, st);
    if (e == cudaSuccess && !s->opt.inputs_on_device) {
        e = cudaMemcpyAsync(grad_unary, d_gu, sizeof(float) * s->sum_unary, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && s->sum_pair)
            e = cudaMemcpyAsync(grad_pairwise, d_gp, sizeof(float) * s->sum_pair, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_gu) cudaFree(d_gu);
    if (d_gp) cudaFree(d_gp);
    if (e != cudaSuccess) return bfail(s, MPLPP_E_CUDA, std::string("backward: ") + cudaGetErrorString(e));
    return mplpp_sync(s);
}
