// api.cu -- the C ABI (include/mplpp.h): solver creation, device layout,
// mapping choice, the iteration drivers, bound, rounding and state I/O.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mplpp.h"
#include "backward.h"
#include "host.h"
#include "kernels.h"
#include "solver.h"

using namespace mplpp;

namespace {

thread_local std::string g_create_error;

long long round4(long long x) { return (x + 3) & ~3LL; }

mplpp_status fail(mplpp_solver *s, mplpp_status st, const std::string &msg)
{
    if (s) s->err = msg;
    else g_create_error = msg;
    return st;
}

mplpp_status cuda_fail(mplpp_solver *s, cudaError_t e, const char *what)
{
    return fail(s, MPLPP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(s, call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

uint64_t fnv(uint64_t h, const void *data, size_t n)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

}  // namespace

mplpp_solver::~mplpp_solver()
{
    if (stream_ok) cudaStreamSynchronize(stream);
    for (void *p : allocations) cudaFree(p);
    if (g_looped) cudaGraphExecDestroy(g_looped);
    if (g_persist) cudaGraphExecDestroy(g_persist);
    if (cap_stream) cudaStreamDestroy(cap_stream);
}

extern "C" void mplpp_options_default(mplpp_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->mode = MPLPP_MODE_AUTO;
    opt->use_graph = 1;
    opt->inputs_on_device = 0;
    opt->record_every = 0;
    opt->cluster = 0;
    opt->threads = 0;
    opt->spin_limit = 1LL << 22;
}

extern "C" const char *mplpp_last_error(const mplpp_solver *s)
{
    return s ? s->err.c_str() : g_create_error.c_str();
}

// Mapping for one candidate cluster size C: per-CTA tile and vector sizes.
// The smallest block (a multiple of 32 threads, 64..512) whose warps hold all
// of a CTA's rows in the register-resident passes for wide rows, or 0.
static int rr_fit_threads(int rows, int Q, int tile_floats)
{
    for (int T = 64; T <= 512; T += 32)
        if (hs_rr_fits(rows, Q, T, tile_floats)) return T;
    return 0;
}

static void mapping_for(mplpp_solver *s, int C, int threads = 0)
{
    long long tile = 0, rows = 0;
    int ldmax = 4, lmax = 1;
    for (auto &ed : s->h_edges) {
        const long long R = (ed.Lu + C - 1) / C;
        tile = std::max(tile, R * ed.ld);
        rows = std::max(rows, R);
        ldmax = std::max(ldmax, ed.ld);
        lmax = std::max(lmax, std::max(ed.Lu, ed.ld));
    }
    s->lmax = lmax;
    const int tile_floats = static_cast<int>(round4(std::max(4LL, tile)));
    int T = threads > 0 ? threads : s->opt.threads;
    if (T <= 0) {
        T = (4 * tile >= 48 * 1024) ? 512 : (4 * tile <= 4096 ? 128 : 256);
        // register-resident passes for wide rows: just enough warps for the rows
        const int fit = rr_fit_threads(static_cast<int>(rows), ldmax >> 2, tile_floats);
        if (fit) T = fit;
    }
    s->C = C;
    s->T = T;
    s->tile_floats = tile_floats;
    s->rmax = static_cast<int>(round4(std::max(4LL, rows)));
    s->ldmax = ldmax;
    s->rr = hs_rr_fits(static_cast<int>(rows), ldmax >> 2, T, s->tile_floats);
    // a spare warp beyond those holding the rows becomes node u's poller
    s->pw = s->rr && hs_pw_fits(static_cast<int>(rows), ldmax >> 2, T, s->tile_floats);
    s->smem_looped = hs_smem_bytes(1, s->tile_floats, s->rmax, s->ldmax, s->T, C);
    s->smem_persist = hs_smem_bytes(2, s->tile_floats, s->rmax, s->ldmax, s->T, C);
}

// Chooses CTAs per edge (C).  A matching's edges should run in one round of
// co-resident clusters (the persistent driver's critical path is one edge
// update per matching and round), and within that the CTA slices should be
// small (less work per update).  Cost model per matching:
//   rounds(C) * (3 us of dependency latency + slice bytes / 40 GB/s per SM).
// Candidates whose double-buffered slice does not fit shared memory can only
// run looped.
static void choose_mapping(mplpp_solver *s, int sms, int optin)
{
    int max_phase = 1;
    for (size_t p = 0; p + 1 < s->phase_off.size(); ++p)
        max_phase = std::max(max_phase, s->phase_off[p + 1] - s->phase_off[p]);
    s->max_phase = max_phase;
    if (s->opt.cluster > 0) {
        mapping_for(s, s->opt.cluster);
        return;
    }
    double best = 1e300;
    int bestC = 0;
    for (int C = 1; C <= 8; ++C) {
        mapping_for(s, C);
        if (s->smem_persist > static_cast<size_t>(optin)) continue;
        if (C > 1 && static_cast<long long>(C) * max_phase > 2LL * sms) break;
        const int avail = std::min(hs_max_active_clusters(C, s->T, s->smem_persist, s->rr), max_phase);
        if (avail < 1) continue;
        const int rounds = (max_phase + avail - 1) / avail;
        const double cost = rounds * (3e-6 + 4.0 * s->tile_floats / 40e9);
        if (cost < best * 0.999) {
            best = cost;
            bestC = C;
        }
    }
    if (bestC == 0) {  // nothing fits twice: the smallest slice, looped only
        bestC = 8;
        for (int C = 1; C <= 8; ++C) {
            mapping_for(s, C);
            if (s->smem_looped <= static_cast<size_t>(optin)) {
                bestC = C;
                break;
            }
        }
    }
    mapping_for(s, bestC);
    (void)sms;
}

// Persistent driver: distribute each matching's edges over the clusters
// (largest table first onto the least loaded cluster); each cluster's list
// stays in schedule order, so every wait is on an earlier matching.
static void build_work(mplpp_solver *s, int clusters)
{
    const int N = s->N;
    std::vector<int> pos(N, 0), deg(N, 0);
    for (int e : s->phase_edges) {
        deg[s->h_edges[e].gu]++;
        deg[s->h_edges[e].gv]++;
    }
    std::vector<std::vector<WorkItem>> lists(clusters);
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < clusters; ++c) heap.push({0, c});
    for (size_t p = 0; p + 1 < s->phase_off.size(); ++p) {
        std::vector<int> es(s->phase_edges.begin() + s->phase_off[p], s->phase_edges.begin() + s->phase_off[p + 1]);
        std::stable_sort(es.begin(), es.end(), [&](int a, int b) {
            return 1LL * s->h_edges[a].Lu * s->h_edges[a].Lv > 1LL * s->h_edges[b].Lu * s->h_edges[b].Lv;
        });
        for (int e : es) {
            Load l = heap.top();
            heap.pop();
            const EdgeDesc &ed = s->h_edges[e];
            WorkItem w = {};
            w.ed = ed;
            w.edge = e;
            w.pos_u = pos[ed.gu]++;
            w.pos_v = pos[ed.gv]++;
            w.deg_u = deg[ed.gu];
            w.deg_v = deg[ed.gv];
            w.rows = (ed.Lu + s->C - 1) / s->C;
            lists[l.second].push_back(w);
            heap.push({l.first + 4LL * ed.Lu * ed.ld + 16LL * (ed.Lu + ed.Lv), l.second});
        }
    }
    s->work_off.assign(1, 0);
    s->work.clear();
    for (auto &l : lists) {
        s->work.insert(s->work.end(), l.begin(), l.end());
        s->work_off.push_back(static_cast<int>(s->work.size()));
    }
    s->max_deg = 0;
    for (int d : deg) s->max_deg = std::max(s->max_deg, d);
}

// Queue driver: one list of every update of an iteration.  A model's items
// keep its schedule order; the models are interleaved by their progress
// through an iteration (item of matching p of a model with P matchings at
// position (p + 1/2) / P), so consecutive matchings of one model lie far
// apart in the queue and a CTA rarely waits for an input.  Every item's
// inputs come from items earlier in the list (or in an earlier iteration).
static void build_queue(mplpp_solver *s)
{
    const int N = s->N;
    std::vector<int> pos(N, 0), deg(N, 0);
    for (int e : s->phase_edges) {
        deg[s->h_edges[e].gu]++;
        deg[s->h_edges[e].gv]++;
    }
    struct Q {
        double key;
        int seq;
        WorkItem w;
    };
    std::vector<Q> q;
    q.reserve(s->phase_edges.size());
    for (size_t p = 0; p + 1 < s->phase_off.size(); ++p)
        for (int i = s->phase_off[p]; i < s->phase_off[p + 1]; ++i) {
            const int e = s->phase_edges[i];
            const EdgeDesc &ed = s->h_edges[e];
            const int Pm = static_cast<int>(s->models[ed.model].off.size()) - 1;
            WorkItem w = {};
            w.ed = ed;
            w.edge = e;
            w.pos_u = pos[ed.gu]++;
            w.pos_v = pos[ed.gv]++;
            w.deg_u = deg[ed.gu];
            w.deg_v = deg[ed.gv];
            w.rows = ed.Lu;
            q.push_back({(static_cast<double>(p) + 0.5) / std::max(1, Pm), static_cast<int>(q.size()), w});
        }
    std::stable_sort(q.begin(), q.end(), [](const Q &a, const Q &b) { return a.key < b.key; });
    s->work.clear();
    for (auto &x : q) s->work.push_back(x.w);
    s->work_off.assign({0, static_cast<int>(s->work.size())});
}

static void drop_graphs(mplpp_solver *s)
{
    if (s->g_looped) {
        cudaGraphExecDestroy(s->g_looped);
        s->g_looped = nullptr;
    }
    if (s->g_persist) {
        cudaGraphExecDestroy(s->g_persist);
        s->g_persist = nullptr;
        s->g_persist_iters = -1;
    }
}

// The warp driver (one warp per edge) with T threads per block: per-warp
// vectors sized for the largest label count, as many warp workers as are
// co-resident (at most one per edge of the largest matching), work lists as
// for the cluster driver.
static mplpp_status apply_warp_mapping(mplpp_solver *s, int T, int optin)
{
    if (T % 32 || T < 0 || T > 512) return fail(s, MPLPP_E_INVALID, "threads must be a multiple of 32 in 32..512");
    mapping_for(s, 1, T > 0 ? T : 256);  // sizes of the other drivers stay consistent
    if (T == 0) {  // the block size (<= 256 threads) with the most co-resident warps
        T = 32;
        int best = 0;
        for (int t : {256, 128, 64, 32}) {
            const size_t b =
                static_cast<size_t>(t / 32) * hs_warp_bytes_per_warp(static_cast<int>(round4(s->lmax)), 32 * s->ldmax);
            if (b > static_cast<size_t>(optin)) continue;
            const int w = hs_warp_max_blocks(t, b) * (t / 32);
            if (w > best) {
                best = w;
                T = t;
            }
        }
    }
    s->T = T;
    if (s->EE == 0) return fail(s, MPLPP_E_UNSUPPORTED, "the warp driver needs edges");
    if (s->lmax > kWarpMaxL)
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "the warp driver takes label counts up to " + std::to_string(kWarpMaxL) + " (largest here " +
                        std::to_string(s->lmax) + ")");
    const int lw = static_cast<int>(round4(s->lmax));
    const int wpb = T / 32;
    // table buffers of 32 rows of the widest table (the fewest bytes per warp:
    // the most warps per SM); smaller tables are resident, larger ones stream
    const int cap = 32 * s->ldmax;
    const size_t smem = static_cast<size_t>(wpb) * hs_warp_bytes_per_warp(lw, cap);
    if (smem > static_cast<size_t>(optin)) return fail(s, MPLPP_E_UNSUPPORTED, "warp driver: shared memory");
    const int blocks_max = hs_warp_max_blocks(T, smem);
    if (blocks_max < 1) return fail(s, MPLPP_E_UNSUPPORTED, "warp driver: no block fits");
    int workers = std::min(blocks_max * wpb, s->max_phase);
    workers = std::min(workers, s->work_off_cap - 1);
    if (workers < 1) return fail(s, MPLPP_E_UNSUPPORTED, "warp driver: no worker fits");
    build_work(s, workers);
    CK(s, cudaMemcpyAsync(s->d_work_off, s->work_off.data(), s->work_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                          s->stream));
    CK(s, cudaMemcpyAsync(s->d_work, s->work.data(), s->work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                          s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    s->mode = MPLPP_MODE_WARP;
    s->clusters = workers;
    s->warp_blocks = (workers + wpb - 1) / wpb;
    s->lw = lw;
    s->cap = cap;
    s->smem_warp = smem;
    drop_graphs(s);
    return MPLPP_OK;
}

// Makes (C, T, mode) the solver's mapping: sizes, kernel attributes, and for
// the persistent driver the per-cluster work lists (uploaded to the device).
// want: MPLPP_MODE_AUTO (persistent if possible), _LOOPED or _PERSISTENT.
static_assert(kRuleH == MPLPP_RULE_H && kRuleM == MPLPP_RULE_M && kRuleU == MPLPP_RULE_U, "rule ids");

// The M and U updates: one CTA of 256 threads per edge, looped driver only;
// the node vectors of the largest edge must fit shared memory.
static mplpp_status apply_rule_mapping(mplpp_solver *s, int optin)
{
    mapping_for(s, 1, 256);  // sizes of the other drivers stay consistent
    int lumax = 1;
    for (auto &ed : s->h_edges) lumax = std::max(lumax, ed.Lu);
    s->smem_rule = rule_smem_bytes(lumax, s->ldmax);
    if (s->smem_rule > static_cast<size_t>(optin))
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "the node vectors of the largest edge need " + std::to_string(s->smem_rule) +
                        " B of shared memory (limit " + std::to_string(optin) + ")");
    cudaError_t ce = rule_prepare(s->smem_rule);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "kernel attributes");
    s->mode = MPLPP_MODE_LOOPED;
    drop_graphs(s);
    return MPLPP_OK;
}

// The structured Handshake kernel: every model truncated-linear or -quadratic, one warp per
// edge, vectors of up to kStructMaxL labels in shared memory.
static bool struct_fits(mplpp_solver *s)
{
    int lmax = 1;
    for (auto &nd : s->h_nodes) lmax = std::max(lmax, nd.L);
    return lmax <= kStructMaxL;
}

static mplpp_status apply_struct_mapping(mplpp_solver *s, int optin, bool queue = false)
{
    if (!s->all_structured)
        return fail(s, MPLPP_E_UNSUPPORTED, "structured mode needs every model's costs as MPLPP_PAIR_TRUNC_*");
    if (!struct_fits(s))
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "structured mode takes label counts up to " + std::to_string(kStructMaxL));
    mapping_for(s, 1, 256);  // sizes of the other drivers stay consistent
    int lmax = 1;
    for (auto &nd : s->h_nodes) lmax = std::max(lmax, nd.L);
    s->struct_lmax = static_cast<int>(round4(lmax));
    if (8 * struct_bytes_per_warp(s->struct_lmax) > static_cast<size_t>(optin))
        return fail(s, MPLPP_E_UNSUPPORTED, "structured mode: vectors exceed shared memory");
    cudaError_t ce = struct_prepare(s->struct_lmax);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "kernel attributes");
    s->mode = MPLPP_MODE_STRUCTURED;
    if (queue) {  // persistent: the queue list, co-resident blocks of 8 warps
        int blocks = std::min(struct_queue_max_blocks(s->struct_lmax), (s->EE + 7) / 8);
        if (blocks < 1) return fail(s, MPLPP_E_UNSUPPORTED, "structured queue driver: no block fits");
        if (!s->d_queue) CK(s, s->alloc(&s->d_queue, 1));
        build_queue(s);
        CK(s, cudaMemcpyAsync(s->d_work, s->work.data(), s->work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                              s->stream));
        CK(s, cudaStreamSynchronize(s->stream));
        s->queue_blocks = blocks;
        s->mode = MPLPP_MODE_STRUCTURED_QUEUE;
    }
    drop_graphs(s);
    return MPLPP_OK;
}

namespace mplpp {
cudaError_t raise_smem_limit_ptr(const void *kernel, size_t smem)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if (static_cast<size_t>(a.maxDynamicSharedSizeBytes) >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}
}  // namespace mplpp

// The queue driver: CTAs of 128 threads, vectors and the column partials in
// shared memory, tables read from memory by every pass (from L2 after the
// first); as many CTAs as are co-resident (at most one per edge): the items
// in flight per SM set its throughput.
static mplpp_status apply_queue_mapping(mplpp_solver *s, int T, int optin)
{
    if (T == 0) T = 128;
    if (T % 32 || T < 64 || T > 512) return fail(s, MPLPP_E_INVALID, "threads must be a multiple of 32 in 64..512");
    if (T != 128) return fail(s, MPLPP_E_UNSUPPORTED, "the queue driver runs 128 threads per CTA");
    if (s->EE == 0) return fail(s, MPLPP_E_UNSUPPORTED, "the queue driver needs edges");
    mapping_for(s, 1, T);  // sizes of the other drivers stay consistent
    s->smem_queue = hs_smem_bytes(2, 4, s->rmax, s->ldmax, T, 1);
    if (s->smem_queue > static_cast<size_t>(optin)) return fail(s, MPLPP_E_UNSUPPORTED, "queue driver: shared memory");
    int blocks = hs_queue_max_blocks(T, s->smem_queue);
    blocks = std::min(blocks, s->EE);
    if (blocks < 1) return fail(s, MPLPP_E_UNSUPPORTED, "queue driver: no block fits");
    if (!s->d_queue) CK(s, s->alloc(&s->d_queue, 1));
    build_queue(s);
    CK(s, cudaMemcpyAsync(s->d_work, s->work.data(), s->work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                          s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    s->mode = MPLPP_MODE_QUEUE;
    s->queue_blocks = blocks;
    s->T = T;
    drop_graphs(s);
    return MPLPP_OK;
}

// The resident driver: one CTA per model with the model's state in shared
// memory; a group of 8, 16 or 32 lanes per edge of a matching (threads: enough
// warps for the largest matching, at most 16, unless given).
static mplpp_status apply_resident_mapping(mplpp_solver *s, int T, int optin)
{
    if (T % 32 || T < 0 || T > 512) return fail(s, MPLPP_E_INVALID, "threads must be a multiple of 32 in 32..512");
    if (s->EE == 0) return fail(s, MPLPP_E_UNSUPPORTED, "the resident driver needs edges");
    int lmax = 1, wmax = 1;
    for (auto &nd : s->h_nodes) lmax = std::max(lmax, nd.L);
    if (lmax > kResMaxL)
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "the resident driver takes label counts up to " + std::to_string(kResMaxL) + " (largest here " +
                        std::to_string(lmax) + ")");
    const int nm = static_cast<int>(s->models.size());
    std::vector<ResModel> rm(nm);
    std::vector<int> off;
    std::vector<int4> desc;  // the scheduled edges, relative to their models
    long long state_max = 0, sched_max = 0;
    for (int m = 0; m < nm; ++m) {
        const ModelHost &mh = s->models[m];
        const int n0 = mh.node_base, n1 = mh.node_base + mh.n;
        rm[m].agg_base = s->h_nodes[n0].aoff;
        rm[m].agg_n = (n1 < s->N ? s->h_nodes[n1].aoff : s->aggN) - rm[m].agg_base;
        if (mh.E > 0) {
            rm[m].msg_base = s->h_edges[mh.edge_base].mu;
            const int e1 = mh.edge_base + mh.E;
            rm[m].msg_n = (e1 < s->EE ? s->h_edges[e1].mu : s->msgN) - rm[m].msg_base;
        } else {
            rm[m].msg_base = 0;
            rm[m].msg_n = 0;
        }
        if (mh.E > 0) {
            rm[m].tab_base = s->h_edges[mh.edge_base].toff;
            const int e1 = mh.edge_base + mh.E;
            rm[m].tab_n = (e1 < s->EE ? s->h_edges[e1].toff : s->tabN) - rm[m].tab_base;
        } else {
            rm[m].tab_base = 0;
            rm[m].tab_n = 0;
        }
        sched_max = std::max(sched_max, static_cast<long long>(mh.off.size()));
        rm[m].sched = static_cast<int>(off.size());
        rm[m].P = static_cast<int>(mh.off.size()) - 1;
        for (size_t k = 0; k < mh.off.size(); ++k) off.push_back(static_cast<int>(desc.size()) + mh.off[k]);
        for (int i = 0; i < mh.E; ++i) {
            const EdgeDesc &ed = s->h_edges[mh.edge_base + mh.order[i]];
            const long long t = ed.toff - rm[m].tab_base;
            const long long au = ed.au - rm[m].agg_base, av = ed.av - rm[m].agg_base;
            const long long mu = ed.mu - rm[m].msg_base, mv = ed.mv - rm[m].msg_base;
            if (t > INT32_MAX || au > 0xffff || av > 0xffff || mu > 0xffff || mv > 0xffff)
                return fail(s, MPLPP_E_UNSUPPORTED, "the resident driver takes models of at most 65,536 state entries");
            desc.push_back(make_int4(static_cast<int>(t), static_cast<int>(au | (av << 16)),
                                     static_cast<int>(mu | (mv << 16)), ed.Lu | (ed.Lv << 8) | (ed.ld << 16)));
        }
        for (size_t k = 0; k + 1 < mh.off.size(); ++k) wmax = std::max(wmax, mh.off[k + 1] - mh.off[k]);
        state_max = std::max(state_max, rm[m].agg_n + rm[m].msg_n);
    }
    // a warp updates 32 / res_lanes(lmax) edges at once: enough warps for the
    // largest matching, at most 16
    const int epw = 32 / res_lanes(lmax);
    if (T == 0) T = 32 * std::min(16, (wmax + epw - 1) / epw);
    // the state, the groups' vectors and the model's matching offsets; the
    // tables and edge descriptors are read from memory (staging the tables in
    // shared memory as well measured slower on the K_20 replicas: fewer
    // models per SM)
    size_t smem = static_cast<size_t>(state_max) * sizeof(float2) + 8 /* alignment of the vectors */ +
                  static_cast<size_t>(T / 32) * kResWarpBytes + static_cast<size_t>(sched_max) * sizeof(int);
    smem = (smem + 15) / 16 * 16;
    if (smem > static_cast<size_t>(optin))
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "the resident driver needs " + std::to_string(smem) + " B of shared memory for the largest model");
    mapping_for(s, 1, 256);  // sizes of the other drivers stay consistent
    cudaError_t ce = res_prepare(smem);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "kernel attributes");
    if (!s->d_res_models) {
        CK(s, s->alloc(&s->d_res_models, nm));
        CK(s, s->alloc(&s->d_res_off, off.size()));
        CK(s, s->alloc(&s->d_res_desc, std::max<size_t>(1, desc.size())));
        CK(s, cudaMemcpyAsync(s->d_res_models, rm.data(), sizeof(ResModel) * nm, cudaMemcpyHostToDevice, s->stream));
        CK(s, cudaMemcpyAsync(s->d_res_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s->stream));
        CK(s, cudaMemcpyAsync(s->d_res_desc, desc.data(), sizeof(int4) * desc.size(), cudaMemcpyHostToDevice,
                              s->stream));
        CK(s, cudaStreamSynchronize(s->stream));
    }
    s->mode = MPLPP_MODE_RESIDENT;
    s->T = T;
    s->smem_res = smem;
    drop_graphs(s);
    return MPLPP_OK;
}

static mplpp_status apply_mapping(mplpp_solver *s, int C, int T, int want)
{
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (s->opt.rule != kRuleH) return apply_rule_mapping(s, optin);
    if (want == MPLPP_MODE_STRUCTURED || (want == MPLPP_MODE_AUTO && s->all_structured && struct_fits(s)))
        return apply_struct_mapping(s, optin);
    if (want == MPLPP_MODE_STRUCTURED_QUEUE) return apply_struct_mapping(s, optin, true);
    if (want == MPLPP_MODE_WARP) return apply_warp_mapping(s, T, optin);
    if (want == MPLPP_MODE_QUEUE) return apply_queue_mapping(s, T, optin);
    if (want == MPLPP_MODE_RESIDENT) return apply_resident_mapping(s, T, optin);
    mapping_for(s, C, T);
    if (s->smem_looped > static_cast<size_t>(optin))
        return fail(s, MPLPP_E_UNSUPPORTED,
                    "largest table needs " + std::to_string(s->smem_looped) + " B of shared memory per CTA with " +
                        std::to_string(C) + " CTAs per edge (limit " + std::to_string(optin) + ")");
    cudaError_t ce = hs_prepare(std::max(s->smem_looped, std::min(s->smem_persist, static_cast<size_t>(optin))));
    if (ce != cudaSuccess) return cuda_fail(s, ce, "kernel attributes");
    int mode = MPLPP_MODE_LOOPED;
    if (want != MPLPP_MODE_LOOPED && s->smem_persist <= static_cast<size_t>(optin) && s->EE > 0) {
        int clusters = hs_max_active_clusters(C, s->T, s->smem_persist, s->rr);
        clusters = std::min(clusters, s->max_phase);
        if (clusters >= 1 && clusters + 1 <= s->work_off_cap) {
            mode = MPLPP_MODE_PERSISTENT;
            s->clusters = clusters;
            build_work(s, clusters);
            CK(s, cudaMemcpyAsync(s->d_work_off, s->work_off.data(), s->work_off.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, s->stream));
            CK(s, cudaMemcpyAsync(s->d_work, s->work.data(), s->work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                  s->stream));
            CK(s, cudaStreamSynchronize(s->stream));
        }
    }
    if (want == MPLPP_MODE_PERSISTENT && mode != MPLPP_MODE_PERSISTENT)
        return fail(s, MPLPP_E_UNSUPPORTED, "persistent mode is not possible for these shapes on this device");
    s->mode = mode;
    drop_graphs(s);
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_create(const mplpp_model *models, int32_t n_models, const mplpp_options *opt,
                                     void *stream, mplpp_solver **out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, MPLPP_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!models || n_models < 1) return fail(nullptr, MPLPP_E_INVALID, "need at least one model");
    std::unique_ptr<mplpp_solver> s(new mplpp_solver());
    if (opt) s->opt = *opt;
    else mplpp_options_default(&s->opt);
    if (s->opt.spin_limit <= 0) s->opt.spin_limit = 1LL << 22;
    s->stream = static_cast<cudaStream_t>(stream);
    {
        const mplpp_options &o = s->opt;
        if (o.mode < MPLPP_MODE_AUTO || o.mode > MPLPP_MODE_STRUCTURED_QUEUE)
            return fail(nullptr, MPLPP_E_INVALID, "unknown mode");
        if (o.cluster < 0 || o.cluster > 8) return fail(nullptr, MPLPP_E_INVALID, "cluster must be 0 or 1..8");
        if (o.rule < MPLPP_RULE_H || o.rule > MPLPP_RULE_U) return fail(nullptr, MPLPP_E_INVALID, "unknown rule");
        if (o.rule != MPLPP_RULE_H && o.record_every > 0)
            return fail(nullptr, MPLPP_E_INVALID, "backward is defined for the Handshake update only");
        if (o.rule != MPLPP_RULE_H &&
            (o.mode == MPLPP_MODE_PERSISTENT || o.mode == MPLPP_MODE_WARP || o.mode == MPLPP_MODE_STRUCTURED ||
             o.mode == MPLPP_MODE_QUEUE || o.mode == MPLPP_MODE_RESIDENT || o.mode == MPLPP_MODE_STRUCTURED_QUEUE))
            return fail(nullptr, MPLPP_E_UNSUPPORTED, "the M and U updates run in the looped driver only");
        // a CTA of the cluster drivers splits its warps between the two node
        // vectors, so it needs two warps at least
        const int tmin = o.mode == MPLPP_MODE_WARP ? 32 : 64;
        if (o.threads != 0 && (o.threads % 32 || o.threads < tmin || o.threads > 512))
            return fail(nullptr, MPLPP_E_INVALID,
                        "threads must be 0 or a multiple of 32 in " + std::to_string(tmin) + "..512");
    }

    // ---- host-side validation, schedules, layout --------------------------------
    s->models.resize(n_models);
    long long aoff = 0, moff = 0, toff = 0;
    int P = 0;
    for (int m = 0; m < n_models; ++m) {
        const mplpp_model &md = models[m];
        ModelHost &mh = s->models[m];
        if (md.n_nodes < 1 || md.n_edges < 0) return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": bad sizes");
        if (md.pair_kind < MPLPP_PAIR_DENSE || md.pair_kind > MPLPP_PAIR_TRUNC_QUAD)
            return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": unknown pair_kind");
        mh.structured = md.pair_kind != MPLPP_PAIR_DENSE;
        mh.pair_kind = md.pair_kind;
        const bool pairs_given = mh.structured ? (md.pair_param != nullptr) : (md.pairwise != nullptr);
        if (!md.labels || !md.unary || (md.n_edges > 0 && (!md.edge_u || !md.edge_v || !pairs_given)))
            return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": NULL array");
        if (mh.structured && md.pairwise)
            return fail(nullptr, MPLPP_E_INVALID,
                        "model " + std::to_string(m) + ": structured costs come in pair_param; pairwise must be NULL");
        if (mh.structured && s->opt.record_every > 0)
            return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": no backward for structured costs");
        if (mh.structured && !s->opt.inputs_on_device)
            for (long long i = 0; i < 2LL * md.n_edges; ++i)
                if (!std::isfinite(md.pair_param[i]) || md.pair_param[i] < 0.f)
                    return fail(nullptr, MPLPP_E_INVALID,
                                "model " + std::to_string(m) + ": pair_param must be finite and >= 0");
        mh.n = md.n_nodes;
        mh.E = md.n_edges;
        mh.L.assign(md.labels, md.labels + md.n_nodes);
        mh.eu.assign(md.edge_u, md.edge_u + md.n_edges);
        mh.ev.assign(md.edge_v, md.edge_v + md.n_edges);
        for (int l : mh.L)
            if (l < 1 || l > 65535) return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": labels must be in 1..65535");
        std::string err;
        if (md.schedule_kind == MPLPP_SCHED_USER) {
            if (md.n_matchings < 0 || !md.matching_off || (md.n_edges > 0 && !md.edge_order))
                return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": user schedule missing");
            mh.off.assign(md.matching_off, md.matching_off + md.n_matchings + 1);
            mh.order.assign(md.edge_order, md.edge_order + md.n_edges);
            err = check_graph(mh.n, mh.eu, mh.ev);
            if (err.empty()) err = check_schedule(mh.n, mh.eu, mh.ev, mh.off, mh.order);
        } else {
            err = build_schedule(md.schedule_kind, mh.n, mh.eu, mh.ev, mh.off, mh.order);
        }
        if (!err.empty()) return fail(nullptr, MPLPP_E_INVALID, "model " + std::to_string(m) + ": " + err);
        mh.node_base = s->N;
        mh.edge_base = s->EE;
        long long uoff = 0, poff = 0;
        for (int u = 0; u < mh.n; ++u) {
            NodeDesc nd;
            nd.aoff = aoff;
            nd.uoff = uoff;
            nd.L = mh.L[u];
            nd.model = m;
            s->h_nodes.push_back(nd);
            aoff += round4(mh.L[u]);
            uoff += mh.L[u];
        }
        mh.unary_size = uoff;
        for (int e = 0; e < mh.E; ++e) {
            EdgeDesc ed;
            ed.gu = mh.node_base + mh.eu[e];
            ed.gv = mh.node_base + mh.ev[e];
            ed.Lu = mh.L[mh.eu[e]];
            ed.Lv = mh.L[mh.ev[e]];
            ed.ld = static_cast<int>(round4(ed.Lv));
            ed.toff = toff;
            ed.mu = moff;
            ed.mv = moff + round4(ed.Lu);
            ed.au = s->h_nodes[ed.gu].aoff;
            ed.av = s->h_nodes[ed.gv].aoff;
            ed.poff = poff;
            ed.model = m;
            s->h_edges.push_back(ed);
            toff += 1LL * ed.Lu * ed.ld;
            moff += round4(ed.Lu) + round4(ed.Lv);
            poff += 1LL * ed.Lu * ed.Lv;
            s->bytes_per_iter += 4LL * ed.Lu * ed.Lv + 32LL * (ed.Lu + ed.Lv);
        }
        mh.pair_size = poff;
        s->N += mh.n;
        s->EE += mh.E;
        s->sum_unary += mh.unary_size;
        s->sum_pair += mh.pair_size;
        P = std::max(P, static_cast<int>(mh.off.size()) - 1);
    }
    s->aggN = aoff;
    s->msgN = moff;
    s->tabN = toff;
    s->P = P;
    for (auto &ed : s->h_edges) s->sum_msg += ed.Lu + ed.Lv;
    // phase p = matching p of every model
    s->phase_off.assign(1, 0);
    for (int p = 0; p < P; ++p) {
        for (auto &mh : s->models)
            if (p + 1 < static_cast<int>(mh.off.size()))
                for (int i = mh.off[p]; i < mh.off[p + 1]; ++i) s->phase_edges.push_back(mh.edge_base + mh.order[i]);
        s->phase_off.push_back(static_cast<int>(s->phase_edges.size()));
    }
    // in-edges (edges whose larger end is u), sorted by the smaller end
    s->in_off.assign(s->N + 1, 0);
    for (auto &ed : s->h_edges) s->in_off[ed.gv + 1]++;
    for (int u = 0; u < s->N; ++u) s->in_off[u + 1] += s->in_off[u];
    s->in_edge.assign(s->EE, 0);
    {
        std::vector<int> fill(s->in_off.begin(), s->in_off.end() - 1);
        for (int e = 0; e < s->EE; ++e) s->in_edge[fill[s->h_edges[e].gv]++] = e;
        for (int u = 0; u < s->N; ++u)
            std::sort(s->in_edge.begin() + s->in_off[u], s->in_edge.begin() + s->in_off[u + 1],
                      [&](int a, int b) { return s->h_edges[a].gu < s->h_edges[b].gu; });
        s->in_rec.resize(s->EE);
        for (int k = 0; k < s->EE; ++k) {
            const EdgeDesc &ed = s->h_edges[s->in_edge[k]];
            s->in_rec[k] = InRec{ed.toff, ed.mu, ed.mv, ed.ld, ed.gu};
        }
    }
    // levels of the rounding order: level(u) = 1 + the largest level of u's
    // earlier neighbours (0 without any).  Worth a launch per level only when
    // there are far fewer levels than nodes in the largest model.
    {
        std::vector<int> level(s->N, 0);
        int n_levels = 0, max_n = 0;
        for (int u = 0; u < s->N; ++u) {
            for (int k = s->in_off[u]; k < s->in_off[u + 1]; ++k)
                level[u] = std::max(level[u], level[s->in_rec[k].gu] + 1);
            n_levels = std::max(n_levels, level[u] + 1);
        }
        for (auto &mh : s->models) max_n = std::max(max_n, mh.n);
        s->level_off.clear();
        if (s->N > 0 && 4 * n_levels <= max_n) {
            s->level_off.assign(n_levels + 1, 0);
            for (int u = 0; u < s->N; ++u) s->level_off[level[u] + 1]++;
            for (int l = 0; l < n_levels; ++l) s->level_off[l + 1] += s->level_off[l];
            s->level_nodes.assign(s->N, 0);
            std::vector<int> fill(s->level_off.begin(), s->level_off.end() - 1);
            for (int u = 0; u < s->N; ++u) s->level_nodes[fill[level[u]]++] = u;
        }
    }
    s->mnode_off.assign(1, 0);
    s->medge_off.assign(1, 0);
    for (auto &mh : s->models) {
        s->mnode_off.push_back(mh.node_base + mh.n);
        s->medge_off.push_back(mh.edge_base + mh.E);
    }
    uint64_t h = 1469598103934665603ULL;
    h = fnv(h, &n_models, sizeof(n_models));
    for (auto &mh : s->models) {
        h = fnv(h, mh.L.data(), mh.L.size() * sizeof(int));
        h = fnv(h, mh.eu.data(), mh.eu.size() * sizeof(int));
        h = fnv(h, mh.ev.data(), mh.ev.size() * sizeof(int));
        h = fnv(h, mh.off.data(), mh.off.size() * sizeof(int));
        h = fnv(h, mh.order.data(), mh.order.size() * sizeof(int));
    }
    s->shape_hash = h;

    // ---- device ----------------------------------------------------------------
    mplpp_solver *S = s.get();
    cudaError_t ce = cudaGetDevice(&S->device);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "cudaGetDevice");
    int sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, S->device);
    S->sms = sms;
    choose_mapping(S, sms, optin);
    const int chosenC = S->C;

    ce = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "cudaStreamCreate");
    S->stream_ok = true;
#define CKC(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(nullptr, e_, #call); \
    } while (0)
    CKC(S->alloc(&S->d_edges, S->EE));
    CKC(S->alloc(&S->d_nodes, S->N));
    CKC(S->alloc(&S->d_tab, S->tabN));
    CKC(S->alloc(&S->d_agg, S->aggN));
    CKC(S->alloc(&S->d_un0, S->aggN));
    CKC(S->alloc(&S->d_msg, S->msgN));
    CKC(S->alloc(&S->d_phase_edges, S->phase_edges.size()));
    CKC(S->alloc(&S->d_err, 1));
    CKC(S->alloc(&S->d_in_off, S->in_off.size()));
    CKC(S->alloc(&S->d_in_rec, std::max<size_t>(1, S->in_rec.size())));
    CKC(S->alloc(&S->d_mnode_off, S->mnode_off.size()));
    CKC(S->alloc(&S->d_medge_off, S->medge_off.size()));
    CKC(S->alloc(&S->d_emin, S->EE));
    CKC(S->alloc(&S->d_nmin, S->N));
    CKC(S->alloc(&S->d_out, n_models));
    CKC(S->alloc(&S->d_labels, S->N));
    CKC(S->alloc(&S->d_energy, n_models));
    S->work_off_cap = sms * 64 + 1;  // clusters never exceed the co-resident CTAs
    CKC(S->alloc(&S->d_work_off, S->work_off_cap));
    CKC(S->alloc(&S->d_work, std::max(1, S->EE)));
    cudaStream_t st = S->stream;
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    CKC(h2d(S->d_edges, S->h_edges.data(), S->h_edges.size() * sizeof(EdgeDesc)));
    CKC(h2d(S->d_nodes, S->h_nodes.data(), S->h_nodes.size() * sizeof(NodeDesc)));
    CKC(h2d(S->d_phase_edges, S->phase_edges.data(), S->phase_edges.size() * sizeof(int)));
    CKC(h2d(S->d_in_off, S->in_off.data(), S->in_off.size() * sizeof(int)));
    CKC(h2d(S->d_in_rec, S->in_rec.data(), S->in_rec.size() * sizeof(InRec)));
    if (!S->level_off.empty()) {
        CKC(S->alloc(&S->d_level_nodes, S->level_nodes.size()));
        CKC(h2d(S->d_level_nodes, S->level_nodes.data(), S->level_nodes.size() * sizeof(int)));
    }
    CKC(h2d(S->d_mnode_off, S->mnode_off.data(), S->mnode_off.size() * sizeof(int)));
    CKC(h2d(S->d_medge_off, S->medge_off.data(), S->medge_off.size() * sizeof(int)));
    // structured costs: (w, tau) per edge
    S->all_structured = S->EE > 0;
    bool any_structured = false;
    for (auto &mh : S->models) {
        S->all_structured = S->all_structured && mh.structured;
        any_structured = any_structured || (mh.structured && mh.E > 0);
    }
    if (any_structured) {
        CKC(S->alloc(&S->d_pair_param, S->EE));
        CKC(S->alloc(&S->d_pair_kind, S->EE));
        CKC(cudaMemsetAsync(S->d_pair_param, 0, sizeof(float2) * S->EE, st));
        std::vector<int> kinds;
        kinds.reserve(S->EE);
        for (auto &mh : S->models) kinds.insert(kinds.end(), mh.E, mh.pair_kind);
        CKC(cudaMemcpyAsync(S->d_pair_kind, kinds.data(), sizeof(int) * kinds.size(), cudaMemcpyHostToDevice, st));
        CKC(cudaStreamSynchronize(st));  // kinds is a host temporary
        for (int m = 0; m < n_models; ++m) {
            const ModelHost &mh = S->models[m];
            if (!mh.structured || mh.E == 0) continue;
            CKC(cudaMemcpyAsync(S->d_pair_param + mh.edge_base, models[m].pair_param, sizeof(float2) * mh.E,
                                S->opt.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        }
    }
    {
        mplpp_status ms = apply_mapping(S, chosenC, S->opt.threads, S->opt.mode);
        if (ms != MPLPP_OK) return fail(nullptr, ms, S->err);
    }
    CKC(cudaMemsetAsync(S->d_err, 0, sizeof(int), st));
    CKC(cudaMemsetAsync(S->d_msg, 0, S->msgN * sizeof(ulonglong2), st));  // 0, version 0

    // costs: stage (host inputs) or read in place (device inputs), then pack
    float *stage_u = nullptr, *stage_p = nullptr;
    if (!S->opt.inputs_on_device) {
        CKC(dalloc(&stage_u, S->sum_unary));
        CKC(dalloc(&stage_p, S->sum_pair));
    }
    cudaError_t pe = cudaSuccess;
    long long ub = 0, pb = 0;
    for (int m = 0; m < n_models && pe == cudaSuccess; ++m) {
        const ModelHost &mh = S->models[m];
        const float *su = models[m].unary;
        const float *sp = models[m].pairwise;
        if (!S->opt.inputs_on_device) {
            pe = h2d(stage_u + ub, models[m].unary, mh.unary_size * sizeof(float));
            if (pe == cudaSuccess && mh.pair_size && !mh.structured)
                pe = h2d(stage_p + pb, models[m].pairwise, mh.pair_size * sizeof(float));
            su = stage_u + ub;
            sp = stage_p + pb;
        }
        if (pe == cudaSuccess)
            pe = launch_pack(S->d_edges + mh.edge_base, mh.structured ? 0 : mh.E, S->d_nodes + mh.node_base, mh.n, su,
                             sp, S->d_tab, S->d_un0, S->d_agg, S->d_err, st);
        if (pe == cudaSuccess && mh.structured)
            pe = launch_materialize(S->d_edges + mh.edge_base, S->d_pair_param + mh.edge_base,
                                    S->d_pair_kind + mh.edge_base, mh.E, S->d_tab, S->d_err, st);
        ub += mh.unary_size;
        pb += mh.pair_size;
    }
    cudaError_t se = cudaStreamSynchronize(st);
    if (stage_u) cudaFree(stage_u);
    if (stage_p) cudaFree(stage_p);
    if (pe != cudaSuccess) return cuda_fail(nullptr, pe, "packing the costs");
    if (se != cudaSuccess) return cuda_fail(nullptr, se, "packing the costs");
    int herr = 0;
    CKC(cudaMemcpy(&herr, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(nullptr, MPLPP_E_INVALID, "costs must be finite");
#undef CKC
    *out = s.release();
    return MPLPP_OK;
}

// ---- iteration drivers ------------------------------------------------------------
static mplpp_status check_device_error(mplpp_solver *s);

static HsParams make_params(mplpp_solver *s)
{
    HsParams p = {};
    p.edges = s->d_edges;
    p.tab = s->d_tab;
    p.agg = s->d_agg;
    p.msg = s->d_msg;
    p.items = s->d_phase_edges;
    p.work_off = s->d_work_off;
    p.work = s->d_work;
    p.err = s->d_err;
    p.spin_limit = s->opt.spin_limit;
    p.test_wait = s->opt.test_unreachable_wait ? 1 : 0;
    p.rr = s->rr ? 1 : 0;
    p.pw = s->pw ? 1 : 0;
    p.queue = s->d_queue;
    p.queue_items = s->EE;
    p.C = s->C;
    p.tile_floats = s->tile_floats;
    p.workers = s->mode == MPLPP_MODE_WARP ? s->clusters : 0;
    p.lw = s->lw;
    p.cap = s->cap;
    p.rmax = s->rmax;
    p.ldmax = s->ldmax;
    return p;
}

// One iteration of looped launches (one per matching) on stream st.
cudaError_t enqueue_looped_iteration(mplpp_solver *s, cudaStream_t st)
{
    if (s->mode == MPLPP_MODE_STRUCTURED) {
        StructParams sp = {s->d_edges, nullptr, 0, s->struct_lmax, s->d_pair_param, s->d_pair_kind, s->d_agg,
                           s->d_msg};
        for (int ph = 0; ph + 1 < static_cast<int>(s->phase_off.size()); ++ph) {
            sp.items = s->d_phase_edges + s->phase_off[ph];
            sp.n_items = s->phase_off[ph + 1] - s->phase_off[ph];
            cudaError_t e = launch_struct(sp, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (s->opt.rule != kRuleH) {
        RuleParams rp = {s->d_edges, nullptr, s->d_tab, s->d_agg, s->d_msg};
        for (int ph = 0; ph + 1 < static_cast<int>(s->phase_off.size()); ++ph) {
            rp.items = s->d_phase_edges + s->phase_off[ph];
            cudaError_t e = launch_rule(rp, s->opt.rule, s->phase_off[ph + 1] - s->phase_off[ph], s->smem_rule, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    HsParams p = make_params(s);
    for (int ph = 0; ph + 1 < static_cast<int>(s->phase_off.size()); ++ph) {
        p.items = s->d_phase_edges + s->phase_off[ph];
        const int n = s->phase_off[ph + 1] - s->phase_off[ph];
        cudaError_t e = hs_launch_looped(p, n, s->T, s->smem_looped, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// `iterations` iterations of the persistent kernel.  The versions of the
// state entries count updates from 0 within one launch, so they are reset
// first (whatever ran before: looped launches, an aborted run, load_state).
cudaError_t enqueue_persistent(mplpp_solver *s, cudaStream_t st, int iterations)
{
    if (s->mode == MPLPP_MODE_STRUCTURED_QUEUE) {
        cudaError_t e = launch_restamp(s->d_agg, s->aggN, s->d_msg, s->msgN, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->d_queue, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        StructParams sp = {s->d_edges, nullptr, 0, s->struct_lmax, s->d_pair_param, s->d_pair_kind, s->d_agg,
                           s->d_msg};
        sp.work = s->d_work;
        sp.queue = s->d_queue;
        sp.queue_items = s->EE;
        sp.iterations = iterations;
        sp.test_wait = s->opt.test_unreachable_wait ? 1 : 0;
        sp.err = s->d_err;
        sp.spin_limit = s->opt.spin_limit;
        return launch_struct_queue(sp, s->queue_blocks, st);
    }
    if (s->mode == MPLPP_MODE_RESIDENT) {  // reads values only, writes version 0: no restamp
        ResParams rp = {s->d_tab, s->d_agg, s->d_msg, s->d_res_models, s->d_res_off, s->d_res_desc, iterations};
        int lmax = 1;
        for (auto &nd : s->h_nodes) lmax = std::max(lmax, nd.L);
        return launch_resident(rp, static_cast<int>(s->models.size()), s->T, s->smem_res, lmax, st);
    }
    HsParams p = make_params(s);
    cudaError_t e = launch_restamp(s->d_agg, s->aggN, s->d_msg, s->msgN, st);
    if (e != cudaSuccess) return e;
    p.iterations = iterations;
    if (s->mode == MPLPP_MODE_WARP) return hs_launch_warp(p, s->warp_blocks, s->T, s->smem_warp, st);
    if (s->mode == MPLPP_MODE_QUEUE) {
        e = cudaMemsetAsync(s->d_queue, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        p.tile_floats = 4;  // no staged tables
        return hs_launch_queue(p, s->queue_blocks, s->T, s->smem_queue, st);
    }
    return hs_launch_persistent(p, s->clusters, s->T, s->smem_persist, st);
}

static mplpp_status run_plain(mplpp_solver *s, int iterations)
{
    if (iterations == 0 || s->EE == 0) return MPLPP_OK;
    if (s->mode == MPLPP_MODE_LOOPED || s->mode == MPLPP_MODE_STRUCTURED) {
        if (s->opt.use_graph) {
            if (!s->g_looped) {
                cudaGraph_t g = nullptr;
                CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_looped_iteration(s, s->cap_stream);
                cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
                if (e != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return cuda_fail(s, e, "capturing the looped iteration");
                }
                if (e2 != cudaSuccess) return cuda_fail(s, e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&s->g_looped, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
            }
            for (int it = 0; it < iterations; ++it) CK(s, cudaGraphLaunch(s->g_looped, s->stream));
        } else {
            for (int it = 0; it < iterations; ++it) CK(s, enqueue_looped_iteration(s, s->stream));
        }
        s->launches += static_cast<long long>(iterations) * s->P;
    } else {
        if (s->opt.use_graph) {
            if (!s->g_persist || s->g_persist_iters != iterations) {
                if (s->g_persist) {
                    cudaGraphExecDestroy(s->g_persist);
                    s->g_persist = nullptr;
                }
                cudaGraph_t g = nullptr;
                CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_persistent(s, s->cap_stream, iterations);
                cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
                if (e != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return cuda_fail(s, e, "capturing the persistent launch");
                }
                if (e2 != cudaSuccess) return cuda_fail(s, e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&s->g_persist, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
                s->g_persist_iters = iterations;
            }
            CK(s, cudaGraphLaunch(s->g_persist, s->stream));
        } else {
            CK(s, enqueue_persistent(s, s->stream, iterations));
        }
        s->launches += s->mode == MPLPP_MODE_RESIDENT ? 1 : 2;  // (restamp +) the kernel
    }
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_run(mplpp_solver *s, int32_t iterations)
{
    if (!s) return MPLPP_E_INVALID;
    if (iterations < 0) return fail(s, MPLPP_E_INVALID, "iterations must be >= 0");
    s->err.clear();
    mplpp_status st = run_plain(s, iterations);
    if (st == MPLPP_OK) s->iterations += iterations;
    return st;
}

static mplpp_status check_device_error(mplpp_solver *s)
{
    int herr = 0;
    CK(s, cudaMemcpy(&herr, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        CK(s, cudaMemset(s->d_err, 0, sizeof(int)));
        if (herr == ERR_TIMEOUT)
            return fail(s, MPLPP_E_TIMEOUT, "a device-side wait exceeded spin_limit; the state is undefined");
        return fail(s, MPLPP_E_NONFINITE, "non-finite value on the device");
    }
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_sync(mplpp_solver *s)
{
    if (!s) return MPLPP_E_INVALID;
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

extern "C" mplpp_status mplpp_bound(mplpp_solver *s, double *out, int32_t exact)
{
    if (!s || !out) return MPLPP_E_INVALID;
    s->err.clear();
    CK(s, launch_bound(s->d_edges, s->EE, s->d_nodes, s->N, s->d_tab, s->d_agg, s->d_msg, s->d_emin, s->d_nmin,
                       s->d_mnode_off, s->d_medge_off, static_cast<int>(s->models.size()), exact ? 1 : 0, s->lmax,
                       s->d_out, s->stream));
    CK(s, cudaMemcpyAsync(out, s->d_out, sizeof(double) * s->models.size(), cudaMemcpyDeviceToHost, s->stream));
    mplpp_status st = mplpp_sync(s);
    if (st != MPLPP_OK) return st;
    for (size_t m = 0; m < s->models.size(); ++m)
        if (!std::isfinite(out[m])) return fail(s, MPLPP_E_NONFINITE, "dual bound is not finite");
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_labeling(mplpp_solver *s, int32_t *labels, double *energy)
{
    if (!s || !labels) return MPLPP_E_INVALID;
    s->err.clear();
    CK(s, launch_round(s->d_edges, s->d_nodes, s->d_in_off, s->d_in_rec, s->d_mnode_off, s->d_medge_off,
                       static_cast<int>(s->models.size()), s->d_tab, s->d_agg, s->d_msg, s->d_un0, s->d_labels,
                       s->d_energy, s->d_err, s->d_level_nodes, s->level_off.data(),
                       static_cast<int>(s->level_off.empty() ? 0 : s->level_off.size() - 1), s->stream));
    CK(s, cudaMemcpyAsync(labels, s->d_labels, sizeof(int) * s->N, cudaMemcpyDeviceToHost, s->stream));
    if (energy)
        CK(s, cudaMemcpyAsync(energy, s->d_energy, sizeof(double) * s->models.size(), cudaMemcpyDeviceToHost,
                              s->stream));
    return mplpp_sync(s);
}

extern "C" mplpp_status mplpp_reset(mplpp_solver *s)
{
    if (!s) return MPLPP_E_INVALID;
    s->err.clear();
    CK(s, launch_init_state(s->d_un0, s->d_agg, s->aggN, s->d_msg, s->msgN, s->stream));
    s->iterations = 0;
    s->history_valid = true;
    return MPLPP_OK;
}

// A host array the device reads in place: pinned and mapped host memory
// (cudaHostAlloc memory under unified addressing, which a Grace-attached GPU
// reads over its chip-to-chip link): its device address; else nullptr (the
// caller copies it to device memory first).
static const float *device_view(const float *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA allocation: clear the error
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<const float *>(a.devicePointer);
    return nullptr;
}

extern "C" mplpp_status mplpp_update_costs(mplpp_solver *s, const float *const *unary, const float *const *pairwise)
{
    if (!s || !unary || !pairwise) return MPLPP_E_INVALID;
    s->err.clear();
    const int n_models = static_cast<int>(s->models.size());
    for (int m = 0; m < n_models; ++m)
        if (s->models[m].structured)
            return fail(s, MPLPP_E_UNSUPPORTED, "model " + std::to_string(m) + ": structured costs: create a new solver");
    for (int m = 0; m < n_models; ++m)
        if (!unary[m] || (!pairwise[m] && s->models[m].pair_size))
            return fail(s, MPLPP_E_INVALID, "model " + std::to_string(m) + ": NULL cost array");
    cudaStream_t st = s->stream;
    if (!s->opt.inputs_on_device && !s->d_stage_u) {
        CK(s, s->alloc(&s->d_stage_u, std::max<long long>(1, s->sum_unary)));
        CK(s, s->alloc(&s->d_stage_p, std::max<long long>(1, s->sum_pair)));
    }
    CK(s, cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
    long long ub = 0, pb = 0;
    for (int m = 0; m < n_models; ++m) {
        const ModelHost &mh = s->models[m];
        const float *su = unary[m];
        const float *sp = pairwise[m];
        if (!s->opt.inputs_on_device) {
            // pinned, mapped host arrays are read by the packing kernel in
            // place; others are copied to the staging buffers first
            const float *du = device_view(unary[m]);
            if (du) {
                su = du;
            } else {
                CK(s, cudaMemcpyAsync(s->d_stage_u + ub, unary[m], mh.unary_size * sizeof(float),
                                      cudaMemcpyHostToDevice, st));
                su = s->d_stage_u + ub;
            }
            const float *dp = mh.pair_size ? device_view(pairwise[m]) : nullptr;
            if (dp) {
                sp = dp;
            } else {
                if (mh.pair_size)
                    CK(s, cudaMemcpyAsync(s->d_stage_p + pb, pairwise[m], mh.pair_size * sizeof(float),
                                          cudaMemcpyHostToDevice, st));
                sp = s->d_stage_p + pb;
            }
        }
        CK(s, launch_pack(s->d_edges + mh.edge_base, mh.E, s->d_nodes + mh.node_base, mh.n, su, sp, s->d_tab, s->d_un0,
                          s->d_agg, s->d_err, st));
        ub += mh.unary_size;
        pb += mh.pair_size;
    }
    CK(s, launch_init_state(s->d_un0, s->d_agg, s->aggN, s->d_msg, s->msgN, st));
    s->iterations = 0;
    s->history_valid = true;
    CK(s, cudaStreamSynchronize(st));
    int herr = 0;
    CK(s, cudaMemcpy(&herr, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        CK(s, cudaMemset(s->d_err, 0, sizeof(int)));
        return fail(s, MPLPP_E_INVALID, "costs must be finite");
    }
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_state_size(const mplpp_solver *s, size_t *bytes)
{
    if (!s || !bytes) return MPLPP_E_INVALID;
    *bytes = sizeof(mplpp_state_header) + sizeof(double) * (s->sum_unary + s->sum_msg);
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_save_state(mplpp_solver *s, void *buf, size_t size)
{
    if (!s || !buf) return MPLPP_E_INVALID;
    s->err.clear();
    size_t need = 0;
    mplpp_state_size(s, &need);
    if (size < need) return fail(s, MPLPP_E_INVALID, "state buffer too small");
    std::vector<ulonglong2> agg(s->aggN), msg(s->msgN);
    CK(s, cudaMemcpyAsync(agg.data(), s->d_agg, s->aggN * sizeof(ulonglong2), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaMemcpyAsync(msg.data(), s->d_msg, s->msgN * sizeof(ulonglong2), cudaMemcpyDeviceToHost, s->stream));
    mplpp_status st = mplpp_sync(s);
    if (st != MPLPP_OK) return st;
    mplpp_state_header h;
    h.magic = 0x4D504C50u;
    h.version = 2;
    h.shape_hash = s->shape_hash;
    h.iterations = s->iterations;
    h.n_unary = s->sum_unary;
    h.n_msg = s->sum_msg;
    char *p = static_cast<char *>(buf);
    std::memcpy(p, &h, sizeof(h));
    // portable format: FP64 values hi + lo (exact)
    double *f = reinterpret_cast<double *>(p + sizeof(h));
    auto put = [&](const ulonglong2 *src, int n) {
        for (int i = 0; i < n; ++i) {
            const float2 v = se_df(src[i]);
            *f++ = static_cast<double>(v.x) + static_cast<double>(v.y);
        }
    };
    for (auto &nd : s->h_nodes) put(agg.data() + nd.aoff, nd.L);
    for (auto &ed : s->h_edges) {
        put(msg.data() + ed.mu, ed.Lu);
        put(msg.data() + ed.mv, ed.Lv);
    }
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_load_state(mplpp_solver *s, const void *buf, size_t size)
{
    if (!s || !buf) return MPLPP_E_INVALID;
    s->err.clear();
    size_t need = 0;
    mplpp_state_size(s, &need);
    if (size < need) return fail(s, MPLPP_E_INVALID, "state buffer too small");
    mplpp_state_header h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != 0x4D504C50u || h.version != 2 || h.shape_hash != s->shape_hash || h.n_unary != s->sum_unary ||
        h.n_msg != s->sum_msg)
        return fail(s, MPLPP_E_INVALID, "state does not match this solver's models");
    const ulonglong2 zero = se_make(make_float2(0.f, 0.f), 0u);
    std::vector<ulonglong2> agg(s->aggN, zero), msg(s->msgN, zero);
    const double *f = reinterpret_cast<const double *>(static_cast<const char *>(buf) + sizeof(h));
    // FP64 value -> hi = nearest float, lo = nearest float to the remainder
    auto get = [&](ulonglong2 *dst, int n) {
        for (int i = 0; i < n; ++i, ++f) {
            const float hi = static_cast<float>(*f);
            dst[i] = se_make(make_float2(hi, static_cast<float>(*f - static_cast<double>(hi))), 0u);
        }
    };
    for (auto &nd : s->h_nodes) {
        for (int i = 0; i < nd.L; ++i)
            if (!std::isfinite(f[i]) || std::fabs(f[i]) > 1e37) return fail(s, MPLPP_E_INVALID, "state values must be finite");
        get(agg.data() + nd.aoff, nd.L);
    }
    for (auto &ed : s->h_edges) {
        for (int i = 0; i < ed.Lu + ed.Lv; ++i)
            if (!std::isfinite(f[i]) || std::fabs(f[i]) > 1e37) return fail(s, MPLPP_E_INVALID, "state values must be finite");
        get(msg.data() + ed.mu, ed.Lu);
        get(msg.data() + ed.mv, ed.Lv);
    }
    CK(s, cudaMemcpyAsync(s->d_agg, agg.data(), s->aggN * sizeof(ulonglong2), cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaMemcpyAsync(s->d_msg, msg.data(), s->msgN * sizeof(ulonglong2), cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    s->iterations = h.iterations;
    s->history_valid = false;
    return MPLPP_OK;
}

static const char *mode_name(int mode)
{
    return mode == MPLPP_MODE_PERSISTENT   ? "persistent"
           : mode == MPLPP_MODE_WARP       ? "warp"
           : mode == MPLPP_MODE_STRUCTURED ? "structured"
           : mode == MPLPP_MODE_QUEUE      ? "queue"
           : mode == MPLPP_MODE_RESIDENT   ? "resident"
           : mode == MPLPP_MODE_STRUCTURED_QUEUE ? "structured_queue"
                                           : "looped";
}

// Measured choice of the mapping: every feasible (CTAs per edge, threads per
// CTA, driver) runs `iterations` iterations of the solver's own models from
// the same state, timed with CUDA events on the solver's stream; the fastest
// is kept.  Every mapping computes the same values bit for bit (minima are
// exact and every addition is per element), so only time differs.
extern "C" mplpp_status mplpp_autotune(mplpp_solver *s, int32_t iterations, char *report, size_t report_size)
{
    if (!s || iterations < 1) return MPLPP_E_INVALID;
    s->err.clear();
    if (report && report_size) report[0] = 0;
    if (s->EE == 0) return MPLPP_OK;
    if (s->opt.rule != kRuleH) {  // the M and U updates have one mapping
        if (report && report_size)
            std::snprintf(report, report_size,
                          "{\"best\": {\"cluster\": 1, \"threads\": 256, \"mode\": \"looped\", \"ms\": 0}, "
                          "\"candidates\": []}");
        return MPLPP_OK;
    }
    if (!s->d_save_agg) {
        CK(s, s->alloc(&s->d_save_agg, s->aggN));
        CK(s, s->alloc(&s->d_save_msg, s->msgN));
    }
    cudaStream_t st = s->stream;
    CK(s, cudaMemcpyAsync(s->d_save_agg, s->d_agg, sizeof(ulonglong2) * s->aggN, cudaMemcpyDeviceToDevice, st));
    CK(s, cudaMemcpyAsync(s->d_save_msg, s->d_msg, sizeof(ulonglong2) * s->msgN, cudaMemcpyDeviceToDevice, st));
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(s->d_agg, s->d_save_agg, sizeof(ulonglong2) * s->aggN, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_msg, s->d_save_msg, sizeof(ulonglong2) * s->msgN, cudaMemcpyDeviceToDevice, st);
        return e;
    };
    const int oldC = s->C, oldT = s->T, oldMode = s->mode;
    struct Cand {
        int C, T, mode;
        float ms;
    };
    std::vector<Cand> done;
    cudaEvent_t e0, e1;
    CK(s, cudaEventCreate(&e0));
    CK(s, cudaEventCreate(&e1));
    for (int mode : {MPLPP_MODE_PERSISTENT, MPLPP_MODE_LOOPED, MPLPP_MODE_WARP, MPLPP_MODE_STRUCTURED,
                     MPLPP_MODE_QUEUE, MPLPP_MODE_RESIDENT, MPLPP_MODE_STRUCTURED_QUEUE})
        for (int C : {1, 2, 3, 4, 5, 6, 8})
            for (int T : {128, 256, 512, 0}) {
                if (T == 0) {  // the exact fit of the register-resident passes, if another size
                    if (mode == MPLPP_MODE_WARP || mode == MPLPP_MODE_STRUCTURED || mode == MPLPP_MODE_STRUCTURED_QUEUE)
                        continue;
                    long long tile = 0, rows = 0;
                    int ldm = 4;
                    for (auto &ed : s->h_edges) {
                        const long long R = (ed.Lu + C - 1) / C;
                        tile = std::max(tile, R * ed.ld);
                        rows = std::max(rows, R);
                        ldm = std::max(ldm, ed.ld);
                    }
                    T = rr_fit_threads(static_cast<int>(rows), ldm >> 2,
                                       static_cast<int>(round4(std::max(4LL, tile))));
                    if (T == 0 || T == 128 || T == 256 || T == 512) continue;
                }
                if ((mode == MPLPP_MODE_STRUCTURED || mode == MPLPP_MODE_STRUCTURED_QUEUE) &&
                    (C != 1 || T != 256 || !s->all_structured))
                    continue;
                if (mode == MPLPP_MODE_QUEUE && (C != 1 || T != 128)) continue;
                if (mode == MPLPP_MODE_RESIDENT && (C != 1 || T != 128)) continue;
                const int Tm = mode == MPLPP_MODE_RESIDENT ? 0 : T;  // the resident driver sizes its blocks
                if (mode == MPLPP_MODE_WARP && C != 1) continue;  // one warp per edge
                if (mode == MPLPP_MODE_WARP && T == 512) T = 32;  // small blocks: shared memory per warp
                if (apply_mapping(s, C, Tm, mode) != MPLPP_OK) {
                    s->err.clear();
                    continue;
                }
                if (mode == MPLPP_MODE_RESIDENT) T = s->T;
                // timed over `iterations`; a run under 2 ms again over up to 16 times as
                // many, so that a driver's fixed start-up cost weighs as in a longer
                // run (candidates compare by the time of `iterations`)
                auto timed = [&](int its, float &ms) {
                    return restore() == cudaSuccess && run_plain(s, 1) == MPLPP_OK && restore() == cudaSuccess &&
                           cudaEventRecord(e0, st) == cudaSuccess && run_plain(s, its) == MPLPP_OK &&
                           cudaEventRecord(e1, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess &&
                           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && check_device_error(s) == MPLPP_OK;
                };
                float ms = 0.f;
                bool ok = timed(iterations, ms);
                if (ok && ms < 2.f) {
                    const int k = std::min(16, std::max(2, static_cast<int>(std::ceil(2.f / std::max(ms, 1e-3f)))));
                    float msk = 0.f;
                    ok = timed(iterations * k, msk);
                    ms = msk / static_cast<float>(k);
                }
                if (ok) done.push_back({C, T, mode, ms});
                s->err.clear();
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    Cand best = {oldC, oldT, oldMode, 0.f};
    if (!done.empty()) {
        best = done[0];
        for (auto &c : done)
            if (c.ms < best.ms) best = c;
    }
    mplpp_status stt = apply_mapping(s, best.C, best.T, best.mode);
    if (stt != MPLPP_OK) return stt;
    CK(s, restore());
    CK(s, cudaStreamSynchronize(st));
    if (report && report_size) {
        std::string r = "{\"iterations\": " + std::to_string(iterations) + ", \"best\": {\"cluster\": " +
                        std::to_string(best.C) + ", \"threads\": " + std::to_string(best.T) + ", \"mode\": \"" +
                        mode_name(best.mode) + "\", \"ms\": " +
                        std::to_string(best.ms) + "}, \"candidates\": [";
        for (size_t i = 0; i < done.size(); ++i)
            r += std::string(i ? ", " : "") + "[" + std::to_string(done[i].C) + ", " + std::to_string(done[i].T) +
                 ", \"" + mode_name(done[i].mode) + "\", " +
                 std::to_string(done[i].ms) + "]";
        r += "]}";
        std::snprintf(report, report_size, "%s", r.c_str());
    }
    return MPLPP_OK;
}

extern "C" mplpp_status mplpp_info(const mplpp_solver *s, mplpp_info_t *info)
{
    if (!s || !info) return MPLPP_E_INVALID;
    info->iterations = s->iterations;
    info->bytes_per_iteration = s->bytes_per_iter;
    info->edges = s->EE;
    info->phases = s->P;
    info->mode = s->mode;
    info->cluster = s->C;
    info->threads = s->T;
    info->grid = s->mode == MPLPP_MODE_PERSISTENT ? s->clusters * s->C
                 : s->mode == MPLPP_MODE_WARP     ? s->warp_blocks
                 : (s->mode == MPLPP_MODE_QUEUE || s->mode == MPLPP_MODE_STRUCTURED_QUEUE) ? s->queue_blocks
                 : s->mode == MPLPP_MODE_RESIDENT ? static_cast<int>(s->models.size())
                                                  : 0;
    info->launches_per_iteration = (s->mode == MPLPP_MODE_LOOPED || s->mode == MPLPP_MODE_STRUCTURED) ? s->P : 0;
    info->labeling_launches = (s->level_off.empty() ? 1 : static_cast<int>(s->level_off.size()) - 1) + 1;
    info->poller_warp = (s->mode == MPLPP_MODE_PERSISTENT && s->pw) ? 1 : 0;
    info->device_bytes = s->device_bytes;
    return MPLPP_OK;
}

extern "C" void mplpp_destroy(mplpp_solver *s)
{
    delete s;
}
