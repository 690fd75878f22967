// kernels.h -- host-visible launch interfaces of the solver's kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mplpp {

// Arguments of the Handshake kernels (one struct, passed by value).
struct HsParams {
    const EdgeDesc *edges;
    const float *tab;
    ulonglong2 *agg;         // reparametrized unaries (agg layout, versioned double-float entries)
    ulonglong2 *msg;         // messages (msg layout, versioned double-float entries)
    const int *items;        // looped: edge ids of the phase being launched
    const int *work_off;     // persistent: [clusters + 1] offsets into work
    const WorkItem *work;    // persistent: per-cluster item lists (one iteration)
    int *err;                // device error word (ERR_*)
    long long spin_limit;    // polls before a wait gives up
    int iterations;          // persistent: iterations to run
    int test_wait;           // testing: first item of worker 0 waits for an update that never comes
    int rr;                  // launch the variant with register-resident passes
    int pw;                  // persistent, with rr: the last warp of a CTA polls node u (no rows)
    int C;                   // CTAs per edge (cluster size)
    int tile_floats;         // capacity of one table buffer (floats)
    int workers;             // warp driver: number of warp workers (lists in work_off / work)
    int lw;                  // warp driver: per-warp vector capacity (entries, multiple of 4)
    int cap;                 // warp driver: floats per table buffer (>= 32 rows of any table)
    int rmax;                // capacity of row vectors (floats, multiple of 4)
    int ldmax;               // capacity of column vectors (floats, multiple of 4)
    unsigned long long *queue;  // queue driver: next item index (0 before the launch)
    long long queue_items;      // queue driver: items per iteration (the list in work)
};

// Update counts an item expects of its inputs (persistent drivers): node u's
// and node v's entries carry u / v (earlier updates of the node in this
// launch), the edge's messages carry e (earlier updates of the edge); the
// item writes u + 1, v + 1, e + 1.  `bump` is added to what the u side waits
// for (testing the bounded wait: an update that never comes).
struct Versions {
    unsigned u, v, e, bump;
};

size_t hs_smem_bytes(int nbuf, int tile_floats, int rmax, int ldmax, int threads, int C);

// warp.cu: one warp per edge (persistent).  Shared memory per warp for vector
// capacity lw and table buffers of cap floats: the work record, two
// mbarriers, two buffers, double-float uh and vh, FP32 w1, alpha, beta.
__host__ __device__ inline size_t hs_warp_bytes_per_warp(int lw, int cap)
{
    return sizeof(WorkItem) + 16 + 8 * static_cast<size_t>(cap) + 28 * static_cast<size_t>(lw);
}
constexpr int kWarpMaxL = 128;  // largest label count (and row stride) the warp driver takes
cudaError_t hs_warp_prepare(size_t smem_bytes);
int hs_warp_max_blocks(int threads, size_t smem_bytes);  // co-resident blocks on the device
cudaError_t hs_launch_warp(const HsParams &p, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t hs_prepare(size_t smem_bytes);
cudaError_t hs_launch_looped(const HsParams &p, int n_items, int threads, size_t smem, cudaStream_t st);
cudaError_t hs_launch_persistent(const HsParams &p, int clusters, int threads, size_t smem, cudaStream_t st);
int hs_max_active_clusters(int C, int threads, size_t smem, bool rr);
bool hs_rr_fits(int nr_max, int Q_max, int threads, int tile_floats);
bool hs_pw_fits(int nr_max, int Q_max, int threads, int tile_floats);  // rr_fits with a poller warp
// queue driver (one launch, a global item queue, tables streamed from memory)
cudaError_t hs_launch_queue(const HsParams &p, int blocks, int threads, size_t smem, cudaStream_t st);
int hs_queue_max_blocks(int threads, size_t smem);  // co-resident blocks on the device

// resident.cu: one CTA per model, the model's state in shared memory for all
// iterations, a block barrier between matchings (label counts <= kResMaxL);
// groups of res_lanes(lmax) lanes update one edge each.
constexpr int kResMaxL = 32;
constexpr int kResWarpBytes = 2 * 32 * 8 + 3 * 32 * 4;  // per-warp vectors (7 words per lane)
__host__ __device__ constexpr int res_lanes(int lmax)
{
    return lmax <= 8 ? 8 : (lmax <= 16 ? 16 : 32);
}
struct ResModel {
    long long agg_base, agg_n;  // the model's entries in agg
    long long msg_base, msg_n;  // ... and in msg
    long long tab_base, tab_n;  // ... and its tables in tab (floats)
    int sched;                  // offset of its matching offsets in sched_off
    int P;                      // its matchings
};
// A scheduled edge of the resident driver, relative to its model (16 bytes,
// one load): x = first table entry (floats after the model's first table),
// y = node u's | node v's first agg entry << 16, z = phi_{v->u}'s | phi_{u->v}'s
// first msg entry << 16 (entries after the model's first), w = L_u | L_v << 8 |
// ld << 16.
struct ResParams {
    const float *tab;
    ulonglong2 *agg;
    ulonglong2 *msg;
    const ResModel *models;
    const int *sched_off;     // per model P + 1 offsets into sched_desc
    const int4 *sched_desc;   // every model's edges in schedule order, as above
    int iterations;
};
cudaError_t res_prepare(size_t smem);
cudaError_t launch_resident(const ResParams &p, int n_models, int threads, size_t smem, int lmax, cudaStream_t st);

// rules.cu: the MPLP (eq. (M)) and uniform (eq. (U)) updates of Sec. 4, one
// CTA per edge, one launch per matching.
constexpr int kRuleH = 0, kRuleM = 1, kRuleU = 2;  // the MPLPP_RULE_* values
struct RuleParams {
    const EdgeDesc *edges;
    const int *items;  // edge ids of the matching being launched
    const float *tab;
    ulonglong2 *agg;
    ulonglong2 *msg;
};
size_t rule_smem_bytes(int lumax, int ldmax);  // lumax >= every L_u, ldmax >= every row stride
cudaError_t rule_prepare(size_t smem_bytes);
cudaError_t launch_rule(const RuleParams &p, int rule, int n_items, size_t smem, cudaStream_t st);

// structured.cu: the Handshake update for truncated-linear costs
// w min(|s - t|, tau) in O(L) per minimization and for truncated-quadratic
// costs w min((s - t)^2, tau) over a window, one warp per edge, looped.
constexpr int kStructMaxL = 256;  // largest label count the structured kernel takes
struct StructParams {
    const EdgeDesc *edges;
    const int *items;      // edge ids of the matching being launched
    int n_items;
    int lmax;              // >= every label count of the solver, multiple of 4
    const float2 *param;   // [edges] (w, tau) per edge id
    const int *kind;       // [edges] MPLPP_PAIR_* per edge id
    ulonglong2 *agg;
    ulonglong2 *msg;
    // persistent form (struct_queue_kernel): every warp takes the next item of
    // the queue driver's list (work, queue_items per iteration); versioned waits
    const WorkItem *work;
    unsigned long long *queue;
    long long queue_items;
    int iterations;
    int test_wait;
    int *err;
    long long spin_limit;
};
__host__ __device__ inline size_t struct_bytes_per_warp(int lmax)
{
    return 40 * static_cast<size_t>(lmax);  // uh, vh double-float; h, m FP32; prefix and suffix (value, index)
}
cudaError_t struct_prepare(int lmax);
cudaError_t launch_struct(const StructParams &p, cudaStream_t st);
cudaError_t launch_struct_queue(const StructParams &p, int blocks, cudaStream_t st);
int struct_queue_max_blocks(int lmax);  // co-resident blocks of 8 warps
// tables of n consecutive edges from their (w, tau) and kind: w min(|s - t|,
// tau) or w min((s - t)^2, tau), rows padded with +inf; a negative or
// non-finite parameter sets ERR_NONFINITE
cudaError_t launch_materialize(const EdgeDesc *edges, const float2 *param, const int *kind, int n, float *tab,
                               int *err, cudaStream_t st);
constexpr int kPairLinear = 1, kPairQuad = 2;  // the MPLPP_PAIR_TRUNC_* values

// dual.cu
cudaError_t launch_pack(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                        const float *unary_src, const float *pair_src, float *tab, float *un0, ulonglong2 *agg,
                        int *err, cudaStream_t st);
cudaError_t launch_bound(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                         const float *tab, const ulonglong2 *agg, const ulonglong2 *msg, double *emin, double *nmin,
                         const int *model_node_off, const int *model_edge_off, int n_models, int exact,
                         int lmax, double *out, cudaStream_t st);  // lmax >= every label count and row stride
// Sequential rounding (one block per model walking its nodes in order), or
// with n_levels > 0 one launch per level of level_nodes (device) delimited by
// level_off (host, [n_levels + 1]): the nodes of a level have all earlier
// neighbours in earlier levels.  Then the energies.
cudaError_t launch_round(const EdgeDesc *edges, const NodeDesc *nodes, const int *in_off, const InRec *in_rec,
                         const int *model_node_off, const int *model_edge_off, int n_models, const float *tab,
                         const ulonglong2 *agg, const ulonglong2 *msg, const float *un0, int *labels, double *energy,
                         int *err, const int *level_nodes, const int *level_off, int n_levels, cudaStream_t st);
cudaError_t launch_init_state(const float *un0, ulonglong2 *agg, long long n_agg, ulonglong2 *msg, long long n_msg,
                              cudaStream_t st);
// Sets the version of every state entry to 0, keeping the values.
cudaError_t launch_restamp(ulonglong2 *agg, long long n_agg, ulonglong2 *msg, long long n_msg, cudaStream_t st);

}  // namespace mplpp
