/*
 * mplpp.h -- C ABI of the GB300 (sm_103a) MPLP++ solver.
 *
 * MPLP++ (Tourani, Shekhovtsov, Rother, Savchynskyy) maximizes the dual lower
 * bound D(phi) of MAP inference in a discrete pairwise graphical model
 * (Sec. 3, eqs. energy-min, reparametrization, LP-lower-bound) by block
 * coordinate ascent over the messages phi_{u<->v} of one edge at a time, with
 * the Handshake update (Sec. 4, eq. (H), three-minimization form).  Edges of
 * one matching of an edge schedule (Sec. 6, Alg. 1) are independent and are
 * updated in parallel; matchings are processed in order.
 *
 * Conventions for every entry point:
 *  - Nodes are 0..n-1; node u has L_u >= 1 labels (0-based).  An edge (u, v)
 *    has u < v (Sec. 3, Notation); its pairwise table is row-major, L_u rows
 *    (labels of u) by L_v columns (labels of v).
 *  - `unary` concatenates the node vectors in node order; `pairwise`
 *    concatenates the tables in edge order.  Offsets are implied by the label
 *    counts.  Costs must be finite.
 *  - Host arrays passed to a call are read during the call only (copied); the
 *    caller keeps ownership.  Device arrays (options.inputs_on_device) are
 *    read during mplpp_create only, except that mplpp_backward writes the
 *    gradients to caller-owned memory of the same kind.
 *  - Every call returns an mplpp_status; nothing throws across the ABI.  On
 *    failure the solver keeps a message readable with mplpp_last_error.
 *  - Calls enqueue work on the CUDA stream given at creation.  Calls that
 *    return host data (bound, labeling, save_state, backward) synchronize that
 *    stream and report device-side errors (a timed-out wait, non-finite
 *    values) through their status.
 *  - A solver is not thread-safe; distinct solvers are independent.
 */
#ifndef MPLPP_H
#define MPLPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mplpp_solver mplpp_solver;

typedef enum {
    MPLPP_OK = 0,
    MPLPP_E_INVALID = -1,     /* bad argument: sizes, edge order, duplicate edge, bad schedule */
    MPLPP_E_NOMEM = -2,       /* host or device allocation failed                              */
    MPLPP_E_CUDA = -3,        /* a CUDA runtime call failed (message has the CUDA error)       */
    MPLPP_E_TIMEOUT = -4,     /* a device-side wait exceeded options.spin_limit polls          */
    MPLPP_E_NONFINITE = -5,   /* a result is NaN or infinite                                   */
    MPLPP_E_STATE = -6,       /* call not valid in the current state (e.g. backward w/o record) */
    MPLPP_E_UNSUPPORTED = -7  /* a shape beyond a compiled limit, or a driver / update / cost
                                 combination not built (the message says which)               */
} mplpp_status;

/* Edge schedule kinds (Sec. 6, Alg. 1). */
enum {
    MPLPP_SCHED_ROUND_ROBIN = 0,  /* complete graph K_n: circle-method 1-factorization            */
    MPLPP_SCHED_GREEDY_COLOR = 1, /* greedy edge colouring, edges in (u,v) order, smallest colour */
    MPLPP_SCHED_ALG1 = 2,         /* Alg. 1: repeated greedy maximal matching of remaining edges  */
    MPLPP_SCHED_USER = 3          /* caller supplies matching_off / edge_order                    */
};

/* How mplpp_run drives the matchings. */
enum {
    MPLPP_MODE_AUTO = 0,       /* STRUCTURED when every model qualifies, else persistent when
                                  the device allows it, else looped                            */
    MPLPP_MODE_LOOPED = 1,     /* one kernel launch per matching (launch boundary = barrier)  */
    MPLPP_MODE_PERSISTENT = 2, /* one launch for all iterations; every state entry carries the
                                  update count that wrote it, which orders the matchings on
                                  the device (a reader polls until the count it needs)        */
    MPLPP_MODE_WARP = 3,       /* as PERSISTENT with one warp per edge instead of a cluster of
                                  CTAs per edge (for many small tables: every label count
                                  <= 128); options.cluster is ignored                          */
    MPLPP_MODE_STRUCTURED = 4, /* every model MPLPP_PAIR_TRUNC_*, rule H, label counts
                                  <= 256: one launch per matching, one warp per edge, no
                                  table reads (see MPLPP_PAIR_*)                               */
    MPLPP_MODE_QUEUE = 5,      /* one launch for all iterations; one CTA per edge at a time,
                                  every CTA taking the next edge from one queue of all models'
                                  updates (each model in schedule order, the models interleaved
                                  by their progress); tables read from memory by every pass
                                  instead of staged, so many CTAs share an SM (for many small
                                  models); options.cluster is ignored                        */
    MPLPP_MODE_RESIDENT = 6,   /* one launch for all iterations; one CTA per model keeps the
                                  model's reparametrization in shared memory and separates
                                  its matchings by a block barrier (many small models: every
                                  label count <= 32, the state of the largest model within
                                  shared memory); options.cluster is ignored                  */
    MPLPP_MODE_STRUCTURED_QUEUE = 7 /* the updates of MPLPP_MODE_STRUCTURED in one launch for
                                  all iterations: every warp takes the next edge from the
                                  queue of MPLPP_MODE_QUEUE and waits for its node entries by
                                  their update counts (as MPLPP_MODE_PERSISTENT)             */
};

/* How a model's pairwise costs are given.  TRUNC_LINEAR: theta_uv(s,t) =
 * w_uv * min(|s - t|, tau_uv) (labels on a line; Potts is tau = 1);
 * TRUNC_QUAD: w_uv * min((s - t)^2, tau_uv).  In both the FP32 product is
 * rounded once, as if the caller had passed those tables.  The solver
 * materializes the tables on the device (bound, rounding, the dense drivers)
 * and, in MPLPP_MODE_STRUCTURED, runs the Handshake update without reading
 * them: O(L) minimizations for truncated-linear costs, a window of the labels
 * within the truncation around each label for truncated-quadratic ones. */
enum {
    MPLPP_PAIR_DENSE = 0,
    MPLPP_PAIR_TRUNC_LINEAR = 1,
    MPLPP_PAIR_TRUNC_QUAD = 2
};

/* Which block-coordinate-ascent update mplpp_run applies to each edge (Sec. 4;
 * g = theta_uv + theta_u + theta_v of the current reparametrization).  H is
 * the solver's purpose; M and U are there for the paper's comparison (Prop. 2:
 * after one update of the same edge D_H >= D_M >= D_U; Thm. 2: the same for
 * one iteration from equal states).  M and U run in the looped driver only
 * (MPLPP_MODE_AUTO or _LOOPED; persistent, warp or structured mode:
 * MPLPP_E_UNSUPPORTED), one CTA per edge, and have no backward (record_every
 * must be 0). */
enum {
    MPLPP_RULE_H = 0, /* eq. (H), the Handshake (MPLP++) update: three minimizations     */
    MPLPP_RULE_M = 1, /* eq. (M), the MPLP update: theta_u := 1/2 min_t g(.,t),
                         theta_v := 1/2 min_s g(s,.)                                     */
    MPLPP_RULE_U = 2  /* eq. (U), the uniform update: theta_u := theta_v := 1/2 min g    */
};

typedef struct {
    int32_t n_nodes;
    int32_t n_edges;
    const int32_t *labels;       /* [n_nodes] host, L_u >= 1                                   */
    const int32_t *edge_u;       /* [n_edges] host, edge_u[e] < edge_v[e], no duplicate pairs  */
    const int32_t *edge_v;       /* [n_edges] host                                             */
    const float *unary;          /* [sum_u L_u]          host, or device if inputs_on_device   */
    const float *pairwise;       /* [sum_e L_u * L_v]    host, or device if inputs_on_device   */
    int32_t schedule_kind;       /* MPLPP_SCHED_*                                              */
    int32_t n_matchings;         /* MPLPP_SCHED_USER only                                      */
    const int32_t *matching_off; /* MPLPP_SCHED_USER only: [n_matchings + 1] host              */
    const int32_t *edge_order;   /* MPLPP_SCHED_USER only: [n_edges] host, edge ids            */
    int32_t pair_kind;           /* MPLPP_PAIR_*; 0 = dense tables in `pairwise`                */
    int32_t reserved;            /* 0                                                          */
    const float *pair_param;     /* MPLPP_PAIR_TRUNC_*: [n_edges][2] = (w, tau) per
                                    edge, w >= 0, tau >= 0, finite (host, or device if
                                    inputs_on_device); `pairwise` must then be NULL            */
} mplpp_model;

typedef struct {
    int32_t mode;             /* MPLPP_MODE_*                                                  */
    int32_t use_graph;        /* nonzero: replay the launches of an iteration from a CUDA graph */
    int32_t inputs_on_device; /* nonzero: model.unary / model.pairwise are device pointers and
                                 mplpp_backward writes device gradients                         */
    int32_t record_every;     /* > 0: enables mplpp_backward, which replays the run in FP64:
                                 recording the argmins of every iteration in one replay when
                                 those records fit 1 GiB, else with a state checkpoint every k
                                 iterations (memory ~ T/k states) and a second replay of each
                                 segment; 0: backward disabled.  Rule H and dense costs only. */
    int32_t cluster;          /* CTAs sharing one edge (1..8); 0 = chosen from the shapes      */
    int32_t threads;          /* threads per CTA: 0 = chosen from the shapes, else a multiple
                                 of 32 in 64..512 (32..512 for MPLPP_MODE_WARP)                */
    int32_t test_unreachable_wait; /* testing only (0 otherwise): in the persistent driver the
                                 first edge of the first worker waits for one node update more
                                 than will ever happen, so the bounded wait must run out and the
                                 run must end with MPLPP_E_TIMEOUT instead of hanging            */
    int32_t rule;             /* MPLPP_RULE_* (0 = the Handshake update)                        */
    int64_t spin_limit;       /* polls before a device-side wait gives up with MPLPP_E_TIMEOUT */
    int32_t test_backward;    /* testing only (0 otherwise), bit flags for mplpp_backward:
                                 1 = replay every minimization in FP64 instead of screening
                                 it in FP32 first; 2 = checkpoints and a second replay per
                                 segment even where every record fits (both paths give the
                                 same argmins and gradient bit for bit)                       */
    int32_t reserved;         /* 0                                                             */
} mplpp_options;

/* Fills *opt with defaults: AUTO mode, graphs on, host inputs, no record,
 * automatic mapping, spin_limit = 2^26 (well above any legitimate wait). */
void mplpp_options_default(mplpp_options *opt);

/* Builds an edge schedule (Sec. 6, Alg. 1) for one graph.
 *   kind: MPLPP_SCHED_ROUND_ROBIN (needs the complete graph), _GREEDY_COLOR or _ALG1.
 *   matching_off: out, capacity n_edges + 1 (n_edges + 1 >= 1); edge_order: out, [n_edges].
 *   *n_matchings: out.  Matching k is edge_order[matching_off[k] .. matching_off[k+1]);
 *   no two of its edges share a node, and every edge appears once.
 * Host only; MPLPP_E_INVALID on a malformed graph. */
mplpp_status mplpp_schedule(int32_t kind, int32_t n_nodes, int32_t n_edges, const int32_t *edge_u,
                            const int32_t *edge_v, int32_t *matching_off, int32_t *edge_order,
                            int32_t *n_matchings);

/* Creates a solver for n_models independent models, solved together (the
 * batched form: matching k of every model runs in the same phase).  Copies the
 * costs to the device into the solver's layout and sets phi = 0 (the
 * reparametrized costs start as the given ones).  `stream` is a cudaStream_t
 * (NULL = legacy default stream) on the current device.  opt may be NULL
 * (defaults).  On success *out owns all device memory until mplpp_destroy. */
mplpp_status mplpp_create(const mplpp_model *models, int32_t n_models, const mplpp_options *opt,
                          void *stream, mplpp_solver **out);

/* Runs `iterations` >= 0 BCA iterations (Sec. 5: every edge updated once, in
 * schedule order) with the Handshake update, continuing from the current
 * state.  Asynchronous on the solver's stream. */
mplpp_status mplpp_run(mplpp_solver *s, int32_t iterations);

/* Dual bound D (eq. LP-lower-bound) of the current reparametrization, one per
 * model, into host out[n_models].  exact != 0: node minima plus the minimum of
 * every reparametrized pairwise table (reads all tables); exact == 0: node
 * minima only, which equals D when every table's minimum is 0, as it is after
 * a full iteration (Def. 1 normalization).  FP64 throughout (the state is FP64,
 * the tables FP32).
 * Synchronizes. */
mplpp_status mplpp_bound(mplpp_solver *s, double *out, int32_t exact);

/* Primal rounding (Sec. 4, Primal Rounding) of the current reparametrization:
 * nodes in increasing order, x_u = argmin_s [theta^phi_u(s) + sum over earlier
 * neighbours v (increasing v) of theta^phi_vu(x_v, s)], FP64 sums, lowest index
 * on ties.  labels: host [sum of n_nodes over models], model after model;
 * energy: host [n_models] (may be NULL), E(x | original costs) in FP64
 * (eq. energy-min).  Synchronizes. */
mplpp_status mplpp_labeling(mplpp_solver *s, int32_t *labels, double *energy);

/* Gradient of sum_m dD[m] * D_m, where D_m is model m's exact dual bound after
 * the iterations run since the last reset, with respect to the original unary
 * and pairwise costs.  D is piecewise linear; the gradient is that of the
 * linear piece selected by the argmins (lowest index on ties) of the same
 * iterations replayed in FP64 -- the FP32 run can sit on a different piece
 * near ties, the FP64 replay follows the exact-arithmetic one.
 * Requires options.record_every > 0 and a run that started from phi = 0
 * (creation or mplpp_reset, no mplpp_load_state since).
 * dD: host [n_models]; grad_unary [sum L], grad_pairwise [sum L_u L_v] in the
 * input layout, host or device as options.inputs_on_device says.
 * Synchronizes. */
mplpp_status mplpp_backward(mplpp_solver *s, const float *dD, float *grad_unary,
                            float *grad_pairwise);

/* Resets phi = 0 and the iteration count. */
mplpp_status mplpp_reset(mplpp_solver *s);

/* Replaces the costs of every model by new ones of the same shapes (same
 * labels, edges and schedules; eq. energy-min's theta) and resets phi = 0 and
 * the iteration count, as a new solver with these costs would start: the
 * device layout, mapping, work lists and captured graphs are kept, so a loop
 * over many cost sets (learning, serving) pays only the copy and the packing.
 *   unary[m], pairwise[m]: model m's costs in the layout of mplpp_model, host
 *   pointers or device pointers if options.inputs_on_device.  Host arrays in
 *   pinned, mapped memory (cudaHostAlloc) are read in place by the packing
 *   kernel; other host arrays are copied through a device staging buffer
 *   allocated on the first call and kept.  The arrays must stay unchanged
 *   until the call returns.
 * Non-finite costs: MPLPP_E_INVALID (the state is then reset but the costs
 * are undefined until a successful call).  Models with structured costs
 * (MPLPP_PAIR_TRUNC_LINEAR or MPLPP_PAIR_TRUNC_QUAD): MPLPP_E_UNSUPPORTED
 * (create a new solver).  Synchronizes. */
mplpp_status mplpp_update_costs(mplpp_solver *s, const float *const *unary, const float *const *pairwise);

/* Solver state (the reparametrization) in a portable host format:
 *   header (see mplpp_state_header), then FP64 theta^phi_u for every node
 *   ([sum L], model after model, node order), then per edge phi_{v->u} [L_u]
 *   followed by phi_{u->v} [L_v] (edge order).  theta^phi_uv is implied:
 *   theta_uv(s,t) - phi_{v->u}(s) - phi_{u->v}(t) (eq. reparametrization).
 * mplpp_state_size gives the byte count; save/load need a buffer of that size.
 * Loading checks the header against the solver's shapes (MPLPP_E_INVALID). */
typedef struct {
    uint32_t magic;       /* 0x4D504C50 "MPLP" */
    uint32_t version;     /* 2 (FP64 values) */
    uint64_t shape_hash;  /* FNV-1a of labels, edges and schedules of all models */
    int64_t iterations;   /* iterations run since the last reset */
    int64_t n_unary;      /* sum L over all models */
    int64_t n_msg;        /* sum (L_u + L_v) over all edges */
} mplpp_state_header;
mplpp_status mplpp_state_size(const mplpp_solver *s, size_t *bytes);
mplpp_status mplpp_save_state(mplpp_solver *s, void *buf, size_t size);
mplpp_status mplpp_load_state(mplpp_solver *s, const void *buf, size_t size);

/* Facts about a solver, for benchmarks and tests. */
typedef struct {
    int64_t iterations;         /* iterations run since the last reset                        */
    int64_t bytes_per_iteration;/* HBM bytes of one iteration in this layout: sum_e 4 L_u L_v
                                   + 32 (L_u + L_v) (tables once; double-float agg and msg
                                   values of both ends read and written)                      */
    int64_t edges;              /* total edges over all models                                */
    int32_t phases;             /* matchings per iteration (max over models)                 */
    int32_t mode;               /* MPLPP_MODE_LOOPED or _PERSISTENT actually used             */
    int32_t cluster;            /* CTAs per edge                                              */
    int32_t threads;            /* threads per CTA                                            */
    int32_t grid;               /* persistent mode: CTAs launched                             */
    int32_t launches_per_iteration; /* kernel launches one iteration takes (looped: phases)   */
    int32_t labeling_launches;  /* kernel launches of one mplpp_labeling: the rounding (one,
                                   or one per level of the rounding order) and the energy      */
    int32_t poller_warp;        /* 1: the persistent driver's CTAs have one warp beyond those
                                   holding table rows, which fetches node u's vector while
                                   the others start on node v's (threads permitting)          */
    int64_t device_bytes;       /* device memory the solver holds now (its allocations,
                                   including the backward's replay buffers once allocated)   */
} mplpp_info_t;
mplpp_status mplpp_info(const mplpp_solver *s, mplpp_info_t *info);

/* Waits for the solver's stream and reports device-side errors. */
mplpp_status mplpp_sync(mplpp_solver *s);

/* Self-measured choice of the mapping (not in the paper): runs `iterations`
 * iterations of the solver's own models under every feasible combination of
 * CTAs per edge (1..8), threads per CTA (128, 256, 512 and the exact fit of
 * the register-resident passes) and driver (persistent, looped, warp, queue,
 * resident, structured, structured-queue), timed with CUDA events on the
 * solver's stream, and keeps the fastest.  A candidate whose run takes under
 * 2 ms is timed again over up to 16 times as many iterations and reported per
 * `iterations`, so that fixed start-up costs weigh as in a longer run.  All
 * mappings compute bit-identical results; the state before the call is
 * restored afterwards.  report (may be NULL): host buffer receiving a JSON
 * summary (best mapping and every candidate's time in ms).  Synchronizes. */
mplpp_status mplpp_autotune(mplpp_solver *s, int32_t iterations, char *report, size_t report_size);

/* Dual bound of one model's reparametrized costs without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- code that owns a fixed device arena
 * and allows no allocation after start-up, real-time loops that cannot pay an
 * allocation's latency or implicit synchronization, plugins whose host
 * runtime must see every device byte.  It computes what mplpp_bound(exact = 1)
 * computes, from buffers the caller owns:
 *   labels [n_nodes], edge_u, edge_v [n_edges]   int32, device (L_u in 1..65535, u < v)
 *   pairwise [sum L_u L_v]  FP32, device, the ORIGINAL tables, caller layout
 *   agg [sum L_u]           FP32, device, theta^phi_u per node (state layout)
 *   msg [sum (L_u + L_v)]   FP32, device, phi_{v->u} then phi_{u->v} per edge
 *                           (state layout, as in mplpp_save_state)
 *   out [1]                 FP64, device, receives D
 * Working memory (offsets, per-node and per-edge minima) is one file-scope
 * device array of MPLPP_NOALLOC_SCRATCH_BYTES (about 5.8 MB) that every GPU
 * loading the library holds until the process exits; hence the size limits
 * below, beyond which the call returns MPLPP_E_UNSUPPORTED.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current) and keeps it for that device's context (a call after
 * the context was destroyed and recreated, e.g. by cudaDeviceReset, looks it
 * up again).  All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads)
 * race on it.  Work runs on `stream` (a cudaStream_t, NULL = legacy default);
 * every call then waits for that stream to finish, to read back the check of
 * the labels and edges (MPLPP_E_INVALID, with out left untouched).  The call
 * trusts that the array lengths above match labels, edge_u and edge_v.  Calls
 * no cudaMalloc, cudaFree or allocating library routine.  Message of a
 * failure: mplpp_noalloc_last_error(). */
#define MPLPP_NOALLOC_MAX_NODES 65536
#define MPLPP_NOALLOC_MAX_EDGES 262144
#define MPLPP_NOALLOC_SCRATCH_BYTES 6030336
mplpp_status mplpp_bound_noalloc(int32_t n_nodes, int32_t n_edges, const int32_t *labels, const int32_t *edge_u,
                                 const int32_t *edge_v, const float *pairwise, const float *agg, const float *msg,
                                 double *out, void *stream);
const char *mplpp_noalloc_last_error(void);

/* Message of the last failed call on this solver ("" if none).  Valid until the
 * next call on the solver.  s may be NULL: then the last mplpp_create failure. */
const char *mplpp_last_error(const mplpp_solver *s);

/* Frees the solver and its device memory (after synchronizing its stream). */
void mplpp_destroy(mplpp_solver *s);

#ifdef __cplusplus
}
#endif
#endif /* MPLPP_H */
