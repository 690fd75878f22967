// solver.h -- the opaque mplpp_solver (host bookkeeping + device buffers).
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mplpp.h"
#include "common.cuh"
#include "kernels.h"

namespace mplpp {
struct ModelHost {
    int n = 0, E = 0;
    int node_base = 0, edge_base = 0;
    long long unary_size = 0, pair_size = 0;
    bool structured = false;  // MPLPP_PAIR_TRUNC_*
    int pair_kind = 0;        // MPLPP_PAIR_*
    std::vector<int> L, eu, ev, off, order;
};
}  // namespace mplpp

struct mplpp_solver {
    ~mplpp_solver();
    template <typename Ty>
    cudaError_t alloc(Ty **p, size_t count);
    cudaError_t release(void *p);  // frees one of the solver's allocations (nullptr: nothing)

    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool stream_ok = false;
    mplpp_options opt = {};
    std::string err;
    std::vector<mplpp::ModelHost> models;

    int N = 0, EE = 0, P = 0;
    long long aggN = 0, msgN = 0, tabN = 0;
    long long sum_unary = 0, sum_pair = 0, sum_msg = 0;
    long long bytes_per_iter = 0;
    uint64_t shape_hash = 0;
    std::vector<mplpp::EdgeDesc> h_edges;
    std::vector<mplpp::NodeDesc> h_nodes;
    std::vector<int> phase_off, phase_edges;
    std::vector<int> in_off, in_edge, mnode_off, medge_off;
    std::vector<mplpp::InRec> in_rec;  // in_edge's records (rounding)
    std::vector<int> work_off;
    std::vector<mplpp::WorkItem> work;

    // mapping
    int mode = MPLPP_MODE_LOOPED;
    int C = 1, T = 256, tile_floats = 4, rmax = 4, ldmax = 4, max_phase = 1, clusters = 0, max_deg = 0;
    int lmax = 1;          // >= every label count and row stride (exact bound's buffers)
    int work_off_cap = 0;  // capacity of d_work_off
    bool rr = false;       // register-resident pass variant
    bool pw = false;       // with rr, persistent: a poller warp for node u (threads beyond the rows' warps)
    size_t smem_looped = 0, smem_persist = 0;
    int warp_blocks = 0, lw = 0, cap = 0;  // warp driver: blocks, per-warp vector and buffer capacity
    int queue_blocks = 0;                  // queue drivers: co-resident CTAs launched
    size_t smem_res = 0;                   // resident driver: shared memory per CTA
    mplpp::ResModel *d_res_models = nullptr;
    int *d_res_off = nullptr;
    int4 *d_res_desc = nullptr;
    size_t smem_queue = 0;
    unsigned long long *d_queue = nullptr; // queue driver: next item index
    size_t smem_warp = 0;
    size_t smem_rule = 0;  // M and U updates (rules.cu)
    bool all_structured = false;  // every model MPLPP_PAIR_TRUNC_LINEAR (and at least one edge)
    int struct_lmax = 0;          // structured kernel: vector capacity (multiple of 4)
    float2 *d_pair_param = nullptr;  // [EE] (w, tau) per edge (structured models)
    int *d_pair_kind = nullptr;      // [EE] MPLPP_PAIR_* per edge
    // rounding by levels (nodes whose earlier neighbours lie in earlier levels)
    std::vector<int> level_off;      // [n_levels + 1] into d_level_nodes; empty: sequential rounding
    std::vector<int> level_nodes;    // node ids by level
    int *d_level_nodes = nullptr;

    // device
    std::vector<void *> allocations;
    long long device_bytes = 0;  // sum of the sizes in `allocations`
    std::vector<size_t> allocation_bytes;
    mplpp::EdgeDesc *d_edges = nullptr;
    mplpp::NodeDesc *d_nodes = nullptr;
    float *d_tab = nullptr, *d_un0 = nullptr;
    ulonglong2 *d_agg = nullptr, *d_msg = nullptr;  // double-float state, versioned entries
    int *d_phase_edges = nullptr, *d_err = nullptr;
    int *d_work_off = nullptr;
    mplpp::WorkItem *d_work = nullptr;
    int *d_in_off = nullptr, *d_mnode_off = nullptr, *d_medge_off = nullptr;
    mplpp::InRec *d_in_rec = nullptr;
    double *d_emin = nullptr, *d_nmin = nullptr;
    double *d_out = nullptr, *d_energy = nullptr;
    int *d_labels = nullptr;

    // backward: FP64 replay buffers (allocated on first use)
    long long *d_rec_off = nullptr;        // per edge byte offset of its argmin records
    mplpp::EdgeDesc *d_sched_desc = nullptr;  // backward: every edge in schedule order
    long long *d_sched_rec_off = nullptr;     // ... and its record offset
    long long rec_stride = 0;
    std::vector<double *> ckpt64;    // FP64 (agg, msg) every record_every iterations of the replay
    bool history_valid = true;       // the state is T iterations from phi = 0 (false after load_state)
    double *d_agg64 = nullptr, *d_msg64 = nullptr;
    double *d_adj_agg = nullptr, *d_adj_msg = nullptr, *d_gtab = nullptr;
    unsigned char *d_rec = nullptr;  // argmin records of one segment, or of every iteration
    long long rec_slots = 0;         // iterations d_rec holds
    float *d_dD = nullptr;
    long long *d_pbase = nullptr, *d_ubase = nullptr;  // per-model offsets of the caller's layouts
    ulonglong2 *d_save_agg = nullptr, *d_save_msg = nullptr;
    float *d_stage_u = nullptr, *d_stage_p = nullptr;  // update_costs: host inputs staged here  // autotuner: state kept across candidates

    long long iterations = 0;
    long long launches = 0;

    cudaGraphExec_t g_looped = nullptr;
    cudaGraphExec_t g_persist = nullptr;
    int g_persist_iters = -1;
};

template <typename Ty>
cudaError_t mplpp_solver::alloc(Ty **p, size_t count)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(Ty));
    if (e == cudaSuccess) {
        allocations.push_back(*p);
        allocation_bytes.push_back((count ? count : 1) * sizeof(Ty));
        device_bytes += static_cast<long long>(allocation_bytes.back());
    }
    return e;
}

inline cudaError_t mplpp_solver::release(void *p)
{
    if (!p) return cudaSuccess;
    for (size_t i = 0; i < allocations.size(); ++i)
        if (allocations[i] == p) {
            device_bytes -= static_cast<long long>(allocation_bytes[i]);
            allocations.erase(allocations.begin() + static_cast<long>(i));
            allocation_bytes.erase(allocation_bytes.begin() + static_cast<long>(i));
            return cudaFree(p);
        }
    return cudaSuccess;
}

// api.cu
cudaError_t enqueue_looped_iteration(mplpp_solver *s, cudaStream_t st);
cudaError_t enqueue_persistent(mplpp_solver *s, cudaStream_t st, int iterations);
