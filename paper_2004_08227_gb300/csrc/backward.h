// backward.h -- recorded runs and the reverse sweep (gradient of the dual bound).
#pragma once
#include <cuda_runtime.h>

#include "../../include/mplpp.h"
#include "common.cuh"

struct mplpp_solver;

namespace mplpp {

struct BwParams {
    const EdgeDesc *edges;
    const NodeDesc *nodes;
    const float *tab;
    const unsigned char *rec;   // argmin records of one iteration (t1, s2, t3 as uint16 per edge)
    const long long *rec_off;   // per edge byte offset within an iteration's records
    float *adj_agg;             // adjoint of agg (agg layout)
    float *adj_msg;             // adjoint of msg (msg layout)
    float *gtab;                // adjoint of the original tables (tab layout)
    int lmax;                   // largest label count
};

cudaError_t launch_bw_init(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes, const float *tab,
                           const float *agg, const float *msg, const float *dD, float *adj_agg, float *adj_msg,
                           float *gtab, cudaStream_t st);
cudaError_t launch_bw_phase(const BwParams &p, const int *items, int n_items, cudaStream_t st);
cudaError_t launch_unpack_grad(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                               const long long *pair_base, const long long *unary_base, const float *gtab,
                               const float *adj_agg, float *grad_pair, float *grad_un, cudaStream_t st);

}  // namespace mplpp

mplpp_status run_recorded(mplpp_solver *s, int iterations);
