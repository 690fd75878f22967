// backward.h -- FP64 replay of the iterations and the reverse sweep (gradient
// of the dual bound with respect to the original costs).
#pragma once
#include <cstddef>

#include <cuda_runtime.h>

#include "mplpp.h"
#include "common.cuh"

namespace mplpp {

// record.cu
size_t rec64_smem_bytes(int lmax);
cudaError_t launch_rec64_phase(const EdgeDesc *edges, const int *items, int n_items, const float *tab, double *agg,
                               double *msg, unsigned char *rec, const long long *rec_off, int lmax, cudaStream_t st);
cudaError_t launch_widen(const float *src, double *dst, long long n, cudaStream_t st);
// the same update with an FP32 screen and FP64 only for the candidates (bit for
// bit the same minima and argmins); tab_floats >= L_u * (ld | 1) of every edge;
// descs and rec_off: the matching's edges and record offsets in schedule order
size_t rec_screen_smem_bytes(int lmax, long long tab_floats);
cudaError_t launch_rec_screen_phase(const EdgeDesc *descs, int n_items, const float *tab,
                                    double *agg, double *msg, unsigned char *rec, const long long *rec_off, int lmax,
                                    long long tab_floats, cudaStream_t st);

// backward.cu
struct BwParams {
    const EdgeDesc *descs;      // every scheduled edge, in schedule order
    const unsigned char *rec;   // argmin records of one iteration (t1, s2, t3 as uint16 per edge)
    const long long *rec_off;   // per scheduled edge (schedule order) byte offset within an iteration's records
    double *adj_agg;            // adjoint of agg (agg layout)
    double *adj_msg;            // adjoint of msg (msg layout)
    double *gtab;               // adjoint of the original tables (tab layout)
    int lmax;                   // largest label count
};

cudaError_t launch_bw_init(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes, const float *tab,
                           const double *agg, const double *msg, const float *dD, double *adj_agg, double *adj_msg,
                           double *gtab, cudaStream_t st);
size_t bw_phase_smem_bytes(int lmax);
// the edges of one matching: schedule positions first .. first + n_items - 1
cudaError_t launch_bw_phase(const BwParams &p, int first, int n_items, cudaStream_t st);
cudaError_t launch_unpack_grad(const EdgeDesc *edges, int n_edges, const NodeDesc *nodes, int n_nodes,
                               const long long *pair_base, const long long *unary_base, const double *gtab,
                               const double *adj_agg, float *grad_pair, float *grad_un, cudaStream_t st);

}  // namespace mplpp
