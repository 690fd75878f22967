// warp.cu -- the MPLP++ Handshake edge update with one warp per edge
// (persistent driver), for models whose label counts are small (<= 128).
//
// The update is the one of handshake.cu (Sec. 4, eq. (H), three-minimization
// form, message-form state, double-float O(L) arithmetic, FP32 minimizations
// on shifted operands) with the same operations in the same order, so every
// mapping gives bit-identical results.  What differs is the mapping: with
// thousands of small, mutually independent edges per matching (a batch of
// models), a whole CTA per edge leaves most of its threads idle and one
// shared-memory tile per CTA limits how many edges an SM holds.  Here every
// warp is an independent persistent worker with its own list of edges in
// schedule order; it waits only for the earlier updates of its edge's two
// nodes (versioned state entries, see common.cuh) and uses no block-wide
// barrier.  Each warp owns two shared-memory buffers of `cap` floats (at least
// 32 table rows) filled by bulk asynchronous copies (mbarrier transaction
// counts): a table that fits one buffer is copied once and serves all three
// passes; a larger one streams through both buffers in chunks of whole
// 32-row groups, once per pass, the copy of the next chunk in flight while
// the current one is processed.  The next edge's first chunk is copied while
// the current edge is processed.  Lane q holds column chunk q (4 columns):
// row minima are formed 32 rows at a time and finished by a reduce-scatter
// over the warp (31 shuffles), after which lane r owns row r of the group;
// column minima accumulate per lane over the rows.
#include <cfloat>
#include <cstdint>

#include "kernels.h"

namespace mplpp {

namespace {

// Per-warp shared memory (see hs_warp_bytes_per_warp): the work record being
// processed, two mbarriers, two table buffers of `cap` floats, the vectors.
struct WarpSmem {
    WorkItem *wi;
    uint64_t *bar;             // [2]
    float *buf[2];
    float2 *uh, *vh;           // double-float unaries without this edge's messages
    float *w1, *alpha, *beta;  // FP32 shifted operands of passes 1, 2 and 3
};

__device__ __forceinline__ WarpSmem warp_carve(char *base, int lw, int cap, int warp)
{
    char *b = base + static_cast<size_t>(warp) * hs_warp_bytes_per_warp(lw, cap);
    WarpSmem s;
    s.wi = reinterpret_cast<WorkItem *>(b);
    b += sizeof(WorkItem);
    s.bar = reinterpret_cast<uint64_t *>(b);
    b += 16;
    s.buf[0] = reinterpret_cast<float *>(b);
    b += 4 * static_cast<size_t>(cap);
    s.buf[1] = reinterpret_cast<float *>(b);
    b += 4 * static_cast<size_t>(cap);
    s.uh = reinterpret_cast<float2 *>(b);
    b += 8 * static_cast<size_t>(lw);
    s.vh = reinterpret_cast<float2 *>(b);
    b += 8 * static_cast<size_t>(lw);
    s.w1 = reinterpret_cast<float *>(b);
    b += 4 * static_cast<size_t>(lw);
    s.alpha = reinterpret_cast<float *>(b);
    b += 4 * static_cast<size_t>(lw);
    s.beta = reinterpret_cast<float *>(b);
    return s;
}

__device__ __forceinline__ void warp_set_err(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// Entries j = j0 + 32 k (k < K, j < n) of node vectors A/M (node u or v) and
// B/N (the other node): all 2K pairs are requested at once, then each is
// polled until its words carry the expected versions (va, vm for A/M; vb, vm
// for B/N; messages carry the edge's count vm).  fa(j, A[j] - M[j]) and
// fb(j, B[j] - N[j]) receive the double-float differences.  Bounded: past
// spin_limit polls ERR_TIMEOUT is recorded and the (stale) values are used;
// once the error word is set the wait gives up at the next check.
template <int K, typename FA, typename FB>
__device__ __forceinline__ void poll_two(const HsParams &p, const ulonglong2 *A, const ulonglong2 *M, int na,
                                         unsigned va, const ulonglong2 *B, const ulonglong2 *N, int nb, unsigned vb,
                                         unsigned vm, int j0, FA fa, FB fb)
{
    ulonglong2 x[K], y[K], z[K], w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = j0 + 32 * k;
        if (j < na) {
            x[k] = ld_se(A + j);
            y[k] = ld_se(M + j);
        }
        if (j < nb) {
            z[k] = ld_se(B + j);
            w[k] = ld_se(N + j);
        }
    }
    for (long long spins = 1;; ++spins) {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + 32 * k;
            if (j < na) ok = ok && se_ok(x[k], va) && se_ok(y[k], vm);
            if (j < nb) ok = ok && se_ok(z[k], vb) && se_ok(w[k], vm);
        }
        if (ok) break;
        if ((spins & 63) == 0 && *reinterpret_cast<volatile int *>(p.err) != 0) break;  // draining
        if (spins > p.spin_limit) {
            warp_set_err(p.err, ERR_TIMEOUT);
            break;
        }
        if (spins > 64) __nanosleep(64);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = j0 + 32 * k;
            if (j < na) {
                if (!se_ok(x[k], va)) x[k] = ld_se(A + j);
                if (!se_ok(y[k], vm)) y[k] = ld_se(M + j);
            }
            if (j < nb) {
                if (!se_ok(z[k], vb)) z[k] = ld_se(B + j);
                if (!se_ok(w[k], vm)) w[k] = ld_se(N + j);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = j0 + 32 * k;
        if (j < na) fa(j, df_sub(se_df(x[k]), se_df(y[k])));
        if (j < nb) fb(j, df_sub(se_df(z[k]), se_df(w[k])));
    }
}

// Minimum over the warp of each of 32 row values, reduce-scatter style: at
// the step with offset o a lane keeps the upper or lower half of its rows (bit
// o of its lane id) and receives the partner's partial minima of that half.
// Lane r ends with the minimum of row r (31 shuffles for 32 rows).
__device__ __forceinline__ float warp_min_rows32(float (&a)[32], int lane)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? a[i] : a[i + o];
            const float keep = up ? a[i + o] : a[i];
            a[i] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    return a[0];
}

// One bulk copy of table rows into a warp's buffer.
struct Copy {
    const float *src;
    uint32_t bytes;  // multiple of 16 (rows of ld floats, ld a multiple of 4)
};

// Rows per chunk: all of them if the table fits one buffer, else the most
// whole 32-row groups that fit (cap >= 32 * ld, so at least one group).
__device__ __forceinline__ int chunk_rows(int Lu, int ld, int cap)
{
    return Lu * ld <= cap ? Lu : (cap / ld) & ~31;
}

__device__ __forceinline__ Copy chunk_copy(const float *tab, long long toff, int Lu, int ld, int R, int j)
{
    const int r0 = j * R;
    const int rows = min(R, Lu - r0);
    return Copy{tab + toff + static_cast<long long>(r0) * ld, static_cast<uint32_t>(rows) * static_cast<uint32_t>(ld) * 4u};
}

// The warp's stream of bulk copies: copy g goes to buffer g & 1 and completes
// phase g >> 1 of mbarrier g & 1; copies are consumed in the order issued,
// and copy g is issued only once copy g - 2 (same buffer) has been used up.
struct Stream {
    unsigned g, c;  // copies issued, copies consumed (the same in every lane)
};

__device__ __forceinline__ void issue(const WarpSmem &sm, Stream &st, Copy cp, int lane)
{
    __syncwarp();  // every lane is done with the buffer's previous contents
    if (lane == 0) {
        const int b = static_cast<int>(st.g & 1u);
        fence_proxy_async();
        if (cp.bytes) {
            mbar_arrive_expect_tx(&sm.bar[b], cp.bytes);
            bulk_g2s(sm.buf[b], cp.src, cp.bytes, &sm.bar[b]);
        } else {
            mbar_arrive(&sm.bar[b]);
        }
    }
    ++st.g;
}

__device__ __forceinline__ const float *acquire(const HsParams &p, const WarpSmem &sm, Stream &st)
{
    const int b = static_cast<int>(st.c & 1u);
    if (!mbar_wait(&sm.bar[b], (st.c >> 1) & 1u, p.spin_limit)) warp_set_err(p.err, ERR_TIMEOUT);
    ++st.c;
    return sm.buf[b];
}

// One Handshake update of edge ed by one warp.  Its first chunk has been
// issued; `next` is the next edge's first chunk (issued from here).
__device__ void warp_item(const HsParams &p, const EdgeDesc &ed, const WarpSmem &sm, Versions ver, int lane,
                          Stream &st, bool has_next, Copy next)
{
    const int Lu = ed.Lu, Lv = ed.Lv, ld = ed.ld, Q = ld >> 2;
    ulonglong2 *agg = p.agg;
    ulonglong2 *msg = p.msg;
    const int R = chunk_rows(Lu, ld, p.cap);
    const int nc = (Lu + R - 1) / R;
    const bool resident = nc == 1;  // one copy serves all three passes

    // node v's vector and node u's rows, requested together
    constexpr int K = 2;
    const int Lm = Lu > Lv ? Lu : Lv;
    for (int j0 = lane; j0 < Lm; j0 += 32 * K)
        poll_two<K>(
            p, agg + ed.av, msg + ed.mv, Lv, ver.v, agg + ed.au, msg + ed.mu, Lu, ver.u + ver.bump, ver.e, j0,
            [&](int j, float2 d) { sm.vh[j] = d; }, [&](int j, float2 d) { sm.uh[j] = d; });
    __syncwarp();
    // w1(t) = vh(t) - vh(0), rounded once to FP32; padding columns 0
    const float2 vref = sm.vh[0];
    for (int t = lane; t < ld; t += 32) sm.w1[t] = t < Lv ? df_to_f(df_sub(sm.vh[t], vref)) : 0.f;
    __syncwarp();

    // the copy that follows chunk j of pass `pass` (1..3) in the stream
    auto follow = [&](int pass, int j) {
        if (!resident && j + 1 < nc)
            issue(sm, st, chunk_copy(p.tab, ed.toff, Lu, ld, R, j + 1), lane);
        else if (!resident && pass < 3)
            issue(sm, st, chunk_copy(p.tab, ed.toff, Lu, ld, R, 0), lane);
        else if (has_next && (resident || pass == 3))
            issue(sm, st, next, lane);
    };
    const float4 inf4 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    // row minima of a chunk (rows r0 .. r0 + rows), 32 at a time; lane r of a
    // group calls emit(row, minimum)
    auto row_chunk = [&](const float *buf, int r0, int rows, float4 wv, auto emit) {
        for (int g0 = 0; g0 < rows; g0 += 32) {
            float a[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) a[r] = INFINITY;
            if (lane < Q) {
                const float4 *col = reinterpret_cast<const float4 *>(buf + static_cast<size_t>(g0) * ld) + lane;
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    if (g0 + r < rows) a[r] = min_add4(a[r], col[r * Q], wv);
            }
            const float m = warp_min_rows32(a, lane);
            if (g0 + lane < rows) emit(r0 + g0 + lane, m);
        }
    };

    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + w1(t)] + vh(0) + uh(s));  alpha = uh - a
    const float *buf = nullptr;
    {
        const float4 wv = lane < Q ? reinterpret_cast<const float4 *>(sm.w1)[lane] : inf4;
        for (int j = 0; j < nc; ++j) {
            buf = acquire(p, sm, st);
            follow(1, j);
            row_chunk(buf, j * R, min(R, Lu - j * R), wv, [&](int s, float m) {
                // alpha = uh - a = 1/2 (uh - vh(0) - m), its value in exact arithmetic
                sm.alpha[s] = df_to_f(df_half(df_add_f(df_sub(sm.uh[s], vref), -m)));
            });
        }
    }
    __syncwarp();

    // pass 2: b(t) = min_s [theta(s,t) + alpha(s)] + vh(t), beta = vh - b; node
    // v's new vector is stored (visible to its next update) right away
    {
        float4 m = inf4;
        for (int j = 0; j < nc; ++j) {
            if (!resident) {
                buf = acquire(p, sm, st);
                follow(2, j);
            }
            const int r0 = j * R, rows = min(R, Lu - r0);
            if (lane < Q) {
                const float4 *col = reinterpret_cast<const float4 *>(buf) + lane;
#pragma unroll 4
                for (int r = 0; r < rows; ++r) {
                    const float a = sm.alpha[r0 + r];
                    m = min4(m, add4(col[r * Q], make_float4(a, a, a, a)));
                }
            }
        }
        if (lane < Q) {
            const float mc[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int t = 4 * lane + c;
                if (t < Lv) {
                    const float2 vh = sm.vh[t];
                    const float2 b = df_add_f(vh, mc[c]);
                    sm.beta[t] = -mc[c];  // vh - b in exact arithmetic
                    st_se(agg + ed.av + t, se_make(b, ver.v + 1u));
                    st_se(msg + ed.mv + t, se_make(df_sub(b, vh), ver.e + 1u));
                } else {
                    sm.beta[t] = 0.f;
                }
            }
        }
    }
    __syncwarp();

    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s); write node u's rows
    {
        const float4 bv = lane < Q ? reinterpret_cast<const float4 *>(sm.beta)[lane] : inf4;
        for (int j = 0; j < nc; ++j) {
            if (!resident) {
                buf = acquire(p, sm, st);
                follow(3, j);
            }
            row_chunk(buf, j * R, min(R, Lu - j * R), bv, [&](int s, float mm) {
                const float2 u = sm.uh[s];
                const float2 c = df_add_f(u, mm);
                st_se(agg + ed.au + s, se_make(c, ver.u + 1u));
                st_se(msg + ed.mu + s, se_make(df_sub(c, u), ver.e + 1u));
            });
        }
    }
    __syncwarp();  // the next item overwrites the vectors
}

__global__ void __launch_bounds__(512) hs_warp_kernel(HsParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int worker = blockIdx.x * static_cast<int>(blockDim.x >> 5) + wib;
    if (worker >= p.workers) return;  // the whole warp: no block-wide barrier follows
    const WarpSmem sm = warp_carve(smem_raw, p.lw, p.cap, wib);
    const int begin = p.work_off[worker];
    const int n = p.work_off[worker + 1] - begin;
    const long long total = static_cast<long long>(n) * p.iterations;
    if (total == 0) return;
    if (lane == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    constexpr int kRec = static_cast<int>(sizeof(WorkItem) / sizeof(int4));
    if (lane < kRec)
        reinterpret_cast<int4 *>(sm.wi)[lane] = __ldg(reinterpret_cast<const int4 *>(p.work + begin) + lane);
    __syncwarp();
    Stream st = {0u, 0u};
    {
        const EdgeDesc &e0 = sm.wi->ed;
        issue(sm, st, chunk_copy(p.tab, e0.toff, e0.Lu, e0.ld, chunk_rows(e0.Lu, e0.ld, p.cap), 0), lane);
    }
    int i = 0, it = 0;
    for (long long k = 0; k < total; ++k) {
        const EdgeDesc ed = sm.wi->ed;
        const int pos_u = sm.wi->pos_u, pos_v = sm.wi->pos_v, deg_u = sm.wi->deg_u, deg_v = sm.wi->deg_v;
        // the next record, requested now, stored once this item is done; its
        // first chunk (toff from lane 0's 16 bytes, L_u and ld from lane 3's)
        const bool has_next = k + 1 < total;
        const int inext = (i + 1 == n) ? 0 : i + 1;
        int4 nrec = make_int4(0, 0, 0, 0);
        if (has_next && lane < kRec) nrec = __ldg(reinterpret_cast<const int4 *>(p.work + begin + inext) + lane);
        const unsigned lo = __shfl_sync(0xffffffffu, static_cast<unsigned>(nrec.x), 0);
        const unsigned hi = __shfl_sync(0xffffffffu, static_cast<unsigned>(nrec.y), 0);
        const int nLu = __shfl_sync(0xffffffffu, nrec.x, 3);
        const int nld = __shfl_sync(0xffffffffu, nrec.z, 3);
        Copy next = {p.tab, 0u};
        if (has_next) {
            const long long ntoff = static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | lo);
            next = chunk_copy(p.tab, ntoff, nLu, nld, chunk_rows(nLu, nld, p.cap), 0);
        }
        // update counts modulo 2^32 (only equality is tested)
        const Versions ver = {static_cast<unsigned>(it) * static_cast<unsigned>(deg_u) + static_cast<unsigned>(pos_u),
                              static_cast<unsigned>(it) * static_cast<unsigned>(deg_v) + static_cast<unsigned>(pos_v),
                              static_cast<unsigned>(it), (p.test_wait && k == 0 && worker == 0) ? 1u : 0u};
        warp_item(p, ed, sm, ver, lane, st, has_next, next);
        if (has_next && lane < kRec) reinterpret_cast<int4 *>(sm.wi)[lane] = nrec;
        __syncwarp();
        if (++i == n) {
            i = 0;
            ++it;
        }
    }
    // every issued copy has been consumed (the last item issues none)
}

}  // namespace

cudaError_t hs_warp_prepare(size_t smem)
{
    return raise_smem_limit(hs_warp_kernel, smem);
}

int hs_warp_max_blocks(int threads, size_t smem)
{
    if (hs_warp_prepare(smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hs_warp_kernel, threads, smem) != cudaSuccess) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

cudaError_t hs_launch_warp(const HsParams &p, int blocks, int threads, size_t smem, cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;
    hs_warp_kernel<<<blocks, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace mplpp
