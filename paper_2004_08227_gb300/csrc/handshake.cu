// handshake.cu -- the MPLP++ Handshake edge update on sm_103a (FP32 hot path).
//
// One update of edge uv (Sec. 4, eq. (H), three-minimization form) on the
// message-form state of common.cuh:
//   uh(s) = agg_u(s) - phi_{v->u}(s),  vh(t) = agg_v(t) - phi_{u->v}(t)
//           (the unaries without this edge's messages; g = theta_uv + uh + vh)
//   a(s)  = 1/2 (min_t [theta_uv(s,t) + (vh(t) - vh(0))] + vh(0) + uh(s))
//                                                               = 1/2 min_t g(s,t)
//   alpha(s) = uh(s) - a(s) = 1/2 (uh(s) - vh(0) - min_t [...])    (formed as the latter)
//   b(t)  = min_s [theta_uv(s,t) + alpha(s)] + vh(t)            = min_s [g(s,t) - a(s)]
//   beta(t) = vh(t) - b(t) = -min_s [theta_uv(s,t) + alpha(s)]     (formed as the latter)
//   c(s)  = min_t [theta_uv(s,t) + beta(t)] + uh(s)             = min_t [g(s,t) - b(t)]
//   agg_u := c, phi_{v->u} := c - uh;  agg_v := b, phi_{u->v} := b - vh.
// Precision: the O(L) state and vector arithmetic are double-float (hi + lo
// FP32 pairs, ~44 bits; reparametrized unaries grow to large magnitudes, where
// plain FP32 rounding would accumulate over thousands of updates, and GB300's
// FP64 units are too slow for the critical path); the O(L^2) minimizations
// run in FP32 on the table and on small quantities (vh shifted by vh(0),
// alpha, beta), rounded to FP32 once per update.  The pairwise table is only read (4 B per entry, once from
// HBM); all three minimizations run on the copy staged in shared memory.
// Min-plus is not a dense contraction, so this is FP32 ALU work bound by HBM
// bandwidth.
//
// Mapping: a cluster of C CTAs shares one edge; CTA `rank` owns the rows
// [rank*R, rank*R + R) (R = ceil(L_u / C)), loaded with one bulk asynchronous
// copy.  Row minima (passes 1 and 3) are local to the CTA; the partial column
// minima of pass 2 are all-gathered across the cluster: every CTA stores its
// vector into slot `rank` of every CTA's shared memory with st.async, each
// store completing its bytes on the receiving CTA's mbarrier, so a CTA waits
// only for the data it needs (no cluster-wide barrier per edge), then reduces
// the C slots locally.  The slots and their mbarriers alternate between two
// sets from one edge to the next: a CTA writes a set again only after it has
// received the other set from every CTA, i.e. after every CTA has read it.
//
// Two drivers:
//   looped      one launch per matching; the launch boundary orders matchings
//               (Sec. 6, GPU implementation: a barrier between matchings);
//   persistent  one launch for all iterations; every cluster walks a fixed
//               list of edges in schedule order and waits, per edge, only for
//               the earlier updates of its two end nodes, while the next
//               edge's table is already streaming into the second buffer.
//               There are no counters or fences: every state entry carries the
//               number of updates of its node (or edge) that produced it (see
//               common.cuh), and a thread polls the entries it needs until
//               they carry the expected count, so the data and the signal
//               arrive in one L2 round trip.  Node v's new vector is visible
//               as soon as it is stored, before pass 3.  Waits are bounded:
//               past spin_limit polls the kernel records ERR_TIMEOUT and
//               drains without waiting.
#include <cfloat>
#include <cstdint>

#include "kernels.h"

namespace mplpp {

namespace {

struct Smem {
    WorkItem *wi;       // [2] the current and the next work item (persistent driver)
    float *tile;        // nbuf buffers of tile_floats each
    float2 *uh, *vh;    // double-float unaries without this edge's messages (uh: nbuf
                        // buffers, by item parity)
    float *w1;          // vh(t) - vh(0) in FP32 (pass 1)
    float *alpha, *beta, *pm;
    float4 *part;
    uint64_t *bar;      // [6]: table buffers 0 and 1, exchange slots 0 and 1, node u ready 0 and 1
};

__device__ __forceinline__ Smem carve(char *base, const HsParams &p, int nbuf)
{
    Smem s;
    s.wi = reinterpret_cast<WorkItem *>(base);
    float2 *d = reinterpret_cast<float2 *>(base + 2 * sizeof(WorkItem));
    s.uh = d; d += static_cast<size_t>(nbuf) * p.rmax;
    s.vh = d; d += p.ldmax;
    float *f = reinterpret_cast<float *>(d);
    s.tile = f;
    f += static_cast<size_t>(nbuf) * p.tile_floats;
    s.w1 = f; f += p.ldmax;
    s.alpha = f; f += p.rmax;
    s.beta = f; f += p.ldmax;
    s.pm = f; f += static_cast<size_t>(nbuf) * p.ldmax * p.C;  // [item parity][CTA of the cluster][column]
    s.part = reinterpret_cast<float4 *>(f); f += 4 * blockDim.x;
    s.bar = reinterpret_cast<uint64_t *>(f);  // 16-byte aligned: every array above is a multiple of 16 bytes
    return s;
}

// Lanes per row for the row minima: all of the CTA's rows in one round
// (lanes * rows <= threads), at least two float4 chunks per lane, a power of
// two <= 32.  Fewer lanes per row means longer independent chains per lane
// and fewer shuffle steps.
__device__ __forceinline__ int row_lanes(int nr, int Q, int T)
{
    int g = T / (nr > 0 ? nr : 1);
    int h = Q >> 1;
    h = h < 1 ? 1 : h;
    g = g < h ? g : h;
    g = g > 32 ? 32 : (g < 1 ? 1 : g);
    return 1 << (31 - __clz(g));
}

// This CTA's rows [r0, r0 + nr) of edge ed, R = ceil(L_u / C) rows per CTA
// (the persistent driver's work records carry R: no division on the way to
// the first poll).
__device__ __forceinline__ void rows_of_R(const EdgeDesc &ed, int rank, int R, int &r0, int &nr)
{
    r0 = rank * R;
    nr = ed.Lu - r0;
    nr = nr < 0 ? 0 : (nr > R ? R : nr);
}

// Thread 0: start the bulk copy of this CTA's row slice of edge ed's table.
__device__ __forceinline__ void issue_tile(const EdgeDesc &ed, int rank, int R, const float *tab, float *buf,
                                           uint64_t *bar)
{
    int r0, nr;
    rows_of_R(ed, rank, R, r0, nr);
    const uint32_t bytes = static_cast<uint32_t>(nr) * static_cast<uint32_t>(ed.ld) * 4u;
    if (bytes) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(buf, tab + ed.toff + static_cast<long long>(r0) * ed.ld, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

__device__ __forceinline__ void set_err(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// Barrier 1 over `count` threads (a multiple of 32) of the CTA.
__device__ __forceinline__ void named_barrier_1(int count)
{
    asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}


// Persistent driver, next item: its work record (16 bytes per thread of the
// last warp, requested at the start of this item and stored into shared
// memory once the thread's polls are done) and its table slice (started by
// thread 0 once the node vectors have arrived, so that the burst of table
// reads from every SM does not delay the polls of the state entries).
struct Next {
    int4 rec;           // this thread's 16 bytes of the next work record
    int4 *rec_dst;      // where they go (nullptr: none)
    WorkItem *wi;       // the next work record in shared memory
    float *dst;         // the next table buffer
    uint64_t *bar;      // its mbarrier
    bool on;            // there is a next item
};

// f(j, a[j] - m[j]) from the entries x = a[j], y = m[j] already requested;
// CHECK: first poll until a[j] carries version va and m[j] version vm (only
// a word that still carries an older version is requested again).  Returns
// the number of requests of a[j] made.
template <bool CHECK, typename F>
__device__ __forceinline__ long long poll_diff(const HsParams &p, const ulonglong2 *a, const ulonglong2 *m, int j,
                                               unsigned va, unsigned vm, ulonglong2 x, ulonglong2 y, F f)
{
    long long spins = 1;
    if (CHECK) {
        for (; !(se_ok(x, va) && se_ok(y, vm)); ++spins) {
            if ((spins & 63) == 0 && *reinterpret_cast<volatile int *>(p.err) != 0) break;  // draining
            if (spins > p.spin_limit) {
                set_err(p.err, ERR_TIMEOUT);
                break;
            }
            if (spins > 64) __nanosleep(64);
            if (!se_ok(x, va)) x = ld_se(a + j);
            if (!se_ok(y, vm)) y = ld_se(m + j);
        }
    }
    f(j, df_sub(se_df(x), se_df(y)));
    return spins;
}

// min_t [row(t) + w(t)] over this lane's chunks q = lg, lg + G, ... (two chains)
__device__ __forceinline__ float row_min(const float4 *row, const float4 *w, int Q, int lg, int G)
{
    float m0 = INFINITY, m1 = INFINITY;
    int q = lg;
#pragma unroll 4
    for (; q + G < Q; q += 2 * G) {
        m0 = min_add4(m0, row[q], w[q]);
        m1 = min_add4(m1, row[q + G], w[q + G]);
    }
    if (q < Q) m0 = min_add4(m0, row[q], w[q]);
    return fminf(m0, m1);
}

__device__ __forceinline__ void group_min(float &m, int G)
{
    for (int o = G >> 1; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
}

// Register-resident passes: warp w holds rows w + W k (k < kRR) of the CTA's
// slice, lane j the float4 chunks j + 32 i (i < kCR), loaded from shared
// memory once; passes 1 and 3 then reduce in registers (a butterfly over the
// warp per row), and pass 2 reduces the warp's rows in registers and the warps
// through the (by then free) tile buffer.  Shared memory is read once per
// update instead of three times.  For other shapes the passes stream the
// shared-memory copy.
constexpr int kRR = 5;
constexpr int kCR = 3;

// Row stride (float4) of the per-warp column partials of pass 2: = 2 mod 8,
// so that the reduction's reads (4 lanes per column chunk, one per warp
// group) fall into distinct 16-byte bank groups.
__device__ __host__ __forceinline__ int part_stride(int Q)
{
    return Q + ((2 - Q) & 7);
}

__device__ __forceinline__ bool rr_fits(int nr, int Q, int T, int tile_floats)
{
    return Q > 32 && Q <= 32 * kCR && nr <= kRR * (T >> 5) && (T >> 5) * part_stride(Q) * 4 <= tile_floats;
}

// The same with the last warp as node u's poller (it holds no rows); at most
// 3 rows per poller lane.
__device__ __host__ __forceinline__ bool pw_fits(int nr, int Q, int T, int tile_floats)
{
    const int W = (T >> 5) - 1;
    return W >= 1 && Q >= 1 && Q <= 32 * kCR && nr <= kRR * W && nr <= 96 && W * part_stride(Q) * 4 <= tile_floats;
}

// Minimum over the warp of each of the kRR = 5 row values (five independent
// warp reductions in hardware; min.f32 semantics, as fminf).  The result is
// the minimum of row rs_row(lane); lanes 0, 8, 4, 16 and 24 own rows 0..4
// (rs_owner).
static_assert(kRR == 5, "five rows per warp");

__device__ __forceinline__ float warp_min_f32(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ int rs_row(int lane);

__device__ __forceinline__ float warp_min_rows5(const float (&a)[kRR], int lane)
{
    const float m0 = warp_min_f32(a[0]), m1 = warp_min_f32(a[1]), m2 = warp_min_f32(a[2]);
    const float m3 = warp_min_f32(a[3]), m4 = warp_min_f32(a[4]);
    const int k = rs_row(lane);
    return k == 0 ? m0 : (k == 1 ? m1 : (k == 2 ? m2 : (k == 3 ? m3 : m4)));
}

__device__ __forceinline__ int rs_row(int lane)
{
    return (lane & 16) ? ((lane & 8) ? 4 : 3) : ((lane & 8) ? 1 : ((lane & 4) ? 2 : 0));
}

__device__ __forceinline__ bool rs_owner(int lane)
{
    return lane == 0 || lane == 4 || lane == 8 || lane == 16 || lane == 24;
}

// Lane-wise minimum of five float4
__device__ __forceinline__ float4 min5_4(float4 a, float4 b, float4 c, float4 d, float4 e)
{
    return make_float4(min3f(min3f(a.x, b.x, c.x), d.x, e.x), min3f(min3f(a.y, b.y, c.y), d.y, e.y),
                       min3f(min3f(a.z, b.z, c.z), d.z, e.z), min3f(min3f(a.w, b.w, c.w), d.w, e.w));
}

// Register-resident passes for narrow rows (Q <= 32 float4 chunks): lanes
// form slots of G lanes (G the power of two >= Q), lane c of a slot holds
// chunk c of kSR rows: rows (warp * P + slot) + W * P * k, k < kSR, P = 32 / G
// slots per warp.  Row minima reduce over the G lanes of a slot, column minima
// over a thread's rows, the warp's slots, then the warps.
constexpr int kSR = 8;

__device__ __forceinline__ int rs_group(int Q)
{
    return Q <= 1 ? 1 : 1 << (32 - __clz(Q - 1));
}

__device__ __forceinline__ bool rs_fits(int nr, int Q, int T, int tile_floats)
{
    if (Q < 1 || Q > 32) return false;
    const int P = 32 / rs_group(Q), W = T >> 5;
    return nr <= W * P * kSR && W * part_stride(Q) * 4 <= tile_floats;
}

// Minimum over the G lanes of a slot of each of the kSR = 8 row values; lane c
// of the slot receives emit(k, minimum of row k) for the rows it owns.  For G
// >= 8 a reduce-scatter (the lane keeps the half of the rows given by its bits
// G/2, G/4, G/8, then plain exchanges): lanes c with c % (G/8) == 0 own row
// c / (G/8).  For G < 8 every lane gets every row; lane c owns rows c mod G.
static_assert(kSR == 8, "the reduce-scatter below splits exactly eight rows");

template <typename F>
__device__ __forceinline__ void slot_min8(float (&a)[kSR], int c, int G, F emit)
{
    constexpr unsigned kAll = 0xffffffffu;
    if (G >= 8) {
        int o = G >> 1;
        {
            const bool up = (c & o) != 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float send = up ? a[i] : a[i + 4];
                const float keep = up ? a[i + 4] : a[i];
                a[i] = fminf(keep, __shfl_xor_sync(kAll, send, o));
            }
        }
        o >>= 1;
        {
            const bool up = (c & o) != 0;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float send = up ? a[i] : a[i + 2];
                const float keep = up ? a[i + 2] : a[i];
                a[i] = fminf(keep, __shfl_xor_sync(kAll, send, o));
            }
        }
        o >>= 1;
        {
            const bool up = (c & o) != 0;
            const float send = up ? a[0] : a[1];
            const float keep = up ? a[1] : a[0];
            a[0] = fminf(keep, __shfl_xor_sync(kAll, send, o));
        }
        for (o >>= 1; o > 0; o >>= 1) a[0] = fminf(a[0], __shfl_xor_sync(kAll, a[0], o));
        const int sh = 31 - __clz(G >> 3);  // log2(G / 8)
        if ((c & ((G >> 3) - 1)) == 0) emit(c >> sh, a[0]);
    } else {
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < kSR; ++k) a[k] = fminf(a[k], __shfl_xor_sync(kAll, a[k], o));
#pragma unroll
        for (int k = 0; k < kSR; ++k)
            if ((k & (G - 1)) == c) emit(k, a[k]);
    }
}

// One Handshake update of edge ed by this CTA (its row slice); the table slice
// is (or will be) in `tile`, signalled by `bar` completing phase `parity`.
// `xpar` selects the exchange buffer (alternates between consecutive items).
// SIGNAL: wait for the expected versions of the inputs (persistent driver).
// RM: 0 passes over the shared-memory slice, 1 register-resident passes
// (rr_fits must hold), 2 register-resident passes for narrow rows (rs_fits).
// PW (persistent driver, RM == 1 only): the last warp holds no rows; it polls
// node u's rows and stages the next item while the other warps, once node v
// has arrived, run pass 1's minima; node u's unaries are needed only by pass
// 1's emit, which waits for the poller's arrival on `ubar` (phase `upar`).
// STREAM (queue driver): `tile` is the table itself in global memory (read by
// every pass, from L2 after the first), not a staged copy; no mbarrier.
template <bool CLUSTER, bool SIGNAL, int RM, bool PW = false, bool STREAM = false>
__device__ void hs_item(const HsParams &p, const EdgeDesc &ed, const float *tile, const Smem &sm, int rank,
                        int r0, int nr, uint64_t *bar, uint32_t parity, int xpar, Versions ver, Next nx,
                        uint64_t *ubar = nullptr, uint32_t upar = 0)
{
    static_assert(!PW || (SIGNAL && RM == 1), "the poller warp serves the persistent register-resident passes");
    static_assert(!STREAM || (SIGNAL && RM == 0 && !CLUSTER && !PW), "streamed tables: shared-memory-free passes");
    const int T = blockDim.x, tid = threadIdx.x;
    const int C = CLUSTER ? p.C : 1;
    const int ld = ed.ld, Q = ld >> 2, Lv = ed.Lv;
    float2 *const uh = sm.uh + static_cast<size_t>(xpar) * p.rmax;  // pass 3 of the previous item may still read the other
    ulonglong2 *agg = p.agg;
    ulonglong2 *msg = p.msg;

    // The table slice: wait for its bulk copy and, for the register-resident
    // passes, load this thread's fragment.  Independent of the node vectors:
    // both drivers do it while the requests for the vectors are in flight.
    const float4 *t4 = reinterpret_cast<const float4 *>(tile);
    const int lane = tid & 31, warp = tid >> 5, W = (T >> 5) - (PW ? 1 : 0);  // W: warps holding rows
    const bool poller = PW && warp == W;
    const float4 inf4 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    float4 tr[RM == 1 ? kRR : 1][RM == 1 ? kCR : 1];
    float4 ts[RM == 2 ? kSR : 1];
    // narrow-row mapping (RM == 2): slot size, this lane's chunk, its rows
    const int sg = RM == 2 ? rs_group(Q) : 1;
    const int sc = lane & (sg - 1);
    const int sbase = warp * (32 / sg) + lane / sg, sstride = W * (32 / sg);
    // this item's exchange: C CTAs x Q float4 column minima arrive
    if (CLUSTER && tid == 0)
        mbar_arrive_expect_tx(sm.bar + 2 + xpar, static_cast<uint32_t>(C) * static_cast<uint32_t>(Q) * 16u);
    auto load_tile = [&]() {
        if (!STREAM && !mbar_wait(bar, parity, p.spin_limit)) set_err(p.err, ERR_TIMEOUT);
        if (RM == 1 && !poller) {
#pragma unroll
            for (int k = 0; k < kRR; ++k)
#pragma unroll
                for (int i = 0; i < kCR; ++i) {
                    const int s = warp + W * k, q = lane + 32 * i;
                    tr[k][i] = (s < nr && q < Q) ? t4[static_cast<size_t>(s) * Q + q] : inf4;
                }
        }
        if (RM == 2) {
#pragma unroll
            for (int k = 0; k < kSR; ++k) {
                const int s = sbase + sstride * k;
                ts[k] = (s < nr && sc < Q) ? t4[static_cast<size_t>(s) * Q + sc] : inf4;
            }
        }
    };
    // unaries without this edge's messages (written by other SMs: L2 loads).
    // Persistent driver: the first warps poll node v's entries until they
    // carry the expected versions, the last warps node u's rows (warps split
    // in proportion to the entries), so the two waits overlap and every entry
    // is requested at once; the first requests are in flight while the table
    // fragment is loaded.
    if (PW) {
        if (poller) {
            // node u's rows: every request first (at most 3 per lane), then the checks
            const ulonglong2 *A = agg + ed.au + r0;
            const ulonglong2 *M = msg + ed.mu + r0;
            const unsigned va = ver.u + ver.bump;
            ulonglong2 xa[3], ya[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int j = lane + 32 * i;
                xa[i] = ya[i] = make_ulonglong2(0ull, 0ull);
                if (j < nr) {
                    xa[i] = ld_se(A + j);
                    ya[i] = ld_se(M + j);
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int j = lane + 32 * i;
                if (j < nr)
                    poll_diff<true>(p, A, M, j, va, ver.e, xa[i], ya[i], [&](int jj, float2 d) { uh[jj] = d; });
            }
            for (int j = lane + 96; j < nr; j += 32)
                poll_diff<true>(p, A, M, j, va, ver.e, ld_se(A + j), ld_se(M + j),
                                [&](int jj, float2 d) { uh[jj] = d; });
            __syncwarp();
            if (lane == 0) mbar_arrive(ubar);
            // the next item: its work record, then (once the record is in
            // shared memory) its table slice
            if (nx.rec_dst) *nx.rec_dst = nx.rec;
            __syncwarp();
            if (lane == 31 && nx.on) {
                fence_proxy_async();
                issue_tile(nx.wi->ed, rank, nx.wi->rows, p.tab, nx.dst, nx.bar);
            }
        } else {
            // node v's entries over every thread of the row warps
            const int nv = 32 * W;
            const ulonglong2 *A = agg + ed.av;
            const ulonglong2 *M = msg + ed.mv;
            ulonglong2 x = make_ulonglong2(0ull, 0ull), y = x;
            if (tid < Lv) {
                x = ld_se(A + tid);
                y = ld_se(M + tid);
            }
            load_tile();
            for (int j = tid; j < Lv; j += nv) {
                if (j != tid) {
                    x = ld_se(A + j);
                    y = ld_se(M + j);
                }
                poll_diff<true>(p, A, M, j, ver.v, ver.e, x, y, [&](int jj, float2 d) { sm.vh[jj] = d; });
            }
            for (int t = Lv + tid; t < ld; t += nv) sm.vh[t] = make_float2(0.f, 0.f);
            named_barrier_1(nv);
            const float2 vref = sm.vh[0];
            for (int t = tid; t < ld; t += nv) sm.w1[t] = t < Lv ? df_to_f(df_sub(sm.vh[t], vref)) : 0.f;
            asm volatile("bar.sync 2, %0;" ::"r"(nv) : "memory");
        }
    } else if (SIGNAL) {
        // (any split in 1 .. W - 1 is correct: a float estimate, no division)
        const int uw = min(W - 1, max(1, __float2int_rn(static_cast<float>(W * nr) *
                                                         __frcp_rn(static_cast<float>(nr + Lv)))));
        const int nv = T - 32 * uw;  // threads on node v's side
        const bool vside = tid < nv;
        const int i0 = vside ? tid : tid - nv, ni = vside ? nv : T - nv;
        const ulonglong2 *A = vside ? agg + ed.av : agg + ed.au + r0;
        const ulonglong2 *M = vside ? msg + ed.mv : msg + ed.mu + r0;
        const int n = vside ? Lv : nr;
        const unsigned va = vside ? ver.v : ver.u + ver.bump;
        float2 *dst = vside ? sm.vh : uh;
        ulonglong2 x = make_ulonglong2(0ull, 0ull), y = x;
        if (i0 < n) {
            x = ld_se(A + i0);
            y = ld_se(M + i0);
        }
        load_tile();
        for (int j = i0; j < n; j += ni) {
            if (j != i0) {
                x = ld_se(A + j);
                y = ld_se(M + j);
            }
            poll_diff<true>(p, A, M, j, va, ver.e, x, y, [&](int jj, float2 d) { dst[jj] = d; });
        }
        if (vside) {
            for (int t = Lv + i0; t < ld; t += ni) sm.vh[t] = make_float2(0.f, 0.f);
            named_barrier_1(nv);
            // w1(t) = vh(t) - vh(0), rounded once to FP32
            const float2 vref = sm.vh[0];
            for (int t = i0; t < ld; t += ni) sm.w1[t] = t < Lv ? df_to_f(df_sub(sm.vh[t], vref)) : 0.f;
        }
    } else {
        for (int s = tid; s < nr; s += T)
            poll_diff<false>(p, agg + ed.au + r0, msg + ed.mu + r0, s, 0u, 0u, ld_se(agg + ed.au + r0 + s),
                             ld_se(msg + ed.mu + r0 + s), [&](int j, float2 d) { uh[j] = d; });
        for (int t = tid; t < ld; t += T) {
            if (t < Lv)
                poll_diff<false>(p, agg + ed.av, msg + ed.mv, t, 0u, 0u, ld_se(agg + ed.av + t), ld_se(msg + ed.mv + t),
                                 [&](int j, float2 d) { sm.vh[j] = d; });
            else
                sm.vh[t] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 vref = sm.vh[0];
        for (int t = tid; t < ld; t += T) sm.w1[t] = t < Lv ? df_to_f(df_sub(sm.vh[t], vref)) : 0.f;
    }

    if (!PW) {
        if (SIGNAL && nx.rec_dst) *nx.rec_dst = nx.rec;
        if (!SIGNAL) load_tile();
        __syncthreads();
        // the last thread (its warp has the fewest rows in the passes): the buffer's
        // previous item has finished
        if (SIGNAL && tid == T - 1 && nx.on) {
            fence_proxy_async();
            issue_tile(nx.wi->ed, rank, nx.wi->rows, p.tab, nx.dst, nx.bar);
        }
    }

    const int G = row_lanes(nr, Q, T);
    const int gid = tid / G, lg = tid % G, ng = T / G;
    float *xbuf = sm.pm + static_cast<size_t>(xpar) * C * ld;  // this item's exchange slots
    uint64_t *xbar = sm.bar + 2 + xpar;                          // ... and their mbarrier

    // pass 1: a(s) = 1/2 (min_t [theta(s,t) + w1(t)] + vh(0) + uh(s));  alpha = uh - a
    {
        const float4 *w = reinterpret_cast<const float4 *>(sm.w1);
        const float2 vref = sm.vh[0];
        // alpha = uh - a = 1/2 (uh - vh(0) - m), its value in exact arithmetic;
        // d = uh - vh(0) does not depend on the minimum
        auto alpha_of = [&](float2 d, float m) { return df_to_f(df_half(df_add_f(d, -m))); };
        auto emit = [&](int s, float m) { sm.alpha[s] = alpha_of(df_sub(uh[s], vref), m); };
        if (RM == 1) {
          if (!poller) {
            float acc[kRR];
            float4 wv[kCR];
            const int s = warp + W * rs_row(lane);  // the five owners emit at once
            const bool own = rs_owner(lane) && s < nr;
            float2 d = make_float2(0.f, 0.f);
            if (!PW && own) d = df_sub(uh[s], vref);  // node u's rows are in: before the minima
#pragma unroll
            for (int i = 0; i < kCR; ++i) wv[i] = lane + 32 * i < Q ? w[lane + 32 * i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kRR; ++k) {
                acc[k] = INFINITY;
#pragma unroll
                for (int i = 0; i < kCR; ++i) acc[k] = min_add4(acc[k], tr[k][i], wv[i]);
            }
            const float mk = warp_min_rows5(acc, lane);
            if (own) {
                if (PW) {
                    if (!mbar_wait(ubar, upar, p.spin_limit)) set_err(p.err, ERR_TIMEOUT);
                    d = df_sub(uh[s], vref);
                }
                sm.alpha[s] = alpha_of(d, mk);
            }
          }
        } else if (RM == 2) {
            const float4 wv = sc < Q ? w[sc] : make_float4(0.f, 0.f, 0.f, 0.f);
            float acc[kSR];
#pragma unroll
            for (int k = 0; k < kSR; ++k) acc[k] = min_add4(INFINITY, ts[k], wv);
            slot_min8(acc, sc, sg, [&](int k, float m) {
                const int s = sbase + sstride * k;
                if (s < nr) emit(s, m);
            });
        } else {
            for (int base = 0; base < nr; base += ng) {
                const int s = base + gid;
                float m = s < nr ? row_min(t4 + static_cast<size_t>(s) * Q, w, Q, lg, G) : INFINITY;
                group_min(m, G);
                if (s < nr && lg == 0) emit(s, m);
            }
        }
    }
    // The register-resident passes read in pass 2 only the alpha of their own
    // warp's rows, which pass 1 emitted from that warp.
    if (RM)
        __syncwarp();
    else
        __syncthreads();

    // pass 2 (this CTA's rows): pm(t) = min_s [theta(s,t) + alpha(s)], stored
    // into slot `rank` of the pm buffer of every CTA of the cluster
    {
        const uint32_t slot = smem_u32(xbuf) + 4u * static_cast<uint32_t>(ld) * static_cast<uint32_t>(rank);
        const uint32_t xb = smem_u32(xbar);
        auto push = [&](int q, float4 m) {
            if (CLUSTER) {
                for (int r = 0; r < C; ++r) st_async_f4(mapa_shared(slot + 16u * q, r), m, mapa_shared(xb, r));
            } else {
                reinterpret_cast<float4 *>(xbuf)[q] = m;
            }
        };
        const int nsub = RM ? 0 : T / Q;
        if (RM == 1) {
            // the warp's rows in registers, then the warps through the tile buffer
            float4 *part2 = reinterpret_cast<float4 *>(const_cast<float *>(tile));
            float4 al[kRR];
#pragma unroll
            for (int k = 0; k < kRR; ++k) {
                const float a = (!poller && warp + W * k < nr) ? sm.alpha[warp + W * k] : 0.f;
                al[k] = make_float4(a, a, a, a);
            }
            const int Qp = part_stride(Q);
            if (!poller) {
#pragma unroll
                for (int i = 0; i < kCR; ++i) {
                    const float4 m = min5_4(add4(tr[0][i], al[0]), add4(tr[1][i], al[1]), add4(tr[2][i], al[2]),
                                            add4(tr[3][i], al[3]), add4(tr[4][i], al[4]));
                    if (lane + 32 * i < Q) part2[warp * Qp + lane + 32 * i] = m;
                }
            }
            __syncthreads();
            // 4 consecutive lanes per chunk, each over every 4th warp, then 2 shuffles
            for (int base = warp * 32; base < 4 * Q; base += T) {
                const int idx = base + lane, q = idx >> 2, part = idx & 3;
                float4 m = inf4;
                if (idx < 4 * Q) {  // W <= 16 warps: at most four partials per lane, loaded together
                    float4 v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[j] = (part + 4 * j < W) ? part2[(part + 4 * j) * Qp + q] : inf4;
                    m = min4(min4(v[0], v[1]), min4(v[2], v[3]));
                }
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1)
                    m = min4(m, make_float4(__shfl_xor_sync(0xffffffffu, m.x, o), __shfl_xor_sync(0xffffffffu, m.y, o),
                                            __shfl_xor_sync(0xffffffffu, m.z, o), __shfl_xor_sync(0xffffffffu, m.w, o)));
                if (idx < 4 * Q && part == 0) push(q, m);
            }
        } else if (RM == 2) {
            // the thread's rows, the warp's slots (lanes c, c + G, ...), then
            // the warps through the (by then free) tile buffer
            float4 *part2 = reinterpret_cast<float4 *>(const_cast<float *>(tile));
            float4 m = inf4;
#pragma unroll
            for (int k = 0; k < kSR; ++k) {
                const int s = sbase + sstride * k;
                const float a = s < nr ? sm.alpha[s] : 0.f;
                m = min4(m, add4(ts[k], make_float4(a, a, a, a)));
            }
            for (int o = sg; o < 32; o <<= 1)
                m = min4(m, make_float4(__shfl_xor_sync(0xffffffffu, m.x, o), __shfl_xor_sync(0xffffffffu, m.y, o),
                                        __shfl_xor_sync(0xffffffffu, m.z, o), __shfl_xor_sync(0xffffffffu, m.w, o)));
            const int Qp = part_stride(Q);
            if (lane < sg && sc < Q) part2[warp * Qp + sc] = m;
            __syncthreads();
            // one CTA per edge: the combine below reads the warps' partials
            for (int q = tid; q < (CLUSTER ? Q : 0); q += T) {
                float4 mm = part2[q];
                for (int w2 = 1; w2 < W; ++w2) mm = min4(mm, part2[w2 * Qp + q]);
                push(q, mm);
            }
        } else if (nsub >= 1) {
            if (tid < nsub * Q) {
                const int q = tid % Q, sub = tid / Q;
                float4 m = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
                int s = sub;
#pragma unroll 4
                for (; s + nsub < nr; s += 2 * nsub) {  // two rows per step: packed adds, 3-input mins
                    const float a1 = sm.alpha[s], a2 = sm.alpha[s + nsub];
                    const float4 v1 = add4(t4[static_cast<size_t>(s) * Q + q], make_float4(a1, a1, a1, a1));
                    const float4 v2 = add4(t4[static_cast<size_t>(s + nsub) * Q + q], make_float4(a2, a2, a2, a2));
                    m = make_float4(min3f(m.x, v1.x, v2.x), min3f(m.y, v1.y, v2.y), min3f(m.z, v1.z, v2.z),
                                    min3f(m.w, v1.w, v2.w));
                }
                if (s < nr) m = min4(m, add4s(t4[static_cast<size_t>(s) * Q + q], sm.alpha[s]));
                sm.part[sub * Q + q] = m;
            }
            __syncthreads();
        }
        for (int q = tid; q < (RM ? 0 : Q); q += T) {
            float4 m;
            if (nsub >= 1) {
                m = sm.part[q];
                for (int j = 1; j < nsub; ++j) m = min4(m, sm.part[j * Q + q]);
            } else {
                m = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
                for (int s = 0; s < nr; ++s) m = min4(m, add4s(t4[static_cast<size_t>(s) * Q + q], sm.alpha[s]));
            }
            push(q, m);
        }
    }

    // combine the column minima of all CTAs of the edge:
    //   b(t) = min_s [...] + vh(t),  beta(t) = vh(t) - b(t) = -min_s [...]
    // (beta formed as the latter, its value in exact arithmetic); node v's new
    // vector is stored by the CTAs of the cluster, a range of columns each
    const int vper = (Lv + C - 1) / C, vt0 = rank * vper;
    if (CLUSTER) {
        if (!mbar_wait_cluster(xbar, parity, p.spin_limit)) set_err(p.err, ERR_TIMEOUT);
    } else if (RM != 2) {
        __syncthreads();
    }
    for (int t = tid; t < ld; t += T) {
        float m;
        if (!CLUSTER && RM == 2) {  // the minimum over the warps' partial column minima
            const float *pf = tile;
            const int wst = 4 * part_stride(Q);
            m = pf[t];
            for (int w2 = 1; w2 < W; ++w2) m = fminf(m, pf[w2 * wst + t]);
        } else {
            m = xbuf[t];
        }
        if (CLUSTER) {  // C <= 8 slots, loaded together
            float v[7];
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r - 1] = r < C ? xbuf[r * ld + t] : INFINITY;
            m = min3f(m, min3f(v[0], v[1], v[2]), min3f(v[3], v[4], fminf(v[5], v[6])));
        }
        sm.beta[t] = t < Lv ? -m : 0.f;
        // node v's new vector, visible to node v's next update as soon as it
        // is stored
        if (t >= vt0 && t < vt0 + vper && t < Lv) {
            const float2 vh = sm.vh[t];
            const float2 b = df_add_f(vh, m);
            st_se(agg + ed.av + t, se_make(b, ver.v + 1u));
            st_se(msg + ed.mv + t, se_make(df_sub(b, vh), ver.e + 1u));
        }
    }
    // The slots of this parity are written again two items later, by CTAs that
    // have received this CTA's next-item column minima, i.e. after this read.
    __syncthreads();

    // pass 3: c(s) = min_t [theta(s,t) + beta(t)] + uh(s); write node u's rows
    {
        const float4 *w = reinterpret_cast<const float4 *>(sm.beta);
        auto emit = [&](int s, float m) {
            const float2 u = uh[s];
            const float2 c = df_add_f(u, m);
            st_se(agg + ed.au + r0 + s, se_make(c, ver.u + 1u));
            st_se(msg + ed.mu + r0 + s, se_make(df_sub(c, u), ver.e + 1u));
        };
        if (RM == 1) {
          if (!poller) {
            float acc[kRR];
            float4 bw[kCR];
#pragma unroll
            for (int i = 0; i < kCR; ++i) bw[i] = lane + 32 * i < Q ? w[lane + 32 * i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kRR; ++k) {
                acc[k] = INFINITY;
#pragma unroll
                for (int i = 0; i < kCR; ++i) acc[k] = min_add4(acc[k], tr[k][i], bw[i]);
            }
            const float mk = warp_min_rows5(acc, lane);
            const int s = warp + W * rs_row(lane);  // the five owners emit at once
            if (rs_owner(lane) && s < nr) emit(s, mk);
          }
        } else if (RM == 2) {
            const float4 bv = sc < Q ? w[sc] : make_float4(0.f, 0.f, 0.f, 0.f);
            float acc[kSR];
#pragma unroll
            for (int k = 0; k < kSR; ++k) acc[k] = min_add4(INFINITY, ts[k], bv);
            slot_min8(acc, sc, sg, [&](int k, float m) {
                const int s = sbase + sstride * k;
                if (s < nr) emit(s, m);
            });
        } else {
            for (int base = 0; base < nr; base += ng) {
                const int s = base + gid;
                float m = s < nr ? row_min(t4 + static_cast<size_t>(s) * Q, w, Q, lg, G) : INFINITY;
                group_min(m, G);
                if (s < nr && lg == 0) emit(s, m);
            }
        }
    }
    // No barrier before the next item: up to its first block-wide barrier it
    // writes only vh, w1 and the other parity's uh, record and table buffer,
    // none of which pass 3 reads.
}

// RRK: an item whose rows fit takes the register-resident passes for wide rows
// (models with tables wider than 128 labels); without RRK those for narrow
// rows.  Any other item takes the shared-memory passes.
template <bool CLUSTER, bool RRK>
__global__ void __launch_bounds__(512, CLUSTER || RRK ? 1 : 2) hs_looped_kernel(HsParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    Smem sm = carve(smem_raw, p, 1);
    const int C = CLUSTER ? p.C : 1;
    const int rank = CLUSTER ? static_cast<int>(cluster_ctarank()) : 0;
    const EdgeDesc ed = p.edges[p.items[blockIdx.x / C]];
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int R = (ed.Lu + C - 1) / C;
    if (threadIdx.x == 0) issue_tile(ed, rank, R, p.tab, sm.tile, &sm.bar[0]);
    if (CLUSTER) {  // every CTA of the cluster is running before any remote store
        cluster_arrive_relaxed();
        cluster_wait_acquire();
    }
    int r0, nr;
    rows_of_R(ed, rank, R, r0, nr);
    if (RRK && rr_fits(nr, ed.ld >> 2, blockDim.x, p.tile_floats))
        hs_item<CLUSTER, false, 1>(p, ed, sm.tile, sm, rank, r0, nr, &sm.bar[0], 0u, 0, Versions{0u, 0u, 0u, 0u}, Next{});
    else if (!RRK && rs_fits(nr, ed.ld >> 2, blockDim.x, p.tile_floats))
        hs_item<CLUSTER, false, 2>(p, ed, sm.tile, sm, rank, r0, nr, &sm.bar[0], 0u, 0, Versions{0u, 0u, 0u, 0u}, Next{});
    else
        hs_item<CLUSTER, false, 0>(p, ed, sm.tile, sm, rank, r0, nr, &sm.bar[0], 0u, 0, Versions{0u, 0u, 0u, 0u}, Next{});
    if (CLUSTER) {  // no CTA leaves while another may still access its shared memory
        cluster_arrive_release();
        cluster_wait_acquire();
    }
}

template <bool CLUSTER, bool RRK, bool PW>
__global__ void __launch_bounds__(512) hs_persistent_kernel(HsParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    Smem sm = carve(smem_raw, p, 2);
    const int C = CLUSTER ? p.C : 1;
    const int rank = CLUSTER ? static_cast<int>(cluster_ctarank()) : 0;
    const int cid = blockIdx.x / C;
    const int begin = p.work_off[cid];
    const int n = p.work_off[cid + 1] - begin;
    const long long total = static_cast<long long>(n) * p.iterations;
    if (threadIdx.x == 0) {
        for (int j = 0; j < 6; ++j) mbar_init(&sm.bar[j], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (CLUSTER) {  // every CTA of the cluster is running before any remote store
        cluster_arrive_relaxed();
        cluster_wait_acquire();
    }
    if (total == 0) return;
    constexpr int kRec = static_cast<int>(sizeof(WorkItem) / sizeof(int4));
    const int tid = threadIdx.x, T = blockDim.x;
    const bool rec_lane = tid >= T - kRec;  // lanes of the last warp that move work records
    if (rec_lane)
        reinterpret_cast<int4 *>(&sm.wi[0])[tid - (T - kRec)] =
            reinterpret_cast<const int4 *>(p.work + begin)[tid - (T - kRec)];
    __syncthreads();
    if (tid == 0) issue_tile(sm.wi[0].ed, rank, sm.wi[0].rows, p.tab, sm.tile, &sm.bar[0]);
    int i = 0, it = 0;
    unsigned npw = 0;  // items that took the poller-warp passes (their mbarrier phases)
    for (long long k = 0; k < total; ++k) {
        const WorkItem &w = sm.wi[k & 1];
        const EdgeDesc ed = w.ed;
        Next nx = {};
        if (k + 1 < total) {
            const int inext = (i + 1 == n) ? 0 : i + 1;
            const int b1 = static_cast<int>((k + 1) & 1);
            nx.wi = &sm.wi[b1];
            nx.dst = sm.tile + b1 * p.tile_floats;
            nx.bar = sm.bar + b1;
            nx.on = true;
            if (rec_lane) {
                nx.rec = __ldg(reinterpret_cast<const int4 *>(p.work + begin + inext) + (tid - (T - kRec)));
                nx.rec_dst = reinterpret_cast<int4 *>(nx.wi) + (tid - (T - kRec));
            }
        }
        // update counts modulo 2^32 (only equality is tested)
        const Versions ver = {static_cast<unsigned>(it) * static_cast<unsigned>(w.deg_u) + static_cast<unsigned>(w.pos_u),
                              static_cast<unsigned>(it) * static_cast<unsigned>(w.deg_v) + static_cast<unsigned>(w.pos_v),
                              static_cast<unsigned>(it), (p.test_wait && k == 0 && cid == 0) ? 1u : 0u};
        const int b = static_cast<int>(k & 1);
        int r0, nr;
        rows_of_R(ed, rank, w.rows, r0, nr);
        const uint32_t par = static_cast<uint32_t>((k >> 1) & 1);
        if constexpr (PW) {
            // the host launches this variant only when every item fits (hs_pw_fits)
            hs_item<CLUSTER, true, 1, true>(p, ed, sm.tile + b * p.tile_floats, sm, rank, r0, nr, sm.bar + b, par, b,
                                            ver, nx, sm.bar + 4 + (npw & 1), (npw >> 1) & 1);
            ++npw;
        } else {
            if (RRK && rr_fits(nr, ed.ld >> 2, blockDim.x, p.tile_floats))
                hs_item<CLUSTER, true, 1>(p, ed, sm.tile + b * p.tile_floats, sm, rank, r0, nr, sm.bar + b, par, b, ver,
                                          nx);
            else if (!RRK && rs_fits(nr, ed.ld >> 2, blockDim.x, p.tile_floats))
                hs_item<CLUSTER, true, 2>(p, ed, sm.tile + b * p.tile_floats, sm, rank, r0, nr, sm.bar + b, par, b, ver,
                                          nx);
            else
                hs_item<CLUSTER, true, 0>(p, ed, sm.tile + b * p.tile_floats, sm, rank, r0, nr, sm.bar + b, par, b, ver,
                                          nx);
        }
        if (++i == n) {
            i = 0;
            ++it;
        }
    }
    if (CLUSTER) {  // no CTA leaves while another may still access its shared memory
        cluster_arrive_release();
        cluster_wait_acquire();
    }
}

// Queue driver: one CTA per edge at a time, every CTA taking the next item of
// one global queue (an atomic counter over a list that repeats every
// iteration).  The list orders each model's items by its matchings and
// interleaves the models by their progress through an iteration, so an
// item's inputs were produced by items far earlier in the queue; every wait is
// on an earlier item, taken by a co-resident CTA, so the waits end.  Tables
// are read from global memory by every pass (the first pass from HBM, the
// others from L2: nothing staged in shared memory, so many CTAs fit an SM),
// and the next item's table is prefetched into L2 while the current one runs.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(128) hs_queue_kernel(HsParams p)
{
    extern __shared__ __align__(16) char smem_raw[];
    Smem sm = carve(smem_raw, p, 2);  // node u's unaries and the column partials alternate by item parity
    long long *s_g = reinterpret_cast<long long *>(sm.bar + 6);  // [2] item index of this and the next item
    constexpr int kRec = static_cast<int>(sizeof(WorkItem) / sizeof(int4));
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
    const bool last_warp = tid >= T - 32, rec_lane = tid >= T - kRec;
    const long long EE = p.queue_items;
    const long long total = EE * static_cast<long long>(p.iterations);
    if (tid == T - 1) s_g[0] = static_cast<long long>(atomicAdd(p.queue, 1ull));
    __syncthreads();
    long long g = s_g[0];
    if (g < total && rec_lane)
        reinterpret_cast<int4 *>(&sm.wi[0])[tid - (T - kRec)] =
            reinterpret_cast<const int4 *>(p.work + g % EE)[tid - (T - kRec)];
    __syncthreads();
    for (long long k = 0; g < total; ++k) {
        const WorkItem &w = sm.wi[k & 1];
        const EdgeDesc ed = w.ed;
        const long long it = g / EE;
        Next nx = {};
        if (last_warp) {  // the next item: index, work record, table into L2
            unsigned long long v = 0;
            if (lane == 31) v = atomicAdd(p.queue, 1ull);
            v = __shfl_sync(0xffffffffu, v, 31);
            const long long g2 = static_cast<long long>(v);
            if (lane == 31) s_g[(k + 1) & 1] = g2;
            if (g2 < total) {
                const WorkItem *src = p.work + g2 % EE;
                if (rec_lane) {
                    nx.rec = __ldg(reinterpret_cast<const int4 *>(src) + (tid - (T - kRec)));
                    nx.rec_dst = reinterpret_cast<int4 *>(&sm.wi[(k + 1) & 1]) + (tid - (T - kRec));
                }
                if (lane == 31) {
                    const long long toff = __ldg(&src->ed.toff);
                    const int Lu = __ldg(&src->ed.Lu), ld = __ldg(&src->ed.ld);
                    prefetch_l2(p.tab + toff, static_cast<uint32_t>(Lu) * static_cast<uint32_t>(ld) * 4u);
                }
            }
        }
        const Versions ver = {static_cast<unsigned>(it) * static_cast<unsigned>(w.deg_u) + static_cast<unsigned>(w.pos_u),
                              static_cast<unsigned>(it) * static_cast<unsigned>(w.deg_v) + static_cast<unsigned>(w.pos_v),
                              static_cast<unsigned>(it), (p.test_wait && k == 0 && blockIdx.x == 0) ? 1u : 0u};
        hs_item<false, true, 0, false, true>(p, ed, p.tab + ed.toff, sm, 0, 0, ed.Lu, nullptr, 0u,
                                             static_cast<int>(k & 1), ver, nx);
        g = s_g[(k + 1) & 1];
    }
}

template <typename K>
cudaError_t set_attrs(K kernel, size_t smem)
{
    cudaError_t e = raise_smem_limit(kernel, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename K>
cudaError_t launch(K kernel, const HsParams &p, int grid, int threads, size_t smem, int C, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (C > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = static_cast<unsigned>(C);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        na = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

}  // namespace

size_t hs_smem_bytes(int nbuf, int tile_floats, int rmax, int ldmax, int threads, int C)
{
    // 2 work records; double-float uh (nbuf), vh; FP32 tiles, w1, alpha, beta, pm (nbuf x C slots), part (float4 x T);
    // 64 bytes: 6 mbarriers and the queue driver's two item indices
    const size_t d = static_cast<size_t>(nbuf) * rmax + static_cast<size_t>(ldmax);
    const size_t f = static_cast<size_t>(nbuf) * tile_floats + static_cast<size_t>(rmax) +
                     (2 + static_cast<size_t>(nbuf) * C) * static_cast<size_t>(ldmax) + 4 * static_cast<size_t>(threads);
    return 2 * sizeof(WorkItem) + d * 8 + f * 4 + 64;
}

cudaError_t hs_prepare(size_t smem)
{
    cudaError_t e;
    if ((e = set_attrs(hs_looped_kernel<false, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_looped_kernel<true, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_looped_kernel<false, true>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_looped_kernel<true, true>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_persistent_kernel<false, false, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_persistent_kernel<true, false, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_persistent_kernel<false, true, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_persistent_kernel<true, true, false>, smem)) != cudaSuccess) return e;
    if ((e = set_attrs(hs_persistent_kernel<false, true, true>, smem)) != cudaSuccess) return e;
    return set_attrs(hs_persistent_kernel<true, true, true>, smem);
}

cudaError_t hs_launch_looped(const HsParams &p, int n_items, int threads, size_t smem, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    const int grid = n_items * p.C;
    if (p.rr)
        return p.C > 1 ? launch(hs_looped_kernel<true, true>, p, grid, threads, smem, p.C, st)
                       : launch(hs_looped_kernel<false, true>, p, grid, threads, smem, 1, st);
    return p.C > 1 ? launch(hs_looped_kernel<true, false>, p, grid, threads, smem, p.C, st)
                   : launch(hs_looped_kernel<false, false>, p, grid, threads, smem, 1, st);
}

cudaError_t hs_launch_persistent(const HsParams &p, int clusters, int threads, size_t smem, cudaStream_t st)
{
    const int grid = clusters * p.C;
    if (p.rr && p.pw)
        return p.C > 1 ? launch(hs_persistent_kernel<true, true, true>, p, grid, threads, smem, p.C, st)
                       : launch(hs_persistent_kernel<false, true, true>, p, grid, threads, smem, 1, st);
    if (p.rr)
        return p.C > 1 ? launch(hs_persistent_kernel<true, true, false>, p, grid, threads, smem, p.C, st)
                       : launch(hs_persistent_kernel<false, true, false>, p, grid, threads, smem, 1, st);
    return p.C > 1 ? launch(hs_persistent_kernel<true, false, false>, p, grid, threads, smem, p.C, st)
                   : launch(hs_persistent_kernel<false, false, false>, p, grid, threads, smem, 1, st);
}

cudaError_t hs_launch_queue(const HsParams &p, int blocks, int threads, size_t smem, cudaStream_t st)
{
    // (shared memory attribute set by hs_queue_max_blocks when the mapping was made)
    return launch(hs_queue_kernel, p, blocks, threads, smem, 1, st);
}

int hs_queue_max_blocks(int threads, size_t smem)
{
    if (raise_smem_limit(hs_queue_kernel, smem) != cudaSuccess) return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hs_queue_kernel, threads, smem) != cudaSuccess) return 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

bool hs_pw_fits(int nr_max, int Q_max, int threads, int tile_floats)
{
    // every row count up to nr_max and chunk count up to Q_max must fit
    return Q_max > 32 && pw_fits(nr_max, Q_max, threads, tile_floats) &&
           (((threads >> 5) - 1) * (Q_max + 7) * 4 <= tile_floats);
}

bool hs_rr_fits(int nr_max, int Q_max, int threads, int tile_floats)
{
    // every row count up to nr_max and chunk count up to Q_max must fit
    return Q_max > 32 && Q_max <= 32 * kCR && nr_max <= kRR * (threads >> 5) &&
           (threads >> 5) * (Q_max + 7) * 4 <= tile_floats;
}

int hs_max_active_clusters(int C, int threads, size_t smem, bool rr)
{
    if (hs_prepare(smem) != cudaSuccess) return 0;
    if (C <= 1) {
        int per_sm = 0;
        const cudaError_t e = rr ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hs_persistent_kernel<false, true, true>,
                                                                                  threads, smem)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hs_persistent_kernel<false, false, false>,
                                                                                  threads, smem);
        if (e != cudaSuccess) return 0;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return per_sm * sms;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(C));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = rr ? cudaOccupancyMaxActiveClusters(&n, hs_persistent_kernel<true, true, true>, &cfg)
                             : cudaOccupancyMaxActiveClusters(&n, hs_persistent_kernel<true, false, false>, &cfg);
    return e == cudaSuccess ? n : 0;
}

}  // namespace mplpp
