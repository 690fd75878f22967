// common.cuh -- device data layout and sm_103a PTX helpers shared by the
// solver's kernels (Handshake update, dual bound, rounding, backward).
//
// Device layout of a solver (all models concatenated, model after model):
//   agg  [u64 x 2] theta^phi_u of every node (Sec. 3, eq. reparametrization),
//                 each node's vector padded to a multiple of 4 entries, pad 0;
//   msg  [u64 x 2] per edge phi_{v->u} (L_u) then phi_{u->v} (L_v), each
//                 padded to a multiple of 4 entries, pad 0.
//                 Every entry is a double-float (hi + lo, see below) stored as
//                 two self-validating 8-byte words {payload float, version}:
//                 the version counts the updates of the node (agg) or edge
//                 (msg) that wrote it, so a reader on another SM accepts a
//                 value only when its word carries the version it expects
//                 (8-byte aligned accesses are single-copy atomic); no fence
//                 or counter orders the producer and the consumer.
//   tab  [float]  the ORIGINAL pairwise tables theta_uv, never written after
//                 creation; rows of L_v entries padded to a stride `ld`
//                 (multiple of 4) with +inf, tables 16-byte aligned.  The
//                 reparametrized table is implied:
//                 theta^phi_uv(s,t) = theta_uv(s,t) - phi_{v->u}(s) - phi_{u->v}(t).
//   un0  [float]  the original unaries in agg's layout (reset, energy).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace mplpp {
// Raises kernel's limit on dynamic shared memory to at least smem bytes on the
// current device, never lowers it: the limit belongs to the kernel, not to a
// solver, and solvers of one process share it (a lower value set for one
// solver would make another's launches fail).  Serialized by a lock.
cudaError_t raise_smem_limit_ptr(const void *kernel, size_t smem);
template <typename K>
inline cudaError_t raise_smem_limit(K *kernel, size_t smem)
{
    return raise_smem_limit_ptr(reinterpret_cast<const void *>(kernel), smem);
}
}  // namespace mplpp

namespace mplpp {

struct EdgeDesc {
    long long toff;   // float offset of the table in tab (Lu rows, stride ld)
    long long mu;     // entry offset of phi_{v->u} in msg (Lu entries)
    long long mv;     // entry offset of phi_{u->v} in msg (Lv entries)
    long long au;     // entry offset of node u's vector in agg
    long long av;     // entry offset of node v's vector in agg
    long long poff;   // float offset of the table in the caller's (unpadded) layout
    int Lu, Lv, ld;   // label counts and row stride (ld = Lv rounded up to 4)
    int gu, gv;       // global node ids
    int model;        // model index
};
static_assert(sizeof(EdgeDesc) == 72, "EdgeDesc layout");

struct NodeDesc {
    long long aoff;   // float offset in agg / un0
    long long uoff;   // float offset in the caller's (unpadded) unary layout
    int L;
    int model;
};
static_assert(sizeof(NodeDesc) == 24, "NodeDesc layout");

// One entry of a persistent worker's list: the edge's descriptor (one record,
// so that a worker needs a single load per item) plus the number of earlier
// updates of each endpoint within one iteration (its rank among that node's
// edges in schedule order) and the endpoint degrees.
struct WorkItem {
    EdgeDesc ed;
    int pos_u, pos_v;
    int deg_u, deg_v;
    int edge;
    int rows;         // rows per CTA of the edge's cluster of C CTAs: ceil(L_u / C)
};
static_assert(sizeof(WorkItem) == 96 && sizeof(WorkItem) % 16 == 0, "WorkItem layout");

// One earlier neighbour of a node in the rounding order, i.e. an edge (v, u)
// whose first node v precedes u: the edge's table offset and row stride, the
// offsets of its two messages and the neighbour's global id.
struct InRec {
    long long toff;   // table (rows x_v, stride ld)
    long long mu;     // phi of the edge's first node v (indexed by x_v)
    long long mv;     // phi of the edge's second node u (indexed by u's labels)
    int ld;
    int gu;           // v
};
static_assert(sizeof(InRec) == 32, "InRec layout");

constexpr int ERR_TIMEOUT = 1;
constexpr int ERR_NONFINITE = 2;

// ----------------------------------------------------------------------------
// PTX wrappers (sm_90+ features used on sm_103a: mbarrier transaction counts,
// bulk asynchronous copies, thread-block clusters and distributed shared memory)
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with acquire at cluster scope: for data that other CTAs of the
// cluster stored into this CTA's shared memory with st.async.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for an mbarrier phase; returns false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait_cluster(bar, parity)) return true;
    return false;
}

// Bulk (non-tensor) asynchronous copy global -> this CTA's shared memory,
// completing `bytes` transactions on `bar`.  dst and src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 16 bytes into the shared memory of a CTA of the cluster (addr and bar from
// mapa); the store completes 16 transaction bytes on that CTA's mbarrier.
__device__ __forceinline__ void st_async_f4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void st_dsmem_f4(uint32_t addr, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ float4 min4(float4 a, float4 b)
{
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}

__device__ __forceinline__ float4 add4s(float4 a, float s)
{
    return make_float4(a.x + s, a.y + s, a.z + s, a.w + s);
}

__device__ __forceinline__ float hmin_add(float4 x, float4 w)
{
    return fminf(fminf(x.x + w.x, x.y + w.y), fminf(x.z + w.z, x.w + w.w));
}

// ----------------------------------------------------------------------------
// Double-float ("df") numbers: value = hi + lo with |lo| <= ulp(hi) / 2, kept
// as a float2 {hi, lo}.  About 44 bits of precision from FP32 operations only
// (GB300's FP64 units are slow; its FP32 units are not).  Sums use the
// error-free transformations of Knuth (two-sum) and Dekker (fast two-sum).
// FP32 adds are never reassociated here (no fast-math), which these rely on.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 df_renorm(float s, float e)  // |s| >= |e| (fast two-sum)
{
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = ((a.x - (s - bb)) + (b.x - bb)) + (a.y + b.y);
    return df_renorm(s, e);
}

__device__ __forceinline__ float2 df_add_f(float2 a, float b)
{
    const float s = a.x + b;
    const float bb = s - a.x;
    const float e = ((a.x - (s - bb)) + (b - bb)) + a.y;
    return df_renorm(s, e);
}

__device__ __forceinline__ float2 df_sub(float2 a, float2 b)
{
    return df_add(a, make_float2(-b.x, -b.y));
}

__device__ __forceinline__ float2 df_half(float2 a)  // exact
{
    return make_float2(0.5f * a.x, 0.5f * a.y);
}

__device__ __forceinline__ float df_to_f(float2 a)
{
    return a.x + a.y;
}

__device__ __forceinline__ double df_to_d(float2 a)
{
    return static_cast<double>(a.x) + static_cast<double>(a.y);
}

// ----------------------------------------------------------------------------
// State entries: one double-float value as two self-validating 8-byte words,
// x = {hi (low 32 bits), version (high 32 bits)}, y = {lo, version}.
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long se_word(float v, unsigned version)
{
    unsigned bits;
    memcpy(&bits, &v, 4);
    return static_cast<unsigned long long>(bits) | (static_cast<unsigned long long>(version) << 32);
}

__host__ __device__ __forceinline__ float se_val(unsigned long long w)
{
    const unsigned bits = static_cast<unsigned>(w & 0xffffffffull);
    float v;
    memcpy(&v, &bits, 4);
    return v;
}

__host__ __device__ __forceinline__ ulonglong2 se_make(float2 v, unsigned version)
{
    return make_ulonglong2(se_word(v.x, version), se_word(v.y, version));
}

__host__ __device__ __forceinline__ float2 se_df(ulonglong2 e)
{
    return make_float2(se_val(e.x), se_val(e.y));
}

// both words of the entry carry `version` (each word is read atomically)
__device__ __forceinline__ bool se_ok(ulonglong2 e, unsigned version)
{
    return static_cast<unsigned>(e.x >> 32) == version && static_cast<unsigned>(e.y >> 32) == version;
}

__device__ __forceinline__ double se_d(ulonglong2 e)
{
    return static_cast<double>(se_val(e.x)) + static_cast<double>(se_val(e.y));
}

// Loads / stores of one entry at gpu scope (L2), one 8-byte-atomic access per word.
__device__ __forceinline__ ulonglong2 ld_se(const ulonglong2 *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_se(ulonglong2 *p, ulonglong2 v)
{
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(v.x), "l"(v.y) : "memory");
}

// Three-input minimum (one instruction on sm_100+); same value as two fminf.
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// x + w lane by lane with two packed FP32 additions (add.rn.f32x2, sm_100+);
// each lane is rounded exactly as a scalar FP32 addition.
__device__ __forceinline__ float4 add4(float4 x, float4 w)
{
    float4 r;
    asm("{\n\t.reg .b64 a, b, c;\n\t"
        "mov.b64 a, {%4, %5};\n\t"
        "mov.b64 b, {%8, %9};\n\t"
        "add.rn.f32x2 c, a, b;\n\t"
        "mov.b64 {%0, %1}, c;\n\t"
        "mov.b64 a, {%6, %7};\n\t"
        "mov.b64 b, {%10, %11};\n\t"
        "add.rn.f32x2 c, a, b;\n\t"
        "mov.b64 {%2, %3}, c;\n\t}"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "f"(x.x), "f"(x.y), "f"(x.z), "f"(x.w), "f"(w.x), "f"(w.y), "f"(w.z), "f"(w.w));
    return r;
}

// min(m, min over the four lanes of x + w)
__device__ __forceinline__ float min_add4(float m, float4 x, float4 w)
{
    const float4 v = add4(x, w);
    return min3f(min3f(m, v.x, v.y), v.z, v.w);
}

}  // namespace mplpp
