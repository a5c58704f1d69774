// Device helpers shared by the decode kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace acx {

#define ACX_FULL 0xffffffffu

constexpr int kErrCorrupt = -2;
constexpr int kErrTimeout = -5;

// Error stages recorded beside the first error status.
enum : int {
    kStageRans = 1,
    kStageVarint = 2,
    kStageTokens = 3,
    kStageSources = 4,
    kStageWait = 5,
    kStagePlain = 6,
    kStageLimits = 7,
};

// err[0]: first status; err[1]: stage << 24 | detail; err[2]: block index.
__device__ __forceinline__ void set_err(int* err, int code, int where, uint32_t block) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = where;
        err[2] = (int)block;
    }
}

// The same, also recorded as archive a's own status in a batched job.
__device__ __forceinline__ void set_err_arc(const JobDev& job, int a, int code, int where, uint32_t block) {
    set_err(job.err, code, where, block);
    if (job.arc_err && a >= 0) atomicCAS(job.arc_err + a, 0, code);
}

// Limit of a wait for a bulk copy from global memory into shared memory.
// Copies complete by themselves, so this bound only guards against a broken
// device; the caller's timeout (JobDev::timeout_ns) bounds the waits on other
// work (pieces, barriers, published blocks).
constexpr uint64_t kCopyWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory loads at 32-bit shared-window addresses (volatile: they stay
// in program order with the mbarrier waits that guard the data they read).
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {  // zero-extended into a 32-bit register
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts_u8(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint4 lds_u128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
                 : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Acquire-release fence at GPU scope: with relaxed loads before it, an
// acquire pattern; with relaxed writes after it, a release pattern (neither
// needs the sequentially consistent fence that __threadfence() is).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Atomic AND without ordering of its own: after a fence (fence + strong write
// is a release pattern), several of them share that one fence.
__device__ __forceinline__ void red_and_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- mbarrier / TMA (1-D bulk copies) ---------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_1d_s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int find_arc(const JobDev& job, uint32_t item) {
    if (!job.arcs) return 0;
    int lo = 0, hi = (int)job.n_arcs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (job.arcs[mid].item_base <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ ArcJob load_arc(const JobDev& job, int a) { return job.arcs ? job.arcs[a] : job.one; }

// Where a work item's block goes: its block id, output slot, pending-piece
// base and decoded-stream offset (idx counted from the archive's item_base).
struct ItemRef {
    uint32_t blk, slot, span_base, need_off, need_n;
    uint64_t scratch;
};
__device__ __forceinline__ ItemRef item_ref(const ArcJob& J, uint32_t idx) {
    ItemRef r;
    if (J.items) {
        const ItemDev it = J.items[idx];
        r.blk = it.block;
        r.slot = it.slot;
        r.span_base = it.span_base;
        r.scratch = it.scratch;
        r.need_off = it.need_off;
        r.need_n = it.need_n;
    } else {
        r.blk = J.lo + idx;
        r.slot = r.blk;
        r.need_off = 0;
        r.need_n = 0;
        r.span_base = J.blk[r.blk].span_base;
        r.scratch = J.blk[r.blk].scratch;
    }
    return r;
}
// Output slot of block a, and the output offset of absolute position pos.
__device__ __forceinline__ uint64_t slot_of(const ArcJob& J, uint64_t a) { return J.slot ? J.slot[a] : a; }
__device__ __forceinline__ uint64_t out_off(const ArcJob& J, uint64_t pos) {
    return J.slot ? (uint64_t)J.slot[pos >> 14] * kBlock + (pos & (kBlock - 1)) : pos;
}

// Is block id a in the ascending list dl[0, n)?
__device__ __forceinline__ bool listed(const uint32_t* dl, uint32_t n, uint32_t a) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        const uint32_t v = dl[m];
        if (v == a) return true;
        if (v < a) lo = m + 1; else hi = m;
    }
    return false;
}

// Bit masks of the bytes [s, e) of a 16 KiB block bitmap, word by word.
__device__ __forceinline__ uint32_t range_mask(uint32_t w, uint32_t s, uint32_t e) {
    uint32_t m = 0xffffffffu;
    if (w == (s >> 5)) m &= 0xffffffffu << (s & 31);
    if (w == ((e - 1) >> 5)) m &= 0xffffffffu >> (31 - ((e - 1) & 31));
    return m;
}

// Cut a pending match (destination offset o in its block, absolute source src,
// length ml, distance d = destination - source) into pieces of at most kPiece
// bytes at slots out[0..); returns the number of pieces.
__device__ __forceinline__ uint32_t emit_pieces(SpanRec* out, uint32_t o, uint64_t src, uint32_t ml, uint64_t d,
                                                uint32_t level = 0) {
    uint32_t k = 0;
    for (uint32_t q = 0; q < ml; q += kPiece, k++) {
        const uint32_t len = ml - q < kPiece ? ml - q : kPiece;
        uint64_t s;
        uint32_t phase = 0, period = 0;
        if (d >= ml) {
            s = src + q;
        } else {
            s = src;
            period = (uint32_t)d;
            phase = q % period;
        }
        out[k] = SpanRec{(uint32_t)s, (uint32_t)(s >> 32) | (phase << 8) | (level << 24), (o + q) | (len << 16),
                         period};
    }
    return k;
}
__host__ __device__ inline uint32_t pieces_of(uint32_t ml) { return (ml + kPiece - 1) / kPiece; }

}  // namespace acx
