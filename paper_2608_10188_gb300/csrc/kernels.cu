// Decode kernels for format v1 of the blockwise absolute-offset LZ77 codec,
// written for GB300 (sm_103a).
//
//  k_rans      entropy stage: interleaved-rANS lane decoders, one warp per
//              block (cmd, len, off, lit streams in turn).  Decode tables live
//              in shared memory; the 16-bit renormalisation words stream into
//              a per-warp shared-memory ring through 1-D TMA bulk copies
//              (cp.async.bulk + mbarrier).  Each step is one symbol per lane;
//              the lanes that renormalise take consecutive words in lane
//              order (ballot + popc), the textbook interleaved-rANS order.
//  k_assemble  parse + match layer, one CTA per block (persistent, tickets in
//              ascending block order):
//                * varint boundaries by compaction (byte < 0x80 ends a value)
//                  and a CTA prefix count -> LL_i, ML_i   (paper, "The Last
//                  Sequential Element": varints are 0.61% of commands)
//                * prefix sums of LL+ML, LL and #NEW -> token positions,
//                  literal positions and offset indices (the 93.94% that a
//                  prefix sum handles)
//                * the 4-entry distance history as a monoid scan (each
//                  token is a map on the history; maps compose
//                  associatively), skipped when a block has no repeat code
//                  (history-free encoding)
//                * literal placement into a shared-memory copy of the block
//                * matches as periodic fills out[dst+k] = out[src + k mod d]
//                  (paper, "What Does: Periods, Not Chains"), in rounds while
//                  their in-block sources become final
//                * one coalesced 16 KiB write of the block, then bytes whose
//                  source chain leaves the block are resolved by bounded
//                  waits on the source blocks' publish state and pending-
//                  byte bitmaps (no whole-block waits, so neighbour
//                  references do not chain the blocks)
//  k_plain     comparison decoder: same entropy stage output, but one thread
//              per block parses sequentially with the history and copies
//              byte by byte, with the same publish protocol.
//
// Every device-side wait is bounded by %globaltimer; on expiry the kernel
// records ACEAPEX_E_TIMEOUT and the block is abandoned (no trap, no hang).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace acx {

#define ACX_FULL 0xffffffffu

constexpr int kErrCorrupt = -2;
constexpr int kErrTimeout = -5;

// err[0]: first status; err[1]: where it was raised (stage << 24 | detail);
// err[2]: block index.  Stages: 1 rANS (detail = stream), 2 varints, 3 tokens,
// 4 offsets/history, 5 dependency wait, 6 plain decoder.
__device__ __forceinline__ void set_err(int* err, int code, int where = 0, uint32_t block = 0) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = where;
        err[2] = (int)block;
    }
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint8_t ld_cg_u8(const uint8_t* p) {
    unsigned short v;
    asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint8_t)v;
}

// ---- mbarrier / TMA (1-D bulk) -----------------------------------------------------------
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
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// =====================================================================================
// Entropy stage
// =====================================================================================
constexpr int kRansWarps = 16;
constexpr int kRingWords = 1024;   // 2 KiB of 16-bit words per warp
constexpr int kChunkWords = 256;   // one TMA chunk = 512 B
constexpr int kSlots = kRingWords / kChunkWords;

struct RansSmem {
    uint32_t tab[4][kM];                     // 64 KiB: decode entries of the four stream types
    uint16_t ring[kRansWarps][kRingWords];   // 32 KiB
    uint64_t bar[kRansWarps][kSlots];
    int arc;                                 // archive whose tables are loaded
    int next_arc;
};

// Decode one rANS stream with one warp.  S states per lane: K <= 32 uses
// one state on lanes < K; K = 64 / 128 gives each lane 2 / 4 independent
// states (lane j of the stream lives on warp lane j mod 32), which keeps
// several table lookups in flight per lane.  Returns false on a format
// violation or an expired wait.  `seq` counts the TMA chunks this warp has
// used so far (mbarrier phase bookkeeping across streams).
template <int S>
__device__ bool rans_stream(const uint32_t* __restrict__ tab, const uint8_t* __restrict__ body, uint32_t enc,
                            uint32_t n, uint32_t K, uint8_t* __restrict__ out, uint16_t* ring, uint64_t* bar,
                            uint32_t& seq, int lane, uint64_t deadline) {
    const uint32_t hdr = (4 * K + 15) & ~15u;
    if (enc < hdr || ((enc - hdr) & 1)) return false;
    const uint32_t W = (enc - hdr) >> 1;
    const uint8_t* words = body + hdr;
    const uint32_t wbytes = (2 * W + 15) & ~15u;
    const uint32_t nchunks = (wbytes + 511) / 512;
    uint32_t x[S];
    bool ok = true;
#pragma unroll
    for (int s = 0; s < S; s++) {
        const uint32_t j = 32 * s + lane;
        x[s] = j < K ? *reinterpret_cast<const uint32_t*>(body + 4 * j) : 0;
        ok = ok && (j >= K || x[s] >= kL);
    }
    ok = __all_sync(ACX_FULL, ok);
    const uint32_t seq0 = seq;
    // local chunk c lands in ring slot (seq0 + c) % kSlots, so word w of this
    // stream sits at ring[(rbase + w) % kRingWords]
    const uint32_t rbase = (seq0 % kSlots) * kChunkWords;
    uint32_t issued = 0, ready = 0;
    while (issued < nchunks && issued < (uint32_t)kSlots) {
        uint32_t q = seq0 + issued, slot = q % kSlots;
        uint32_t bytes = min(512u, wbytes - 512 * issued);
        if (lane == 0) {
            mbar_arrive_tx(&bar[slot], bytes);
            tma_load_1d(ring + slot * kChunkWords, words + 512 * issued, bytes, &bar[slot]);
        }
        issued++;
    }
    const uint32_t lt_mask = (1u << lane) - 1;
    uint32_t p = 0;
    const uint32_t steps = ok ? (n + K - 1) / K : 0;
    for (uint32_t t = 0; t < steps; t++) {
        // words [p, p + 32*S) must be resident before the renormalisation loads
        while (ready < nchunks && ready * kChunkWords < p + 32 * S) {
            uint32_t q = seq0 + ready;
            uint32_t spins = 0;
            while (!mbar_try_wait(&bar[q % kSlots], (q / kSlots) & 1)) {
                if ((++spins & 1023) == 0 && gtimer() > deadline) { ok = false; break; }
            }
            ok = __all_sync(ACX_FULL, ok);
            if (!ok) break;
            ready++;
        }
        if (!ok) break;
        // refill slots whose previous chunk has been fully consumed
        if (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots) {
            __syncwarp();
            do {
                uint32_t q = seq0 + issued, slot = q % kSlots;
                uint32_t bytes = min(512u, wbytes - 512 * issued);
                if (lane == 0) {
                    mbar_arrive_tx(&bar[slot], bytes);
                    tma_load_1d(ring + slot * kChunkWords, words + 512 * issued, bytes, &bar[slot]);
                }
                issued++;
            } while (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots);
        }
        bool need[S];
#pragma unroll
        for (int s = 0; s < S; s++) {
            const uint32_t j = 32 * s + lane, i = t * K + j;
            need[s] = false;
            if (j < K && i < n) {
                const uint32_t e = tab[x[s] & (kM - 1)];
                out[i] = (uint8_t)e;
                const uint32_t q = x[s] >> kProbBits;
                x[s] = ((e >> 8) & 0xfffu) * q + q + (e >> 20);  // f * (x >> 12) + (slot - c)
                need[s] = x[s] < kL;
            }
        }
        // words are taken in stream-lane order j = 0..K-1 within the step
        uint32_t base = p;
#pragma unroll
        for (int s = 0; s < S; s++) {
            const uint32_t b = __ballot_sync(ACX_FULL, need[s]);
            if (need[s]) x[s] = (x[s] << 16) | ring[(rbase + base + __popc(b & lt_mask)) & (kRingWords - 1)];
            base += __popc(b);
        }
        if (base > W) { ok = false; break; }
        p = base;
    }
    // drain chunks still in flight so the barrier phases stay in step
    while (ready < issued) {
        uint32_t q = seq0 + ready;
        uint32_t spins = 0;
        bool w = true;
        while (!mbar_try_wait(&bar[q % kSlots], (q / kSlots) & 1)) {
            if ((++spins & 1023) == 0 && gtimer() > deadline) { w = false; break; }
        }
        if (!__all_sync(ACX_FULL, w)) { ok = false; break; }
        ready++;
    }
    seq = seq0 + issued;
    ok = ok && p == W;
    bool fin = true;
#pragma unroll
    for (int s = 0; s < S; s++) fin = fin && (32 * s + lane >= K || x[s] == kL);
    return __all_sync(ACX_FULL, ok && fin);
}

__device__ void copy_stored(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n, int lane) {
    const uint32_t nv = (n + 15) / 16;  // bodies and scratch streams are 16-aligned and padded
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = lane; i < nv; i += 32) d[i] = s[i];
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

// Start of a decode call: a new epoch tags this call's block states (so the
// state words need no clearing), and every ticket restarts at zero.
__global__ void k_prologue(uint32_t* counters, uint32_t n_counters) {
    for (uint32_t i = threadIdx.x; i < n_counters; i += blockDim.x) {
        if (i == 0) {
            uint32_t e = (counters[0] + 1) & 0x3fffffffu;
            counters[0] = e ? e : 1;
        } else {
            counters[i] = 0;
        }
    }
}

// counters layout: [0] epoch, [1] assembly ticket, [2 + a] rANS ticket of archive a
__global__ void __launch_bounds__(kRansWarps * 32) k_rans(JobDev job) {
    extern __shared__ __align__(128) uint8_t smraw[];
    RansSmem& S = *reinterpret_cast<RansSmem*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kSlots) mbar_init(&S.bar[warp][lane], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (threadIdx.x == 0) {
        // start on the archive holding this CTA's share of the item space
        uint64_t target = (uint64_t)blockIdx.x * job.n_items / gridDim.x;
        S.next_arc = job.n_arcs > 1 ? find_arc(job, (uint32_t)target) : 0;
        S.arc = -1;
    }
    __syncthreads();
    const uint64_t deadline = gtimer() + job.timeout_ns;
    uint32_t seq = 0;
    uint32_t* tickets = job.counters + 2;
    for (;;) {
        const int a = S.next_arc;
        if (a < 0) break;
        const ArcJob J = load_arc(job, a);
        if (S.arc != a) {
            // (all warps are past their use of the previous tables here)
            const uint4* src = reinterpret_cast<const uint4*>(J.dtab);
            uint4* dst = reinterpret_cast<uint4*>(&S.tab[0][0]);
            for (int i = threadIdx.x; i < (int)(4 * kM / 4); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) S.arc = a;
        }
        const uint32_t n_a = J.hi - J.lo;
        for (;;) {
            uint32_t it = 0;
            if (lane == 0) it = atomicAdd(&tickets[a], 1u);
            it = __shfl_sync(ACX_FULL, it, 0);
            if (it >= n_a) break;
            const uint32_t b = J.lo + it;
            const BlockDev& bd = J.blk[b];
            const uint8_t* pay = J.arc + bd.payload;
            uint8_t* scr = J.scratch + bd.scratch;
            bool ok = true;
            int fs = 0;
            for (int s = 0; s < 4 && ok; s++) {
                fs = s;
                const uint32_t n = bd.s_raw[s];
                if (n == 0) continue;
                if (bd.rans_mask & (1u << s)) {
                    const uint32_t K = bd.s_K[s];
                    const uint32_t* tb = &S.tab[s][0];
                    uint8_t* o = scr + bd.s_off[s];
                    const uint8_t* body = pay + bd.s_body[s];
                    if (K <= 32)
                        ok = rans_stream<1>(tb, body, bd.s_enc[s], n, K, o, &S.ring[warp][0], &S.bar[warp][0], seq,
                                            lane, deadline);
                    else if (K == 64)
                        ok = rans_stream<2>(tb, body, bd.s_enc[s], n, K, o, &S.ring[warp][0], &S.bar[warp][0], seq,
                                            lane, deadline);
                    else
                        ok = rans_stream<4>(tb, body, bd.s_enc[s], n, K, o, &S.ring[warp][0], &S.bar[warp][0], seq,
                                            lane, deadline);
                } else {
                    copy_stored(pay + bd.s_body[s], scr + bd.s_off[s], n, lane);
                }
            }
            if (!ok && lane == 0) set_err(job.err, kErrCorrupt, (1 << 24) | fs, b);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // move to the archive with the most remaining blocks
            int best = -1;
            uint32_t best_left = 0;
            for (uint32_t k = 0; k < job.n_arcs; k++) {
                const ArcJob Jk = load_arc(job, (int)k);
                uint32_t taken = *((volatile uint32_t*)&tickets[k]);
                uint32_t n_k = Jk.hi - Jk.lo;
                uint32_t left = taken < n_k ? n_k - taken : 0;
                if (left > best_left) { best_left = left; best = (int)k; }
            }
            S.next_arc = best;
        }
        __syncthreads();
    }
}

// =====================================================================================
// Assembly: parse + literals + matches + cross-block dataflow
// =====================================================================================
constexpr int kAsmThreads = 256;
constexpr int kAsmWarps = kAsmThreads / 32;
constexpr uint64_t kRefTag = 1ull << 63;  // history map entry "copy input entry k"

struct AsmLayout {
    uint32_t out, pend, tpos, tll, tml, tlit, tsrc, tcmd, tstat, lenb, scan, misc, total;
};

__host__ __device__ inline AsmLayout asm_layout(uint32_t T, uint32_t LB) {
    AsmLayout L;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) & ~(align - 1);
        uint32_t r = o;
        o += bytes;
        return r;
    };
    L.out = take(kBlock, 16);
    L.pend = take(kBlock / 8, 16);
    L.tsrc = take(8 * T, 16);
    L.tpos = take(2 * T, 16);
    L.tll = take(2 * T, 16);
    L.tml = take(2 * T, 16);
    L.tlit = take(2 * T, 16);
    L.tcmd = take(T, 16);
    L.tstat = take(T, 16);
    L.lenb = take(LB + 16, 16);
    L.scan = take(kAsmWarps * 4 * 8 + 64, 16);
    L.misc = take(64, 16);
    L.total = (o + 127) & ~127u;
    return L;
}

// Block-wide exclusive scan of up to three u32 values per thread.  Returns
// the per-thread exclusive prefixes and block totals.
__device__ __forceinline__ void block_scan3(uint32_t v[3], uint32_t tot[3], uint32_t* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t y = __shfl_up_sync(ACX_FULL, inc[k], o);
            if (lane >= o) inc[k] += y;
        }
    }
    if (lane == 31) {
        for (int k = 0; k < 3; k++) buf[warp * 3 + k] = inc[k];
    }
    __syncthreads();
    uint32_t wpre[3] = {0, 0, 0}, t[3] = {0, 0, 0};
    for (int w = 0; w < kAsmWarps; w++) {
        for (int k = 0; k < 3; k++) {
            uint32_t s = buf[w * 3 + k];
            if (w < warp) wpre[k] += s;
            t[k] += s;
        }
    }
    for (int k = 0; k < 3; k++) {
        v[k] = wpre[k] + inc[k] - v[k];
        tot[k] = t[k];
    }
    __syncthreads();
}

// History map: 4 entries, each a constant distance or kRefTag|k (copy input k).
struct HMap {
    uint64_t e[4];
};
__device__ __forceinline__ HMap hmap_identity() {
    HMap m;
#pragma unroll
    for (int k = 0; k < 4; k++) m.e[k] = kRefTag | k;
    return m;
}
// (first f, then g)
__device__ __forceinline__ HMap hmap_compose(const HMap& f, const HMap& g) {
    HMap r;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        uint64_t x = g.e[k];
        r.e[k] = (x & kRefTag) ? f.e[x & 3] : x;
    }
    return r;
}
__device__ __forceinline__ HMap hmap_token(uint8_t cmd, uint64_t d_new) {
    HMap m = hmap_identity();
    if (cmd == kNew) {
        m.e[0] = d_new;
        m.e[1] = kRefTag | 0;
        m.e[2] = kRefTag | 1;
        m.e[3] = kRefTag | 2;
    } else if (cmd >= 1 && cmd <= 4) {
        const int j = cmd - 1;  // move entry j to the front
        m.e[0] = kRefTag | j;
        for (int k = 1; k <= 3; k++) m.e[k] = kRefTag | (k <= j ? k - 1 : k);
    }
    return m;
}
__device__ __forceinline__ void hmap_apply(const HMap& m, const uint64_t h[4], uint64_t r[4]) {
#pragma unroll
    for (int k = 0; k < 4; k++) r[k] = (m.e[k] & kRefTag) ? h[m.e[k] & 3] : m.e[k];
}

struct BlkCtx {
    uint64_t B;          // absolute start of the block
    uint32_t R;          // raw length
    uint32_t n;          // tokens
    uint8_t* gout;       // global output of this block
    uint32_t epoch;      // this call's epoch
};

__device__ __forceinline__ bool pend_clear_smem(const uint32_t* pend, uint32_t s, uint32_t e) {
    // bits [s, e) all zero?
    if (s >= e) return true;
    uint32_t w0 = s >> 5, w1 = (e - 1) >> 5;
    for (uint32_t w = w0; w <= w1; w++) {
        uint32_t m = 0xffffffffu;
        if (w == w0) m &= 0xffffffffu << (s & 31);
        if (w == w1) m &= 0xffffffffu >> (31 - ((e - 1) & 31));
        if (((volatile const uint32_t*)pend)[w] & m) return false;
    }
    return true;
}
__device__ __forceinline__ void pend_set_smem(uint32_t* pend, uint32_t s, uint32_t e, bool set) {
    if (s >= e) return;
    uint32_t w0 = s >> 5, w1 = (e - 1) >> 5;
    for (uint32_t w = w0; w <= w1; w++) {
        uint32_t m = 0xffffffffu;
        if (w == w0) m &= 0xffffffffu << (s & 31);
        if (w == w1) m &= 0xffffffffu >> (31 - ((e - 1) & 31));
        if (set) atomicOr(&pend[w], m); else atomicAnd(&pend[w], ~m);
    }
}
__device__ __forceinline__ bool pend_clear_global(const uint32_t* pm, uint32_t s, uint32_t e) {
    if (s >= e) return true;
    uint32_t w0 = s >> 5, w1 = (e - 1) >> 5;
    for (uint32_t w = w0; w <= w1; w++) {
        uint32_t m = 0xffffffffu;
        if (w == w0) m &= 0xffffffffu << (s & 31);
        if (w == w1) m &= 0xffffffffu >> (31 - ((e - 1) & 31));
        if (ld_relaxed_u32(pm + w) & m) return false;
    }
    return true;
}
__device__ __forceinline__ void pend_clear_global_bits(uint32_t* pm, uint32_t s, uint32_t e) {
    if (s >= e) return;
    uint32_t w0 = s >> 5, w1 = (e - 1) >> 5;
    for (uint32_t w = w0; w <= w1; w++) {
        uint32_t m = 0xffffffffu;
        if (w == w0) m &= 0xffffffffu << (s & 31);
        if (w == w1) m &= 0xffffffffu >> (31 - ((e - 1) & 31));
        atomicAnd(pm + w, ~m);
    }
}

// Are the bytes [s, e) (absolute, all in blocks before the current one) final?
__device__ bool ext_ready(const ArcJob& J, uint32_t epoch, uint64_t s, uint64_t e) {
    const uint32_t done = (epoch << 2) | kStComplete, pub = (epoch << 2) | kStPublished;
    for (uint64_t a = s >> 14; a <= (e - 1) >> 14; a++) {
        const uint32_t st = ld_acquire_u32(J.state + a);
        if (st == done || st == kStAlways) continue;
        if (st != pub) return false;
        const uint64_t A = a << 14;
        const uint32_t lo = (uint32_t)((s > A ? s : A) - A);
        const uint32_t hi = (uint32_t)((e < A + kBlock ? e : A + kBlock) - A);
        if (!pend_clear_global(J.pmap + a * (kBlock / 32), lo, hi)) return false;
    }
    __threadfence();
    return true;
}

// Byte at absolute position q: from the shared block copy when q is in the
// current block, else from the global output (L2, bypassing L1).
__device__ __forceinline__ uint8_t src_byte(const ArcJob& J, const BlkCtx& C, const uint8_t* sout, uint64_t q) {
    return q >= C.B ? sout[q - C.B] : ld_cg_u8(J.out + q);
}

// Is every source byte of match (dst, src, ml) final right now?
__device__ __forceinline__ bool match_ready(const ArcJob& J, const BlkCtx& C, const uint32_t* pend, uint64_t dst,
                                            uint64_t src, uint32_t ml) {
    const uint32_t epoch = C.epoch;
    const uint64_t d = dst - src;
    const uint64_t se = src + (d < ml ? d : ml);  // periodic source window [src, se)
    if (se > C.B) {
        const uint64_t s0 = src > C.B ? src : C.B;
        if (!pend_clear_smem(pend, (uint32_t)(s0 - C.B), (uint32_t)(se - C.B))) return false;
    }
    if (src < C.B) {
        if (!ext_ready(J, epoch, src, se < C.B ? se : C.B)) return false;
    }
    return true;
}

__device__ __forceinline__ void match_fill(const ArcJob& J, const BlkCtx& C, uint8_t* sout, uint64_t dst, uint64_t src,
                                           uint32_t ml, bool to_global) {
    const uint64_t d = dst - src;
    const uint32_t o = (uint32_t)(dst - C.B);
    if (d >= ml) {
        for (uint32_t k = 0; k < ml; k++) sout[o + k] = src_byte(J, C, sout, src + k);
    } else {
        const uint32_t dd = (uint32_t)d;
        for (uint32_t k = 0; k < dd; k++) sout[o + k] = src_byte(J, C, sout, src + k);
        for (uint32_t k = dd; k < ml; k++) sout[o + k] = sout[o + k - dd];  // period already in place
    }
    if (to_global) {
        for (uint32_t k = 0; k < ml; k++) C.gout[o + k] = sout[o + k];
    }
}

__global__ void __launch_bounds__(kAsmThreads) k_assemble(JobDev job) {
    extern __shared__ __align__(128) uint8_t sm[];
    const AsmLayout L = asm_layout(job.max_tok, job.max_lenb);
    uint8_t* sout = sm + L.out;
    uint32_t* pend = reinterpret_cast<uint32_t*>(sm + L.pend);
    uint64_t* tsrc = reinterpret_cast<uint64_t*>(sm + L.tsrc);
    uint16_t* tpos = reinterpret_cast<uint16_t*>(sm + L.tpos);
    uint16_t* tll = reinterpret_cast<uint16_t*>(sm + L.tll);
    uint16_t* tml = reinterpret_cast<uint16_t*>(sm + L.tml);
    uint16_t* tlit = reinterpret_cast<uint16_t*>(sm + L.tlit);
    uint8_t* tcmd = sm + L.tcmd;
    uint8_t* tstat = sm + L.tstat;
    uint8_t* lenb = sm + L.lenb;
    uint32_t* scanbuf = reinterpret_cast<uint32_t*>(sm + L.scan);
    volatile uint32_t* misc = reinterpret_cast<volatile uint32_t*>(sm + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t deadline = gtimer() + job.timeout_ns;
    const uint32_t epoch = *((volatile uint32_t*)job.counters);

    for (;;) {
        if (tid == 0) misc[0] = atomicAdd(&job.counters[1], 1u);
        __syncthreads();
        const uint32_t item = misc[0];
        __syncthreads();
        if (item >= job.n_items) return;
        const int a = job.n_arcs > 1 ? find_arc(job, item) : 0;
        const ArcJob J = load_arc(job, a);
        const uint32_t b = J.lo + (item - J.item_base);
        const BlockDev& bd = J.blk[b];
        BlkCtx C;
        C.B = (uint64_t)b * kBlock;
        C.R = bd.raw_len;
        C.n = bd.n_tok;
        C.gout = J.out + C.B;
        C.epoch = epoch;
        const uint8_t* scr = J.scratch + bd.scratch;
        const uint8_t* g_cmd = scr + bd.s_off[kCmd];
        const uint8_t* g_len = scr + bd.s_off[kLen];
        const uint8_t* g_off = scr + bd.s_off[kOff];
        const uint8_t* g_lit = scr + bd.s_off[kLit];
        const uint32_t n = C.n, LB = bd.s_raw[kLen], n_lit = bd.s_raw[kLit], n_new = bd.n_new;
        bool bad = (n > job.max_tok) || (LB > job.max_lenb);
        int stage = bad ? 7 : 0;
        auto mark = [&](bool cond, int st) {
            if (cond && !bad) { bad = true; stage = st; }
        };

        // ---- stage cmd + len bytes, clear the pending bitmap ----
        if (!bad) {
            for (uint32_t i = tid; i < n; i += kAsmThreads) { tcmd[i] = g_cmd[i]; tstat[i] = 0; }
            for (uint32_t i = tid; i < LB; i += kAsmThreads) lenb[i] = g_len[i];
        }
        for (uint32_t i = tid; i < kBlock / 32; i += kAsmThreads) pend[i] = 0;
        if (tid == 0) misc[1] = 0;  // error flag of this block
        __syncthreads();

        // ---- varint boundaries: each byte < 0x80 ends a value ----
        uint32_t v3[3], tot3[3];
        const uint32_t per = (LB + kAsmThreads - 1) / kAsmThreads;
        const uint32_t j0 = min(LB, tid * per), j1 = min(LB, j0 + per);
        {
            uint32_t c = 0;
            bool vbad = false;
            if (!bad)
                for (uint32_t j = j0; j < j1; j++) {
                    const uint8_t by = lenb[j];
                    if (by < 0x80) c++;
                    // a value is at most three bytes: three continuation bytes in a row are invalid
                    if (by >= 0x80 && j >= 2 && lenb[j - 1] >= 0x80 && lenb[j - 2] >= 0x80) vbad = true;
                }
            if (vbad) misc[1] = 1;
            v3[0] = c; v3[1] = 0; v3[2] = 0;
            block_scan3(v3, tot3, scanbuf);
        }
        mark(tot3[0] != 2 * n || (LB > 0 && lenb[LB - 1] >= 0x80) || (LB == 0 && n > 0), 2);
        if (!bad) {
            uint32_t idx = v3[0];
            for (uint32_t j = j0; j < j1; j++) {
                const uint8_t by = lenb[j];
                if (by >= 0x80) continue;
                uint32_t val = by;
                if (j >= 1 && lenb[j - 1] >= 0x80) {
                    val = (val << 7) | (lenb[j - 1] & 0x7f);
                    if (j >= 2 && lenb[j - 2] >= 0x80) val = (val << 7) | (lenb[j - 2] & 0x7f);
                }
                if (val > kBlock) misc[1] = 1;
                const uint32_t tk = idx >> 1;
                if (idx & 1) tml[tk] = (uint16_t)min(val, kBlock); else tll[tk] = (uint16_t)min(val, kBlock);
                idx++;
            }
        }
        __syncthreads();
        mark(misc[1] != 0, 2);

        // ---- token scans: positions, literal positions, NEW indices ----
        const uint32_t tper = (n + kAsmThreads - 1) / kAsmThreads;
        const uint32_t i0 = min(n, tid * tper), i1 = min(n, i0 + tper);
        bool any_rep = false;
        {
            uint32_t s_len = 0, s_ll = 0, s_new = 0;
            bool tbad = false;
            if (!bad)
                for (uint32_t i = i0; i < i1; i++) {
                    const uint32_t ll = tll[i], ml = tml[i], c = tcmd[i];
                    s_len += ll + ml;
                    s_ll += ll;
                    if (c == kNew) s_new++;
                    if (c > kLitOnly) tbad = true;
                    if (c == kLitOnly) { if (ml != 0 || i != n - 1 || ll == 0) tbad = true; }
                    else if (ml < J.min_match) tbad = true;
                    if (c >= 1 && c <= 4) any_rep = true;
                }
            if (tbad) misc[1] = 1;
            v3[0] = s_len; v3[1] = s_ll; v3[2] = s_new;
            block_scan3(v3, tot3, scanbuf);
        }
        mark(tot3[0] != C.R || tot3[1] != n_lit || tot3[2] != n_new || misc[1], 3);
        if (!bad) {
            uint32_t pos = v3[0], lp = v3[1], ni = v3[2];
            for (uint32_t i = i0; i < i1; i++) {
                const uint32_t ll = tll[i], ml = tml[i];
                tpos[i] = (uint16_t)pos;
                tlit[i] = (uint16_t)lp;
                const uint64_t dst = C.B + pos + ll;
                uint64_t src = 0;
                if (tcmd[i] == kNew) {
                    for (int p = 0; p < 5; p++) src |= (uint64_t)g_off[(uint64_t)p * n_new + ni] << (8 * p);
                    ni++;
                    if (src >= dst) misc[1] = 1;  // every absolute offset precedes its destination
                }
                tsrc[i] = src;
                pos += ll + ml;
                lp += ll;
            }
        }
        any_rep = __syncthreads_or(any_rep && !bad);
        mark(misc[1] != 0, 4);

        // ---- 4-entry history as a monoid scan (only if the block has repeat codes) ----
        if (any_rep && !bad) {
            HMap* hbuf = reinterpret_cast<HMap*>(sout);  // the block buffer is free until literal placement
            HMap agg = hmap_identity();
            for (uint32_t i = i0; i < i1; i++) {
                const uint64_t dst = C.B + tpos[i] + tll[i];
                agg = hmap_compose(agg, hmap_token(tcmd[i], dst - tsrc[i]));
            }
            hbuf[tid] = agg;
            __syncthreads();
            // Hillis-Steele inclusive scan over the 256 thread aggregates
            for (int o = 1; o < kAsmThreads; o <<= 1) {
                HMap mine = hbuf[tid];
                HMap prev = tid >= o ? hbuf[tid - o] : hmap_identity();
                __syncthreads();
                if (tid >= o) hbuf[tid] = hmap_compose(prev, mine);
                __syncthreads();
            }
            HMap pre = tid > 0 ? hbuf[tid - 1] : hmap_identity();
            const uint64_t h0[4] = {1, 2, 3, 4};  // initial history, reset per block
            uint64_t h[4];
            hmap_apply(pre, h0, h);
            for (uint32_t i = i0; i < i1; i++) {
                const uint8_t c = tcmd[i];
                const uint64_t dst = C.B + tpos[i] + tll[i];
                if (c == kNew) {
                    const uint64_t d = dst - tsrc[i];
                    h[3] = h[2]; h[2] = h[1]; h[1] = h[0]; h[0] = d;
                } else if (c >= 1 && c <= 4) {
                    const int j = c - 1;
                    const uint64_t d = h[j];
                    if (d < 1 || d > dst) misc[1] = 1;
                    tsrc[i] = dst - d;
                    for (int k = j; k > 0; k--) h[k] = h[k - 1];
                    h[0] = d;
                }
            }
            __syncthreads();
            mark(misc[1] != 0, 4);
        }

        if (!bad) {
            // ---- literal placement: thread t moves literal bytes [64t, 64t+64) ----
            const uint32_t k0 = (uint32_t)tid * 64;
            if (k0 < n_lit) {
                uint4 v[4];
#pragma unroll
                for (int q = 0; q < 4; q++)
                    v[q] = (k0 + 16 * q < n_lit) ? *reinterpret_cast<const uint4*>(g_lit + k0 + 16 * q)
                                                  : make_uint4(0, 0, 0, 0);
                // owner token of literal k0: last i with tlit[i] <= k0 and a non-empty run
                uint32_t lo = 0, hi = n;  // first i with tlit[i] > k0
                while (lo < hi) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (tlit[mid] <= k0) lo = mid + 1; else hi = mid;
                }
                // (tokens sharing a literal position have empty runs except the last one)
                uint32_t i = lo > 0 ? lo - 1 : 0;
                uint32_t end = tlit[i] + tll[i];
                int32_t shift = (int32_t)tpos[i] - (int32_t)tlit[i];
                const uint32_t kend = min(n_lit, k0 + 64);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t w4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                    for (int r = 0; r < 16; r++) {
                        const uint32_t k = k0 + 16 * q + r;
                        if (k < kend) {
                            while (k >= end) {
                                i++;
                                end = tlit[i] + tll[i];
                                shift = (int32_t)tpos[i] - (int32_t)tlit[i];
                            }
                            sout[(int32_t)k + shift] = (uint8_t)(w4[r >> 2] >> (8 * (r & 3)));
                        }
                    }
                }
            }
            // ---- pending bitmap: every match byte starts unresolved ----
            for (uint32_t i = tid; i < n; i += kAsmThreads) {
                const uint32_t ml = tml[i];
                if (ml) {
                    const uint32_t s = tpos[i] + tll[i];
                    pend_set_smem(pend, s, s + ml, true);
                }
            }
        }
        __syncthreads();

        // ---- matches: rounds of ready periodic fills (in-block, and external sources already final) ----
        bool published = false;
        uint32_t rounds = 0;
        if (!bad) {
            for (;;) {
                bool progress = false, left = false;
                for (uint32_t i = tid; i < n; i += kAsmThreads) {
                    const uint32_t ml = tml[i];
                    if (!ml || tstat[i]) continue;
                    const uint64_t dst = C.B + tpos[i] + tll[i], src = tsrc[i];
                    if (match_ready(J, C, pend, dst, src, ml)) {
                        __threadfence_block();  // order the source reads after the readiness reads
                        match_fill(J, C, sout, dst, src, ml, published);
                        if (published) {
                            __threadfence();
                            pend_clear_global_bits(J.pmap + (uint64_t)b * (kBlock / 32), (uint32_t)(dst - C.B),
                                                   (uint32_t)(dst - C.B) + ml);
                        }
                        __threadfence_block();
                        pend_set_smem(pend, (uint32_t)(dst - C.B), (uint32_t)(dst - C.B) + ml, false);
                        tstat[i] = 1;
                        progress = true;
                    } else {
                        left = true;
                    }
                }
                const int any_progress = __syncthreads_or(progress);
                const int any_left = __syncthreads_or(left);
                rounds++;
                if (!any_left) break;
                if (!any_progress) {
                    if (!published) {
                        // publish: the block with its pending map, then resolve the rest as sources arrive
                        uint4* gdst = reinterpret_cast<uint4*>(C.gout);
                        const uint4* ssrc = reinterpret_cast<const uint4*>(sout);
                        const uint32_t nv = (C.R + 15) / 16;
                        for (uint32_t i = tid; i < nv; i += kAsmThreads) {
                            if (16 * (i + 1) <= C.R) gdst[i] = ssrc[i];
                            else for (uint32_t k = 16 * i; k < C.R; k++) C.gout[k] = sout[k];
                        }
                        uint32_t* gp = J.pmap + (uint64_t)b * (kBlock / 32);
                        for (uint32_t i = tid; i < kBlock / 32; i += kAsmThreads) gp[i] = pend[i];
                        __threadfence();
                        __syncthreads();
                        if (tid == 0) st_release_u32(J.state + b, (C.epoch << 2) | kStPublished);
                        published = true;
                    } else {
                        if (tid == 0 && gtimer() > deadline) misc[1] = 2;
                        __nanosleep(200);
                        __syncthreads();
                        if (misc[1] == 2) { mark(true, 5); break; }
                    }
                }
            }
        }
        __syncthreads();
        if (bad) {
            if (tid == 0) set_err(job.err, stage == 5 ? kErrTimeout : kErrCorrupt, stage << 24, b);
        } else if (!published) {
            uint4* gdst = reinterpret_cast<uint4*>(C.gout);
            const uint4* ssrc = reinterpret_cast<const uint4*>(sout);
            const uint32_t nv = (C.R + 15) / 16;
            for (uint32_t i = tid; i < nv; i += kAsmThreads) {
                if (16 * (i + 1) <= C.R) gdst[i] = ssrc[i];
                else for (uint32_t k = 16 * i; k < C.R; k++) C.gout[k] = sout[k];
            }
        }
        __threadfence();
        __syncthreads();
        // a failed block is still marked complete so no other block waits on it forever
        if (tid == 0) st_release_u32(J.state + b, (C.epoch << 2) | kStComplete);
        (void)rounds;
        (void)warp;
        (void)lane;
    }
}

// =====================================================================================
// Plain comparison decoder: one thread per block, sequential parse with the history,
// byte-serial copies; same publish protocol so blocks still overlap.
// =====================================================================================
constexpr int kPlainThreads = 32;

__global__ void __launch_bounds__(kPlainThreads) k_plain(JobDev job, uint32_t max_tok) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* sout = sm;
    uint32_t* pend = reinterpret_cast<uint32_t*>(sm + kBlock);
    uint64_t* dsrc = reinterpret_cast<uint64_t*>(sm + kBlock + kBlock / 8);  // deferred matches
    uint32_t* ddst = reinterpret_cast<uint32_t*>(dsrc + max_tok);
    uint32_t* dml = ddst + max_tok;
    volatile uint32_t* misc = dml + max_tok;
    const int lane = threadIdx.x;
    const uint64_t deadline = gtimer() + job.timeout_ns;
    const uint32_t epoch = *((volatile uint32_t*)job.counters);
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&job.counters[1], 1u);
        item = __shfl_sync(ACX_FULL, item, 0);
        if (item >= job.n_items) return;
        const int a = job.n_arcs > 1 ? find_arc(job, item) : 0;
        const ArcJob J = load_arc(job, a);
        const uint32_t b = J.lo + (item - J.item_base);
        const BlockDev& bd = J.blk[b];
        BlkCtx C;
        C.B = (uint64_t)b * kBlock;
        C.R = bd.raw_len;
        C.n = bd.n_tok;
        C.gout = J.out + C.B;
        C.epoch = epoch;
        for (uint32_t i = lane; i < kBlock / 32; i += 32) pend[i] = 0;
        __syncwarp();
        if (lane == 0) {
            const uint8_t* scr = J.scratch + bd.scratch;
            const uint8_t* cmd = scr + bd.s_off[kCmd];
            const uint8_t* lb = scr + bd.s_off[kLen];
            const uint8_t* off = scr + bd.s_off[kOff];
            const uint8_t* lit = scr + bd.s_off[kLit];
            const uint32_t n = bd.n_tok, LB = bd.s_raw[kLen], n_lit = bd.s_raw[kLit], n_new = bd.n_new;
            uint64_t hist[4] = {1, 2, 3, 4};
            uint64_t pos = C.B, E = C.B + C.R;
            uint32_t lp = 0, ni = 0, vp = 0, nd = 0;
            bool bad = n > max_tok;
            for (uint32_t i = 0; i < n && !bad; i++) {
                uint32_t v[2];
                for (int qv = 0; qv < 2 && !bad; qv++) {
                    uint32_t val = 0;
                    int k = 0;
                    for (;;) {
                        if (vp >= LB || k == 3) { bad = true; break; }
                        const uint8_t c = lb[vp++];
                        val |= (uint32_t)(c & 0x7f) << (7 * k);
                        k++;
                        if (c < 0x80) break;
                    }
                    v[qv] = val;
                }
                if (bad) break;
                const uint32_t LL = v[0], ML = v[1];
                const uint8_t k = cmd[i];
                if (LL > E - pos || LL > n_lit - lp) { bad = true; break; }
                for (uint32_t j = 0; j < LL; j++) sout[pos - C.B + j] = lit[lp + j];
                pos += LL;
                lp += LL;
                uint64_t src = 0;
                if (k == kLitOnly) {
                    if (ML != 0 || i != n - 1 || LL == 0) bad = true;
                    continue;
                } else if (k == kNew) {
                    if (ni >= n_new) { bad = true; break; }
                    for (int p = 0; p < 5; p++) src |= (uint64_t)off[(uint64_t)p * n_new + ni] << (8 * p);
                    ni++;
                    if (src >= pos) { bad = true; break; }
                    hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = pos - src;
                } else if (k <= 4) {
                    const int j = k - 1;
                    const uint64_t d = hist[j];
                    if (d < 1 || d > pos) { bad = true; break; }
                    src = pos - d;
                    for (int q = j; q > 0; q--) hist[q] = hist[q - 1];
                    hist[0] = d;
                } else {
                    bad = true;
                    break;
                }
                if (ML < J.min_match || ML > E - pos) { bad = true; break; }
                if (match_ready(J, C, pend, pos, src, ML)) {
                    const uint32_t o = (uint32_t)(pos - C.B);
                    for (uint32_t j = 0; j < ML; j++) sout[o + j] = src_byte(J, C, sout, src + j);  // byte-serial
                } else {
                    pend_set_smem(pend, (uint32_t)(pos - C.B), (uint32_t)(pos - C.B) + ML, true);
                    dsrc[nd] = src;
                    ddst[nd] = (uint32_t)(pos - C.B);
                    dml[nd] = ML;
                    nd++;
                }
                pos += ML;
            }
            if (!bad && (pos != E || lp != n_lit || ni != n_new || vp != LB)) bad = true;
            misc[0] = bad ? 1 : 0;
            misc[1] = nd;
        }
        __syncwarp();
        const bool bad = misc[0] != 0;
        const uint32_t nd = misc[1];
        // write the block (pending bytes are rewritten when resolved)
        {
            const uint32_t nv = (C.R + 15) / 16;
            uint4* gdst = reinterpret_cast<uint4*>(C.gout);
            const uint4* ssrc = reinterpret_cast<const uint4*>(sout);
            for (uint32_t i = lane; i < nv; i += 32) {
                if (16 * (i + 1) <= C.R) gdst[i] = ssrc[i];
                else for (uint32_t k = 16 * i; k < C.R; k++) C.gout[k] = sout[k];
            }
            if (nd && !bad) {
                uint32_t* gp = J.pmap + (uint64_t)b * (kBlock / 32);
                for (uint32_t i = lane; i < kBlock / 32; i += 32) gp[i] = pend[i];
            }
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            bool bad2 = bad;
            if (nd && !bad) {
                st_release_u32(J.state + b, (C.epoch << 2) | kStPublished);
                for (uint32_t q = 0; q < nd && !bad2; q++) {
                    const uint64_t dst = C.B + ddst[q];
                    uint32_t spins = 0;
                    while (!match_ready(J, C, pend, dst, dsrc[q], dml[q])) {
                        __nanosleep(100);
                        if ((++spins & 63) == 0 && gtimer() > deadline) { bad2 = true; break; }
                    }
                    if (bad2) { set_err(job.err, kErrTimeout, 5 << 24, b); break; }
                    const uint32_t o = ddst[q];
                    for (uint32_t j = 0; j < dml[q]; j++) {
                        const uint8_t by = src_byte(J, C, sout, dsrc[q] + j);
                        sout[o + j] = by;
                        C.gout[o + j] = by;
                    }
                    __threadfence();
                    pend_clear_global_bits(J.pmap + (uint64_t)b * (kBlock / 32), o, o + dml[q]);
                    pend_set_smem(pend, o, o + dml[q], false);
                }
            } else if (bad) {
                set_err(job.err, kErrCorrupt, 6 << 24, b);
            }
            __threadfence();
            st_release_u32(J.state + b, (C.epoch << 2) | kStComplete);
        }
        __syncwarp();
    }
}

// =====================================================================================
// Host-side launch helpers
// =====================================================================================
size_t rans_smem_bytes() { return sizeof(RansSmem); }
size_t asm_smem_bytes(uint32_t T, uint32_t LB) { return asm_layout(T, LB).total; }
size_t plain_smem_bytes(uint32_t T) { return kBlock + kBlock / 8 + (size_t)T * 16 + 64; }

cudaError_t launch_prologue(uint32_t* counters, uint32_t n_counters, cudaStream_t st) {
    k_prologue<<<1, 128, 0, st>>>(counters, n_counters);
    return cudaGetLastError();
}

cudaError_t launch_rans(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = rans_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_rans<<<grid, kRansWarps * 32, sm, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = asm_smem_bytes(job.max_tok, job.max_lenb);
    cudaError_t e = cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_assemble<<<grid, kAsmThreads, sm, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_plain(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = plain_smem_bytes(job.max_tok);
    cudaError_t e = cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_plain<<<grid, kPlainThreads, sm, st>>>(job, job.max_tok);
    return cudaGetLastError();
}

int occupancy(int which, size_t smem) {
    int n = 0;
    cudaError_t e;
    // the dynamic shared-memory limit must be raised before the query
    if (which == 0) cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (which == 1) cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (which == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rans, kRansWarps * 32, smem);
    else if (which == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_assemble, kAsmThreads, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain, kPlainThreads, smem);
    if (e != cudaSuccess) return 0;
    return n;
}

}  // namespace acx
