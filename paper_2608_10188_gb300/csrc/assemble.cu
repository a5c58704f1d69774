// Parse and match layer of the decode (paper: "parse" and "copy"), in two
// passes separated by a kernel boundary.
//
// k_local (one CTA of 128 threads per block, persistent, any order):
//   * varint boundaries by compaction: every byte < 0x80 ends a value; a CTA
//     prefix count gives each value its index (LL_i, ML_i).  The paper finds
//     varints make 0.61% of commands sequential in a serial parse ("The Last
//     Sequential Element"); here they are a scan like everything else.
//   * prefix sums of LL+ML, LL and #NEW give every token's output position,
//     literal position and offset index (the paper's 93.94% scan share).
//   * the 4-entry distance history as a monoid scan: each token is a map on
//     the history (NEW pushes a distance, REPk moves entry k to the front);
//     maps compose associatively, so the history before every token is a
//     prefix "sum" too.  Skipped when a block has no repeat code (history-
//     free encoding, where the parse is a dependency-free prefix scan).
//   * literals: runs of up to 32 bytes are copied by one thread each, all
//     threads at once; longer runs by a warp with 4-byte funnel-shifted copies.
//   * matches whose source lies inside the block are periodic fills
//     out[dst+k] = out[src + (k mod d)] ("What Does: Periods, Not Chains"),
//     done in rounds as their sources become final; matches whose source
//     chain leaves the block become pending spans.
//   * the block is written with coalesced 16-byte stores; its pending-byte
//     bitmap and pending spans go beside it.
// k_external (warps take blocks in ascending order, one lane per span):
//   after the kernel boundary every literal and every in-block match byte is
//   final, so a pending span waits only on the spans its source really
//   depends on, which lie at lower positions and were taken earlier: the
//   ascending order makes the bounded waits deadlock-free.  Spans that wait
//   too long (many pieces, long chains) go to work lists, staged per warp in
//   shared memory; barrier-separated rounds walk the lists until they are
//   empty, each round finishing at least the lowest span.
#include <algorithm>

#include <mutex>

#include "launch.h"
#include "local_dev.cuh"

namespace acx {

__global__ void __launch_bounds__(kLocThreads, 6) k_local(JobDev job) {
    extern __shared__ __align__(128) uint8_t sm[];
    local_worker(job, sm, 0, threadIdx.x);
}

// ---- cross-block pass --------------------------------------------------------------------
// Are the bytes [s, e) (absolute) final?  The local pass writes every
// block's pending-byte bitmap; a clear bit means a final byte.  The loads are
// acquire loads: a lane that sees its piece's source bits clear is ordered
// after the release that cleared them, and the warp barrier before the copy
// carries that order to the lanes that read the bytes (no fence per attempt).
// A range of at most 32 bytes (every piece) covers at most two bitmap words,
// possibly of two blocks: both are loaded before either is tested.
__device__ __forceinline__ bool src_final(const ArcJob& L, uint64_t s, uint64_t e) {
    if (e - s <= 32) {
        const uint64_t l = e - 1;
        const uint64_t s0 = slot_of(L, s >> 14), s1 = slot_of(L, l >> 14);
        if (s0 == kNoSlot || s1 == kNoSlot) return false;  // not in this decode's output: never final
        const uint32_t o0 = (uint32_t)(s & (kBlock - 1)), o1 = (uint32_t)(l & (kBlock - 1));
        const uint32_t* p0 = L.pmap + s0 * (kBlock / 32) + (o0 >> 5);
        const uint32_t* p1 = L.pmap + s1 * (kBlock / 32) + (o1 >> 5);
        const uint32_t lo0 = 0xffffffffu << (o0 & 31);         // bits from o0 on in its word
        const uint32_t hi1 = 0xffffffffu >> (31 - (o1 & 31));  // bits up to o1 in its word
        if (p0 == p1) return (ld_acquire_u32(p0) & lo0 & hi1) == 0;
        const uint32_t w0 = ld_acquire_u32(p0), w1 = ld_acquire_u32(p1);
        return ((w0 & lo0) | (w1 & hi1)) == 0;
    }
    for (uint64_t a = s >> 14; a <= (e - 1) >> 14; a++) {
        const uint64_t A = a << 14;
        const uint32_t lo = (uint32_t)((s > A ? s : A) - A);
        const uint32_t hi = (uint32_t)((e < A + kBlock ? e : A + kBlock) - A);
        const uint64_t sl = slot_of(L, a);
        if (sl == kNoSlot) return false;
        const uint32_t* pm = L.pmap + sl * (kBlock / 32);
        for (uint32_t w = lo >> 5; w <= ((hi - 1) >> 5); w++)
            if (ld_acquire_u32(pm + w) & range_mask(w, lo, hi)) return false;  // pairs with the released clears
    }
    return true;
}

constexpr int kExtThreads = 1024;  // one CTA per SM: grid barriers stay cheap
constexpr uint32_t kRound0WaitNs = 4000;  // wait of a round-0 piece for its sources when they are many
constexpr uint32_t kWaitAllPerLane = 16;   // pieces per grid lane up to which round 0 waits without limit,
constexpr uint32_t kWaitAllPerItem = 256;  // ... and per block: a warp holding a block's pieces on long chains
                                           // would stall its hand-out
constexpr uint32_t kLevelWaitNs = 20000;   // wait of a piece handed out in level order

// Are the bytes a piece reads final?  (period 0: [src, src+len); otherwise the
// residues phase.. of the period window [src, src+period), one or two ranges.)
__device__ __forceinline__ bool piece_final(const ArcJob& L, uint64_t src, uint32_t phase, uint32_t period,
                                            uint32_t len) {
    if (period == 0) return src_final(L, src, src + len);
    if (len >= period) return src_final(L, src, src + period);
    if (phase + len <= period) return src_final(L, src + phase, src + phase + len);
    return src_final(L, src + phase, src + period) && src_final(L, src, src + (phase + len - period));
}

constexpr int kCopyBatch = 8;
constexpr int kPlainBatch = 8;  // loads in flight before their stores, published-address copies (16: no faster)
// A warp's attempt at its lanes' pieces (lane `has` a piece `rec` of the
// block in output slot `dslot`, all of archive L).  Each lane checks its own
// piece; the ready pieces are then copied by the whole warp, lane i moving
// byte i (one coalesced request per piece), eight pieces' loads in flight
// before their stores (in a whole-archive job from addresses that the
// pieces' owners publish); after one fence (the release) the owners clear
// the pieces' pending bits with relaxed atomic ANDs.  Returns true on the
// lanes whose piece is done.
__device__ bool try_pieces(bool has, const ArcJob& L, uint32_t dslot, SpanRec rec, SpanRec* wrec, uint64_t* wdst,
                           int lane) {
    const uint64_t src = (uint64_t)rec.x | ((uint64_t)(rec.y & 0xff) << 32);
    const uint32_t phase = (rec.y >> 8) & 0xffff, period = rec.w, o = rec.z & 0xffff, len = rec.z >> 16;
    const bool ready = has && piece_final(L, src, phase, period, len);
    const uint32_t rmask = __ballot_sync(ACX_FULL, ready);
    if (!rmask) return false;
    uint8_t* g = L.out;
    uint32_t m = rmask;
    if (!L.slot) {
        // a whole-archive job (blocks at their own offsets): each ready lane
        // publishes its piece's source and destination addresses, length and
        // period in the slot of its rank among the ready lanes, and the warp
        // walks the slots in order
        const uint8_t** wsa = reinterpret_cast<const uint8_t**>(wrec);  // [rank]: source address
        uint8_t** wda = reinterpret_cast<uint8_t**>(wrec) + 32;         // [rank]: destination address
        uint32_t* wln = reinterpret_cast<uint32_t*>(wdst);              // [rank]: length | phase << 8
        uint32_t* wpp = wln + 32;                                        // [rank]: period | M << 16
        if (ready) {
            const uint32_t r = __popc(rmask & ((1u << lane) - 1));
            wsa[r] = g + src;
            wda[r] = g + (uint64_t)dslot * kBlock + o;
            wln[r] = len | phase << 8;
            // a period below 32 takes the residue by a multiply-shift: for
            // x < 64, (x * ceil(2048 / p)) >> 11 is floor(x / p)
            wpp[r] = period | (period && period < 32 ? ((2047 + period) / period) << 16 : 0u);
        }
        __syncwarp();
        const uint32_t nr = __popc(rmask);
        // the walk is branch-free: predicated loads and stores, selects for
        // the residue of a periodic piece (byte k reads (phase + k) mod period;
        // phase < period, so with a period of 32 or more one subtraction does)
        for (uint32_t b0 = 0; b0 < nr; b0 += kPlainBatch) {
            uint32_t v[kPlainBatch / 4];
#pragma unroll
            for (int u = 0; u < kPlainBatch / 4; u++) v[u] = 0;
            uint32_t mine = 0;  // bit u: this lane moves a byte of piece b0 + u
#pragma unroll
            for (int u = 0; u < kPlainBatch; u++) {
                const uint32_t i = (b0 + u) & 31;
                const uint32_t a = wln[i], pp = wpp[i];
                const uint32_t per = pp & 0xffff, M = pp >> 16, x = (uint32_t)lane + (a >> 8);
                const uint32_t k = M ? x - per * ((x * M) >> 11) : (per && x >= per ? x - per : x);
                const bool p = b0 + u < nr && (uint32_t)lane < (a & 0xff);
                const uint32_t b = p ? (uint32_t)__ldcg(wsa[i] + k) : 0u;
                v[u >> 2] |= b << (8 * (u & 3));
                mine |= (uint32_t)p << u;
            }
#pragma unroll
            for (int u = 0; u < kPlainBatch; u++)
                if (mine >> u & 1) wda[(b0 + u) & 31][lane] = (uint8_t)(v[u >> 2] >> (8 * (u & 3)));
        }
    } else {
        wrec[lane] = rec;
        wdst[lane] = (uint64_t)dslot * kBlock + o;
        __syncwarp();
        while (m) {
            int ls[kCopyBatch];
#pragma unroll
            for (int u = 0; u < kCopyBatch; u++) {
                ls[u] = m ? __ffs(m) - 1 : -1;
                if (m) m &= m - 1;
            }
            uint32_t v[(kCopyBatch + 3) / 4];
#pragma unroll
            for (int u = 0; u < (kCopyBatch + 3) / 4; u++) v[u] = 0;
#pragma unroll
            for (int u = 0; u < kCopyBatch; u++) {
                if (ls[u] >= 0) {
                    const SpanRec r = wrec[ls[u]];
                    if ((uint32_t)lane < (r.z >> 16)) {
                        const uint64_t rs = (uint64_t)r.x | ((uint64_t)(r.y & 0xff) << 32);
                        const uint32_t rp = r.w;
                        const uint64_t q = rp ? rs + (((r.y >> 8) & 0xffff) + (uint32_t)lane) % rp : rs + lane;
                        v[u >> 2] |= (uint32_t)__ldcg(g + out_off(L, q)) << (8 * (u & 3));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kCopyBatch; u++) {
                if (ls[u] >= 0) {
                    const uint32_t rl = wrec[ls[u]].z >> 16;
                    if ((uint32_t)lane < rl) g[wdst[ls[u]] + lane] = (uint8_t)(v[u >> 2] >> (8 * (u & 3)));
                }
            }
        }
    }
    // release: every lane's stores (to other lanes' pieces too) happen before
    // the warp's fence, and the fence before any owner clears its bits
    __syncwarp();
    fence_acq_rel_gpu();
    if (ready) {
        uint32_t* pm = L.pmap + (uint64_t)dslot * (kBlock / 32);
        for (uint32_t w = o >> 5; w <= ((o + len - 1) >> 5); w++) red_and_relaxed(pm + w, ~range_mask(w, o, o + len));
    }
    __syncwarp();
    return ready;
}

// Grid-wide barrier of a cooperative launch (every CTA resident): bounded
// wait; the last CTA to arrive clears the count `reset` before it releases
// the others.  Returns false when the wait ran out.
__device__ bool grid_barrier(uint32_t* counters, uint32_t reset, uint64_t deadline) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        ok_s = 1;
        const uint32_t gen = ld_acquire_u32(counters + kBarGen);
        __threadfence();
        if (atomicAdd(counters + kBarCount, 1u) == gridDim.x - 1) {
            counters[kBarCount] = 0;
            counters[reset] = 0;
            __threadfence();
            atomicAdd(counters + kBarGen, 1u);
        } else {
            uint32_t spins = 0;
            while (ld_acquire_u32(counters + kBarGen) == gen) {
                __nanosleep(32);
                if ((++spins & 255) == 0 && gtimer() > deadline) { ok_s = 0; break; }
            }
        }
    }
    __syncthreads();
    return ok_s != 0;
}

// Appends to a work list go through a per-warp staging buffer in shared
// memory: the list's count is one word that every warp of the grid would
// otherwise hit with an atomic at every step, so a warp reserves space for
// kStage entries at a time.  `sn` (warp-uniform) counts the staged entries.
typedef JobDev::ListEnt ListEnt;
constexpr uint32_t kStage = 64;
__device__ __forceinline__ void stage_flush(ListEnt* buf, uint32_t& sn, ListEnt* list, uint32_t* cnt, int lane) {
    if (sn == 0) return;
    __syncwarp();
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(cnt, sn);
    base = __shfl_sync(ACX_FULL, base, 0);
    for (uint32_t i = lane; i < sn; i += 32) list[base + i] = buf[i];
    __syncwarp();
    sn = 0;
}
__device__ __forceinline__ void append(bool keep, ListEnt e, ListEnt* buf, uint32_t& sn, ListEnt* list, uint32_t* cnt,
                                       int lane) {
    const uint32_t m = __ballot_sync(ACX_FULL, keep);
    if (!m) return;
    if (sn + __popc(m) > kStage) stage_flush(buf, sn, list, cnt, lane);
    if (keep) buf[sn + __popc(m & ((1u << lane) - 1))] = e;
    sn += __popc(m);
}

// Round trace (diagnostics): work-list size and start time (ns) of every round.
__device__ __forceinline__ void trace_round(const JobDev& job, uint32_t round, uint32_t n) {
    if (round >= kTraceRounds) return;
    job.counters[kTrace + 3 * round] = n;
    const uint64_t t = gtimer();
    job.counters[kTrace + 3 * round + 1] = (uint32_t)t;
    job.counters[kTrace + 3 * round + 2] = (uint32_t)(t >> 32);
}

// A round that finished no piece.  In a valid archive the lowest pending
// piece always has final sources (every source precedes its destination), so
// the pieces left wait on bytes that no piece writes: their archives are
// corrupt.
__device__ void report_stalled(const JobDev& job, uint32_t in, uint32_t n, uint32_t w0, uint32_t nw, int lane) {
    for (uint32_t i = w0 * 32 + lane; i < n; i += nw * 32) {
        const ListEnt e = job.lists[in][i];
        const int a = find_arc(job, e.y);
        const ArcJob J = load_arc(job, a);
        set_err_arc(job, a, kErrCorrupt, kStageSources << 24, item_ref(J, e.y - J.item_base).blk);
    }
}

// One pass over a list of n pieces (a work list, or a level's segment of the
// level list) by warps w0, w0 + nw, ...: every piece is attempted once; the
// unfinished ones go to work list `out`.
__device__ void round_pass(const JobDev& job, const ListEnt* src, uint32_t out, uint32_t n, uint32_t w0, uint32_t nw,
                           SpanRec* wrec, uint64_t* wdst, ListEnt* sbuf, int lane) {
    uint32_t sn = 0;
    for (uint32_t i0 = w0 * 32; i0 < n; i0 += nw * 32) {
        const uint32_t i = i0 + lane;
        const bool has = i < n;
        ListEnt e{0, 0};
        if (has) e = src[i];
        // (the lanes' pieces may come from several archives: one archive at a time)
        const int arc_i = has ? find_arc(job, e.y) : -1;
        bool done = false;
        uint32_t todo = __ballot_sync(ACX_FULL, has);
        while (todo) {
            const int a0 = __shfl_sync(ACX_FULL, arc_i, __ffs(todo) - 1);
            const bool mine = has && arc_i == a0;
            const ArcJob J = load_arc(job, a0);
            SpanRec r{0, 0, 0, 0};
            if (mine) r = J.spans[e.x];
            const bool d2 = try_pieces(mine, J, mine ? item_ref(J, e.y - J.item_base).slot : 0, r, wrec, wdst, lane);
            if (mine) done = d2;
            todo &= ~__ballot_sync(ACX_FULL, mine);
        }
        append(has && !done, e, sbuf, sn, job.lists[out], &job.counters[kListCnt + out], lane);
    }
    stage_flush(sbuf, sn, job.lists[out], &job.counters[kListCnt + out], lane);
}

// The last rounds on one CTA (the other CTAs have left): list `in` holds n
// entries and the count of the other list is zero.  Rounds are separated by
// CTA barriers; the same progress argument as the grid rounds ends them.
constexpr uint32_t kSoloMax = 4 * kExtThreads;  // lists up to four CTA-wide passes
__device__ void solo_rounds(const JobDev& job, uint32_t in, uint32_t n, uint32_t round, uint64_t deadline,
                            SpanRec* wrec, uint64_t* wdst, ListEnt* sbuf, int lane) {
    __shared__ uint32_t n_next;
    const uint32_t warp = threadIdx.x >> 5, nw = kExtThreads / 32;
    for (;;) {
        const uint32_t out = in ^ 1u;
        round_pass(job, job.lists[in], out, n, warp, nw, wrec, wdst, sbuf, lane);
        __syncthreads();  // every append of this round is visible to the CTA
        if (threadIdx.x == 0) {
            n_next = *((volatile uint32_t*)&job.counters[kListCnt + out]);
            job.counters[kListCnt + in] = 0;  // list `in` becomes the next output
            trace_round(job, ++round, n_next);
            if (n_next) atomicAdd(&job.counters[kStatPolls], 1u);
        }
        __syncthreads();
        const uint32_t m = n_next;
        if (m == 0) return;
        if (m == n) {
            report_stalled(job, out, m, warp, nw, lane);
            return;
        }
        if (__syncthreads_or(gtimer() > deadline)) {
            if (threadIdx.x == 0) set_err(job.err, kErrTimeout, kStageWait << 24, 0);
            return;
        }
        in = out;
        n = m;
    }
}

// The level list of a level-ordered decode (whole single-archive jobs with
// kJobLevels), built between the local pass and the cross-block pass, so
// that round l walks a contiguous segment with one piece per lane however
// unevenly the level's pieces are spread over the blocks.
//   lvl_off[(l-1) * n + b]: offset of item b's level-l pieces in level l's
//     segment (k_level_scan: one CTA per level, an exclusive scan over items);
//   lvl_off[Lg * n + l - 1]: level l's total; lvl_off[Lg * n + Lg + l - 1]:
//     its segment's base (l = 1 .. Lg + 1, the last being the list's length);
//   lvl_list[base(l) + offset + k] = {span slot, item} of the item's k-th
//     level-l piece in output order (k_level_fill: one warp per item, reading
//     each piece's level from its record).
constexpr int kScanThreads = 1024;
// Does the cross-block pass hand pieces out in level order?  Only in jobs
// with level tables, and under the automatic policy only when pieces are
// many per lane of the pass: with few, output order with waits that last as
// long as needed resolves the chains at the latency of one copy per level and
// needs no list.  Every kernel after the local pass reads the same final
// count, so they all decide alike.
__device__ __forceinline__ bool few_pieces(const JobDev& job, uint64_t lanes) {
    const uint64_t pieces = *((volatile const uint32_t*)&job.counters[kStatPending]);
    return pieces <= kWaitAllPerLane * lanes && pieces <= (uint64_t)kWaitAllPerItem * job.n_items;
}
__device__ __forceinline__ bool use_level_order(const JobDev& job) {
    if (!job.lvl_tab) return false;
    if (job.wait_ns != 0) return true;
    return !few_pieces(job, job.lvl_min_pieces / kWaitAllPerLane);
}

// A decode whose local pass timed out left blocks unprocessed, so their level
// rows, piece counts and records may be stale: the passes after it do nothing.
__device__ __forceinline__ bool local_pass_timed_out(const JobDev& job) {
    return *((volatile const int*)job.err) == kErrTimeout;
}

__global__ void __launch_bounds__(kScanThreads) k_level_scan(JobDev job) {
    __shared__ uint32_t wsum[kScanThreads / 32];
    if (local_pass_timed_out(job) || !use_level_order(job)) return;
    const uint32_t l = blockIdx.x + 1, Lg = job.n_levels, n = job.n_items;
    const uint32_t per = (n + kScanThreads - 1) / kScanThreads;
    const uint32_t i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
    auto cnt = [&](uint32_t b) {
        const uint32_t* row = job.lvl_tab + (uint64_t)(job.one.lo + b) * (Lg + 1);
        return row[l] - row[l - 1];
    };
    uint32_t s = 0;
    for (uint32_t b = i0; b < i1; b++) s += cnt(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(ACX_FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
        if (w < warp) pre += wsum[w];
        tot += wsum[w];
    }
    uint32_t off = pre + inc - s;
    uint32_t* out = job.lvl_off + (uint64_t)(l - 1) * n;
    for (uint32_t b = i0; b < i1; b++) {
        out[b] = off;
        off += cnt(b);
    }
    if (threadIdx.x == 0) job.lvl_off[(uint64_t)Lg * n + (l - 1)] = tot;  // level l's total
}

__global__ void __launch_bounds__(256) k_level_fill(JobDev job) {
    __shared__ uint32_t base[kMaxLevel + 1];
    __shared__ uint32_t cursor[8][kMaxLevel + 1];  // per warp: the block's entries written so far, per level
    if (local_pass_timed_out(job) || !use_level_order(job)) return;
    const uint32_t Lg = job.n_levels, n = job.n_items;
    const uint32_t* tot = job.lvl_off + (uint64_t)Lg * n;
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        for (uint32_t l = 1; l <= Lg; l++) {
            base[l - 1] = c;
            c += tot[l - 1];
        }
        base[Lg] = c;
    }
    __syncthreads();
    if (blockIdx.x == 0)  // segment bases, read by the cross-block pass
        for (uint32_t l = threadIdx.x; l <= Lg; l += blockDim.x)
            job.lvl_off[(uint64_t)Lg * n + Lg + l] = base[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1;
    uint32_t* cur = cursor[warp];
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    for (uint32_t b = blockIdx.x * (blockDim.x >> 5) + warp; b < n; b += nw) {
        const uint32_t blk = job.one.lo + b;
        const uint32_t* row = job.lvl_tab + (uint64_t)blk * (Lg + 1);
        const uint32_t total = row[Lg];
        if (total == 0) continue;  // no pending pieces
        const BlockDev& bd = job.one.blk[blk];
        const uint32_t sb = bd.span_base;
        if (total > bd.n_tok + kSpanSlack) {  // more pieces than the block's slots: not this decode's row
            if (lane == 0) set_err(job.err, kErrCorrupt, kStageLimits << 24, blk);
            continue;
        }
        for (uint32_t l = lane; l <= Lg; l += 32) cur[l] = 0;
        __syncwarp();
        // the block's pieces in output order, each to its level's segment
        bool bad = false;
        for (uint32_t k0 = 0; k0 < total; k0 += 32) {
            const uint32_t k = k0 + lane;
            const bool has = k < total;
            const uint32_t l = has ? min(max(job.one.spans[sb + k].y >> 24, 1u), Lg) : 0u;
            const uint32_t peers = __match_any_sync(ACX_FULL, has ? l : 0xffffffffu);
            if (has) {
                const uint32_t r = cur[l] + __popc(peers & lt);
                const uint64_t at = (uint64_t)base[l - 1] + job.lvl_off[(uint64_t)(l - 1) * n + b] + r;
                if (r >= row[l] - row[l - 1] || at >= job.lvl_cap) bad = true;
                else job.lvl_list[at] = JobDev::ListEnt{sb + k, b};
            }
            __syncwarp();
            if (has && (peers & lt) == 0) cur[l] += __popc(peers);  // the group's first lane
            __syncwarp();
        }
        if (__any_sync(ACX_FULL, bad) && lane == 0) set_err(job.err, kErrCorrupt, kStageLimits << 24, blk);
    }
}

uint32_t lvl_auto_min_pieces_for(int ext_ctas) { return kWaitAllPerLane * (uint32_t)ext_ctas * kExtThreads; }

cudaError_t launch_level_list(const JobDev& job, cudaStream_t st) {
    k_level_scan<<<job.n_levels, kScanThreads, 0, st>>>(job);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t grid = std::max(1u, std::min(4096u, (job.n_items + 7) / 8));
    k_level_fill<<<grid, 256, 0, st>>>(job);
    return cudaGetLastError();
}

// Cross-block pass in rounds.  Round 0 walks every block's pending spans (in
// ascending order); each later round walks the spans the previous round could
// not finish.  A span is attempted once per round and never waited on, so
// the pass needs no ordering argument: every round finishes at least the
// lowest pending span (its sources are final), and the number of rounds is
// the depth of the cross-block dependency chains.  Spans finished earlier in
// the same round are visible to later ones.  Rounds are separated by a grid
// barrier (cooperative launch).
__global__ void __launch_bounds__(kExtThreads) k_external(JobDev job) {
    __shared__ SpanRec recs[kExtThreads];
    __shared__ uint64_t dsts[kExtThreads];
    __shared__ ListEnt stage[kExtThreads / 32][kStage];
    SpanRec* wrec = recs + (threadIdx.x & ~31u);
    uint64_t* wdst = dsts + (threadIdx.x & ~31u);
    ListEnt* sbuf = stage[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t deadline = gtimer() + job.timeout_ns;
    if (local_pass_timed_out(job)) return;  // (every CTA returns: no barrier is entered)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t t = gtimer();
        job.counters[kTrace] = 0;
        job.counters[kTrace + 1] = (uint32_t)t;
        job.counters[kTrace + 2] = (uint32_t)(t >> 32);
    }
    // round 0: pieces handed out in order; a lane waits a short while for
    // sources that lower pieces are about to finish, then defers its piece to
    // the rounds below.  The order is the output order (warps take blocks from
    // a ticket, idle lanes take the block's next pieces), or, for a
    // level-ordered job, the level list's (warps take 32 entries at a time):
    // every level's pieces come after all pieces of the levels below, so with
    // true level hints a lane only waits for pieces already handed out (the
    // paper's waves, without a barrier between them).
    {
        const bool lv = use_level_order(job);
        uint32_t n_lv = 0;
        if (lv) {
            n_lv = job.lvl_off[(uint64_t)job.n_levels * job.n_items + 2 * job.n_levels];  // the list's length
            if (n_lv > job.lvl_cap) {
                if (threadIdx.x == 0) set_err(job.err, kErrCorrupt, kStageLimits << 24, 0);
                n_lv = 0;
            }
        }
        // wait_ns 0 (automatic): in output order, waiting pieces cost little
        // while pieces are few per lane of the grid; with many (long, wide
        // chains, e.g. text) waiting lanes would clog the hand-out, so a piece
        // that waited kRound0WaitNs goes to the rounds; in level order a piece
        // waits at most kLevelWaitNs
        uint64_t wait_ns;
        if (job.wait_ns == 0) {
            wait_ns = lv ? kLevelWaitNs : few_pieces(job, (uint64_t)gridDim.x * blockDim.x) ? ~0ull : kRound0WaitNs;
        } else {
            wait_ns = job.wait_ns == 0xffffffffu ? ~0ull : job.wait_ns;
        }
        uint32_t blk = 0, dsl = 0, cnt = 0, next = 0, base = 0, item = 0;
        int arc = 0;
        bool exhausted = false;
        ArcJob J = load_arc(job, 0);
        bool has = false;
        SpanRec rec{0, 0, 0, 0};
        uint32_t l_blk = 0, l_dsl = 0, l_span = 0, l_item = 0;
        int l_arc = 0;
        uint64_t t0 = 0;
        uint32_t spins = 0, nap = 64;
        uint32_t sn0 = 0;  // entries staged for list 0
        const uint32_t lt_mask = (1u << lane) - 1;
        for (;;) {
            uint32_t idle = __ballot_sync(ACX_FULL, !has);
            while (idle && !exhausted) {
                if (next >= cnt) {
                    if (lv) {
                        // the next 32 entries of the level list: chunk t * kLvStripes + k
                        // from stripe k's counter, so that the hand-out is not one
                        // counter's atomics in a row (the order stays the list's, up to
                        // how far the stripes drift apart)
                        const uint32_t k = (threadIdx.x >> 5) & (kLvStripes - 1);  // (with 32 warps a CTA: every stripe in every CTA)
                        if (lane == 0) item = atomicAdd(&job.counters[kLvTickets + k], 1u);
                        item = (__shfl_sync(ACX_FULL, item, 0) * kLvStripes + k) * 32;
                    } else {
                        if (lane == 0) item = atomicAdd(&job.counters[2], 1u);
                        item = __shfl_sync(ACX_FULL, item, 0);
                    }
                    if (lv) {
                        if (item >= n_lv) { exhausted = true; break; }
                        base = item;
                        cnt = min(32u, n_lv - item);
                        next = 0;
                        continue;
                    }
                    if (item >= job.n_items) { exhausted = true; break; }
                    arc = find_arc(job, item);
                    J = load_arc(job, arc);
                    const ItemRef ir = item_ref(J, item - J.item_base);
                    blk = ir.blk;
                    dsl = ir.slot;
                    cnt = J.npend[dsl];
                    next = 0;
                    base = ir.span_base;
                    continue;
                }
                const uint32_t avail = cnt - next;
                const uint32_t r = __popc(idle & lt_mask);
                if ((idle >> lane & 1) && r < avail) {
                    if (lv) {
                        const ListEnt e = job.lvl_list[base + next + r];
                        l_span = e.x;
                        l_item = e.y;
                        l_blk = J.lo + e.y;  // a whole-archive job: item i is block lo + i, in slot lo + i
                        l_dsl = l_blk;
                        l_arc = 0;
                    } else {
                        l_span = base + next + r;
                        l_blk = blk;
                        l_dsl = dsl;
                        l_item = item;
                        l_arc = arc;
                    }
                    rec = J.spans[l_span];
                    t0 = gtimer();
                    has = true;
                }
                next += min(avail, (uint32_t)__popc(idle));
                idle = __ballot_sync(ACX_FULL, !has);
            }
            if (!__any_sync(ACX_FULL, has)) break;
            // attempt the held pieces, one archive at a time
            bool progressed = false;
            uint32_t todo = __ballot_sync(ACX_FULL, has);
            while (todo) {
                const int a0 = __shfl_sync(ACX_FULL, l_arc, __ffs(todo) - 1);
                const bool mine = has && l_arc == a0;
                const bool done = try_pieces(mine, load_arc(job, a0), l_dsl, rec, wrec, wdst, lane);
                if (done) { has = false; progressed = true; }
                todo &= ~__ballot_sync(ACX_FULL, mine);
            }
            // give up on pieces that waited too long: the rounds finish them
            const bool giveup = has && gtimer() - t0 > wait_ns;
            append(giveup, ListEnt{l_span, l_item}, sbuf, sn0, job.lists[0], &job.counters[kListCnt], lane);
            if (giveup) has = false;
            if (__any_sync(ACX_FULL, progressed || giveup)) {
                spins = 0;
                nap = 64;
            } else {
                __nanosleep(nap);
                if (wait_ns == ~0ull) nap = min(2 * nap, 1024u);  // long waits: fewer polls of the bitmaps
                if ((++spins & 255) == 0 && __any_sync(ACX_FULL, gtimer() > deadline)) {
                    if (lane == 0) set_err_arc(job, l_arc, kErrTimeout, kStageWait << 24, l_blk);
                    break;
                }
            }
        }
        stage_flush(sbuf, sn0, job.lists[0], &job.counters[kListCnt], lane);
    }
    uint32_t n_prev = 0xffffffffu;
    for (uint32_t round = 1;; round++) {
        const uint32_t in = (round - 1) & 1, out = round & 1;
        if (!grid_barrier(job.counters, kListCnt + out, deadline)) {
            if (threadIdx.x == 0) set_err(job.err, kErrTimeout, kStageWait << 24, 0);
            return;
        }
        const uint32_t n = *((volatile uint32_t*)&job.counters[kListCnt + in]);
        if (blockIdx.x == 0 && threadIdx.x == 0) trace_round(job, round, n);
        if (n == 0) return;
        if (n == n_prev) {
            report_stalled(job, in, n, gwarp, nwarps, lane);
            return;
        }
        n_prev = n;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&job.counters[kStatPolls], 1u);
        if (n <= kSoloMax) {
            // a short list: one CTA finishes the remaining rounds with CTA
            // barriers instead of grid barriers
            if (blockIdx.x == 0) solo_rounds(job, in, n, round, deadline, wrec, wdst, sbuf, lane);
            return;
        }
        round_pass(job, job.lists[in], out, n, gwarp, nwarps, wrec, wdst, sbuf, lane);
    }
}

size_t local_smem_bytes(uint32_t T, uint32_t LB, bool need, bool lvl) { return loc_layout(T, LB, need, lvl).total; }

cudaError_t launch_local(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = local_smem_bytes(job.max_tok, job.max_lenb, (job.flags & kJobNeed) != 0,
                                       (job.flags & kJobLevels) != 0);
    cudaError_t e = cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)  // the whole unified L1 as shared memory: CTAs per SM are set by their workspaces
        e = cudaFuncSetAttribute(k_local, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // a small job (a seek, a serving tick) needs no more CTAs than ticket runs
    const uint64_t runs = (job.n_items + (uint64_t)(job.chunk ? job.chunk : 1) - 1) / (job.chunk ? job.chunk : 1);
    grid = job_grid(grid, runs);
    k_local<<<grid, kLocThreads, sm, st>>>(job);
    return cudaGetLastError();
}

// Cooperative launches (the cross-block pass, the fused decode) run one at a
// time on a device.  A cooperative grid waits at its grid barriers (and its
// lanes on one another's pieces) for CTAs that must all be resident; two such
// grids launched on different streams, each holding part of the SMs, could
// wait for CTAs that cannot start until the other grid ends.  So every
// cooperative launch of the process waits for the completion event of the
// previous one on the same device and records it anew.  A stream that is
// being captured into a graph is left alone (its graph runs its passes on one
// stream).
namespace {
std::mutex g_coop_mu;
constexpr int kCoopDevices = 64;
cudaEvent_t g_coop_ev[kCoopDevices] = {};
}  // namespace

cudaError_t coop_ordered(cudaStream_t st, cudaError_t (*launch)(void*), void* arg) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if (cs != cudaStreamCaptureStatusNone || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCoopDevices)
        return launch(arg);
    std::lock_guard<std::mutex> g(g_coop_mu);
    cudaEvent_t& ev = g_coop_ev[dev];
    if (!ev) {
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            ev = nullptr;
            return e;
        }
    } else if ((e = cudaStreamWaitEvent(st, ev, 0)) != cudaSuccess) {
        return e;
    }
    if ((e = launch(arg)) != cudaSuccess) return e;
    return cudaEventRecord(ev, st);
}

cudaError_t launch_external(const JobDev& job, int grid, cudaStream_t st) {
    struct Arg {
        const JobDev* job;
        int grid;
        cudaStream_t st;
    } a{&job, grid, st};
    return coop_ordered(st, [](void* p) -> cudaError_t {
        const Arg* a = static_cast<const Arg*>(p);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(a->grid);
        cfg.blockDim = dim3(kExtThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = a->st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_external, *a->job);
    }, &a);
}

int local_occupancy(size_t smem) {
    cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_local, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_local, kLocThreads, smem) != cudaSuccess) return 0;
    return n;
}

int external_occupancy() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_external, kExtThreads, 0) != cudaSuccess) return 0;
    return n;
}

}  // namespace acx
