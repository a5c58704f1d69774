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

#include "common.cuh"
#include "launch.h"

namespace acx {

constexpr int kLocThreads = 128;
constexpr int kLocWarps = kLocThreads / 32;
constexpr uint64_t kRefTag = 1ull << 63;  // history map entry "copy input entry k"

struct LocLayout {
    uint32_t out, pend, tsrc, tpos, tll, tml, tlit, tcmd, tstat, lenb, soff, slit, scan, bar, misc, need, total;
};

__host__ __device__ inline LocLayout loc_layout(uint32_t T, uint32_t LB, bool need) {
    LocLayout L;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) & ~(align - 1);
        const uint32_t r = o;
        o += bytes;
        return r;
    };
    const uint32_t T16 = (T + 15) & ~15u;
    L.out = take(kBlock, 16);
    L.pend = take(kBlock / 8, 16);
    L.tsrc = take(8 * T, 16);
    L.tpos = take(2 * T, 16);
    L.tll = take(2 * T, 16);
    L.tml = take(2 * T, 16);
    L.tlit = take(2 * T, 16);
    L.tcmd = take(T16 + 16, 16);
    L.tstat = take(T16, 16);
    L.lenb = take(((LB + 15) & ~15u) + 16, 16);
    L.soff = take(((5 * T + 15) & ~15u) + 16, 16);
    L.slit = take(kBlock + 16, 16);
    L.scan = take(kLocWarps * 4 * 4 + 64, 16);
    L.bar = take(8, 8);
    L.misc = take(64, 16);
    L.need = need ? take(kBlock / 8, 16) : 0;  // wanted-byte bitmap (jobs with kJobNeed)
    L.total = (o + 127) & ~127u;
    return L;
}

// Literal runs up to this many bytes are copied by one thread (a byte at a
// time, every thread of the CTA on its own run); longer ones by a warp.
constexpr uint32_t kLaneBytes = 32;

// Does the match at [o, o + ml) of a block touch a wanted byte?
__device__ __forceinline__ bool wanted(const uint32_t* need, uint32_t o, uint32_t ml) {
    for (uint32_t w = o >> 5; w <= ((o + ml - 1) >> 5); w++)
        if (need[w] & range_mask(w, o, o + ml)) return true;
    return false;
}

// Block-wide exclusive scan of three u32 values per thread.
__device__ __forceinline__ void block_scan3(uint32_t v[3], uint32_t tot[3], uint32_t* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint32_t y = __shfl_up_sync(ACX_FULL, inc[k], o);
            if (lane >= o) inc[k] += y;
        }
    }
    if (lane == 31)
        for (int k = 0; k < 3; k++) buf[warp * 3 + k] = inc[k];
    __syncthreads();
    uint32_t wpre[3] = {0, 0, 0}, t[3] = {0, 0, 0};
#pragma unroll
    for (int w = 0; w < kLocWarps; w++) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint32_t s = buf[w * 3 + k];
            if (w < warp) wpre[k] += s;
            t[k] += s;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        v[k] = wpre[k] + inc[k] - v[k];
        tot[k] = t[k];
    }
    __syncthreads();
}

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
        const uint64_t x = g.e[k];
        const uint32_t j = (uint32_t)x & 3;
        // f.e[j] by selects, so that the maps stay in registers
        uint64_t v = f.e[0];
        v = j == 1 ? f.e[1] : v;
        v = j == 2 ? f.e[2] : v;
        v = j == 3 ? f.e[3] : v;
        r.e[k] = (x & kRefTag) ? v : x;
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
#pragma unroll
        for (int k = 1; k <= 3; k++) m.e[k] = kRefTag | (k <= j ? k - 1 : k);
    }
    return m;
}

__device__ __forceinline__ bool pend_clear_smem(const uint32_t* pend, uint32_t s, uint32_t e) {
    if (s >= e) return true;
    for (uint32_t w = s >> 5; w <= ((e - 1) >> 5); w++)
        if (((volatile const uint32_t*)pend)[w] & range_mask(w, s, e)) return false;
    return true;
}
__device__ __forceinline__ void pend_update_smem(uint32_t* pend, uint32_t s, uint32_t e, bool set) {
    if (s >= e) return;
    for (uint32_t w = s >> 5; w <= ((e - 1) >> 5); w++) {
        const uint32_t m = range_mask(w, s, e);
        if (set) atomicOr(&pend[w], m); else atomicAnd(&pend[w], ~m);
    }
}

// Literal run: out[b, b+L) = lit[a, a+L) (both in shared memory), one warp,
// 4-byte funnel-shifted words in the middle, bytes at the ragged ends.
__device__ __forceinline__ void copy_run(uint8_t* __restrict__ sout, const uint8_t* __restrict__ lit, uint32_t a,
                                         uint32_t b, uint32_t L, int lane) {
    if (!L) return;
    const uint32_t e = b + L;
    const uint32_t w0 = (b + 3) >> 2, w1 = e >> 2;  // whole words [w0, w1)
    if (w0 >= w1) {
        for (uint32_t x = b + lane; x < e; x += 32) sout[x] = lit[a + (x - b)];
        return;
    }
    if (lane < (int)(4 * w0 - b)) sout[b + lane] = lit[a + lane];
    if (lane < (int)(e - 4 * w1)) sout[4 * w1 + lane] = lit[a + (4 * w1 + lane - b)];
    const uint32_t* lw = reinterpret_cast<const uint32_t*>(lit);
    for (uint32_t w = w0 + lane; w < w1; w += 32) {
        const uint32_t src = a + (4 * w - b);
        const uint32_t lo = lw[src >> 2], hi = lw[(src >> 2) + 1];
        reinterpret_cast<uint32_t*>(sout)[w] = __funnelshift_r(lo, hi, 8 * (src & 3));
    }
}

// Issue the 1-D TMA copies of an item's four decoded streams (16-aligned,
// padded) into the stream buffers (one thread).  Nothing is issued for a
// block beyond the job's shared-memory limits (the caller treats it as bad).
__device__ void stage_streams(const JobDev& job, uint32_t item, uint8_t* tcmd, uint8_t* lenb, uint8_t* soff,
                              uint8_t* slit, uint64_t* bar) {
    const ArcJob J = load_arc(job, find_arc(job, item));
    const ItemRef ir = item_ref(J, item - J.item_base);
    const BlockDev& bd = J.blk[ir.blk];
    const uint32_t n = bd.n_tok, LB = bd.s_raw[kLen], n_new = bd.n_new, n_lit = bd.s_raw[kLit];
    if (n > job.max_tok || LB > job.max_lenb || n_new > job.max_tok) return;
    const uint8_t* scr = J.scratch + ir.scratch;
    const uint32_t sz[4] = {(n + 15) & ~15u, (LB + 15) & ~15u, (5 * n_new + 15) & ~15u, (n_lit + 15) & ~15u};
    uint8_t* dsts[4] = {tcmd, lenb, soff, slit};
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic use of the buffers
    mbar_arrive_tx(bar, sz[0] + sz[1] + sz[2] + sz[3]);
    for (int q = 0; q < 4; q++)
        if (sz[q]) tma_load_1d(dsts[q], scr + bd.s_off[q], sz[q], bar);
}

__global__ void __launch_bounds__(kLocThreads, 5) k_local(JobDev job) {
    extern __shared__ __align__(128) uint8_t sm[];
    const LocLayout L = loc_layout(job.max_tok, job.max_lenb, (job.flags & kJobNeed) != 0);
    uint8_t* sout = sm + L.out;
    uint32_t* need = reinterpret_cast<uint32_t*>(sm + L.need);  // valid in kJobNeed jobs
    uint32_t* pend = reinterpret_cast<uint32_t*>(sm + L.pend);
    uint64_t* tsrc = reinterpret_cast<uint64_t*>(sm + L.tsrc);
    uint16_t* tpos = reinterpret_cast<uint16_t*>(sm + L.tpos);
    uint16_t* tll = reinterpret_cast<uint16_t*>(sm + L.tll);
    uint16_t* tml = reinterpret_cast<uint16_t*>(sm + L.tml);
    uint16_t* tlit = reinterpret_cast<uint16_t*>(sm + L.tlit);
    uint8_t* tcmd = sm + L.tcmd;
    uint8_t* tstat = sm + L.tstat;
    uint8_t* lenb = sm + L.lenb;
    uint8_t* soff = sm + L.soff;
    uint8_t* slit = sm + L.slit;
    uint32_t* scanbuf = reinterpret_cast<uint32_t*>(sm + L.scan);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
    volatile uint32_t* misc = reinterpret_cast<volatile uint32_t*>(sm + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t deadline = gtimer() + job.timeout_ns;
    if (tid == 0) mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t chunk = job.chunk ? job.chunk : 1u;
    uint32_t cnext = 0, cleft = 0;  // the CTA's current run of `chunk` tickets
    uint32_t pf_item = 0xffffffffu;  // item whose streams are already in flight (CTA-uniform)

    for (;;) {
        const bool prefetched = pf_item != 0xffffffffu;
        uint32_t item;
        if (prefetched) {
            item = pf_item;
            pf_item = 0xffffffffu;
        } else {
            if (cleft == 0) {
                if (tid == 0) misc[0] = atomicAdd(&job.counters[1], chunk);
                __syncthreads();
                cnext = misc[0];
                cleft = chunk;
            }
            item = cnext++;
            cleft--;
        }
        if (item >= job.n_items) return;
        const int a = find_arc(job, item);
        const ArcJob J = load_arc(job, a);
        const ItemRef ir = item_ref(J, item - J.item_base);
        const uint32_t b = ir.blk;
        const BlockDev& bd = J.blk[b];
        const uint64_t B = (uint64_t)b * kBlock;
        const uint32_t R = bd.raw_len, n = bd.n_tok, LB = bd.s_raw[kLen], n_lit = bd.s_raw[kLit];
        const uint32_t n_new = bd.n_new;
        bool bad = n > job.max_tok || LB > job.max_lenb || n_new > job.max_tok;
        int stage = bad ? kStageLimits : 0;
        auto mark = [&](bool cond, int st) {
            if (cond && !bad) { bad = true; stage = st; }
        };

        // ---- stage the four decoded streams with 1-D TMA bulk copies (unless
        //      they were prefetched during the previous block) ----
        if (!bad && tid == 0 && !prefetched) stage_streams(job, item, tcmd, lenb, soff, slit, bar);
        for (uint32_t i = tid; i < kBlock / 32; i += kLocThreads) pend[i] = 0;
        if (tid == 0) misc[1] = 0;
        // wanted bytes of this item (all when it names none)
        const bool partial = (job.flags & kJobNeed) && ir.need_n != 0;
        if (partial) {
            for (uint32_t i = tid; i < kBlock / 32; i += kLocThreads) need[i] = 0;
            __syncthreads();
            for (uint32_t q = 0; q < ir.need_n; q++) {
                const uint32_t iv = J.need[ir.need_off + q];
                const uint32_t s0 = iv & 0xffff, e0 = min(iv >> 16, kBlock);
                if (s0 < e0)
                    for (uint32_t w = (s0 >> 5) + tid; w <= ((e0 - 1) >> 5); w += kLocThreads)
                        atomicOr(&need[w], range_mask(w, s0, e0));
            }
        }
        bool timed_out = false;
        if (!bad) {
            uint32_t spins = 0;
            while (!mbar_try_wait(bar, phase & 1))
                if ((++spins & 1023) == 0 && gtimer() > deadline) { timed_out = true; break; }
            phase++;
        }
        if (__syncthreads_or(timed_out)) {
            // a copy that never lands: give up on the decode (the barrier phase is lost)
            if (tid == 0) set_err_arc(job, a, kErrTimeout, kStageWait << 24, b);
            return;
        }

        // ---- varints: each byte < 0x80 ends a value ----
        uint32_t v3[3], tot3[3];
        const uint32_t per = (LB + kLocThreads - 1) / kLocThreads;
        const uint32_t j0 = min(LB, tid * per), j1 = min(LB, j0 + per);
        {
            uint32_t c = 0;
            bool vbad = false;
            if (!bad)
                for (uint32_t j = j0; j < j1; j++) {
                    const uint8_t by = lenb[j];
                    if (by < 0x80) c++;
                    // a value has at most three bytes
                    if (by >= 0x80 && j >= 2 && lenb[j - 1] >= 0x80 && lenb[j - 2] >= 0x80) vbad = true;
                }
            if (vbad) misc[1] = 1;
            v3[0] = c; v3[1] = 0; v3[2] = 0;
            block_scan3(v3, tot3, scanbuf);
        }
        mark(tot3[0] != 2 * n || (LB > 0 && lenb[LB - 1] >= 0x80) || (LB == 0 && n > 0) || misc[1], kStageVarint);
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
        mark(misc[1] != 0, kStageVarint);

        // ---- token scans: positions, literal positions, NEW indices ----
        const uint32_t tper = (n + kLocThreads - 1) / kLocThreads;
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
                    s_new += c == kNew;
                    if (c > kLitOnly) tbad = true;
                    if (c == kLitOnly) { if (ml != 0 || i != n - 1 || ll == 0) tbad = true; }
                    else if (ml < J.min_match) tbad = true;
                    any_rep |= c >= 1 && c <= 4;
                }
            if (tbad) misc[1] = 1;
            v3[0] = s_len; v3[1] = s_ll; v3[2] = s_new;
            block_scan3(v3, tot3, scanbuf);
        }
        mark(tot3[0] != R || tot3[1] != n_lit || tot3[2] != n_new || misc[1], kStageTokens);
        if (!bad) {
            uint32_t pos = v3[0], lp = v3[1], ni = v3[2];
            for (uint32_t i = i0; i < i1; i++) {
                const uint32_t ll = tll[i], ml = tml[i];
                tpos[i] = (uint16_t)pos;
                tlit[i] = (uint16_t)lp;
                uint64_t src = 0;
                if (tcmd[i] == kNew) {
#pragma unroll
                    for (int p = 0; p < 5; p++) src |= (uint64_t)soff[p * n_new + ni] << (8 * p);
                    ni++;
                    if (src >= B + pos + ll) misc[1] = 1;  // every absolute offset precedes its destination
                }
                tsrc[i] = src;
                pos += ll + ml;
                lp += ll;
            }
        }
        any_rep = __syncthreads_or(any_rep && !bad);
        mark(misc[1] != 0, kStageSources);

        // ---- the 4-entry history as a monoid scan (blocks with repeat codes only) ----
        if (any_rep && !bad) {
            HMap* hbuf = reinterpret_cast<HMap*>(sout);  // the block buffer is free until literal placement
            HMap agg = hmap_identity();
            for (uint32_t i = i0; i < i1; i++)
                agg = hmap_compose(agg, hmap_token(tcmd[i], B + tpos[i] + tll[i] - tsrc[i]));
            // inclusive scan of the maps: shuffles inside each warp, then the
            // warps' totals (earlier maps act first)
            HMap inc = agg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                HMap prev;
#pragma unroll
                for (int k = 0; k < 4; k++) prev.e[k] = __shfl_up_sync(ACX_FULL, inc.e[k], o);
                if (lane >= o) inc = hmap_compose(prev, inc);
            }
            if (lane == 31) hbuf[warp] = inc;
            __syncthreads();
            HMap pre = hmap_identity();
            for (int w = 0; w < warp; w++) pre = hmap_compose(pre, hbuf[w]);
            HMap ex;
#pragma unroll
            for (int k = 0; k < 4; k++) ex.e[k] = __shfl_up_sync(ACX_FULL, inc.e[k], 1);
            if (lane > 0) pre = hmap_compose(pre, ex);
            uint64_t h[4];
            const uint64_t h0[4] = {1, 2, 3, 4};  // initial history, reset per block
#pragma unroll
            for (int k = 0; k < 4; k++) h[k] = (pre.e[k] & kRefTag) ? h0[pre.e[k] & 3] : pre.e[k];
            for (uint32_t i = i0; i < i1; i++) {
                const uint8_t c = tcmd[i];
                const uint64_t dst = B + tpos[i] + tll[i];
                if (c == kNew) {
                    h[3] = h[2]; h[2] = h[1]; h[1] = h[0]; h[0] = dst - tsrc[i];
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
            mark(misc[1] != 0, kStageSources);
        }

        // ---- with dependency lists: every block a match reads outside its own
        //      block must be listed (range decodes read only the listed closure) ----
        if (J.deps && !bad) {
            const uint32_t* dl = J.deps + bd.dep_off;
            const uint32_t nd = bd.n_deps;
            bool dbad = false;
            for (uint32_t i = i0; i < i1; i++) {
                const uint32_t ml = tml[i];
                if (!ml || tsrc[i] >= B) continue;
                const uint64_t d = B + tpos[i] + tll[i] - tsrc[i];
                const uint64_t e = tsrc[i] + (d < ml ? d : ml);
                for (uint64_t a = tsrc[i] >> 14; a <= (e - 1) >> 14 && a < b && !dbad; a++)
                    dbad = !listed(dl, nd, (uint32_t)a);
            }
            if (dbad) misc[1] = 1;
            __syncthreads();
            mark(misc[1] != 0, kStageSources);
        }

        if (job.flags & kJobIndex) {
            // parse only: one record per token (source, destination offset,
            // match length, command)
            if (!bad)
                for (uint32_t i = tid; i < n; i += kLocThreads)
                    J.spans[ir.span_base + i] = SpanRec{(uint32_t)tsrc[i], (uint32_t)(tsrc[i] >> 32),
                                                        (uint32_t)(tpos[i] + tll[i]) | ((uint32_t)tml[i] << 16), tcmd[i]};
            if (bad && tid == 0) {
                set_err_arc(job, a, kErrCorrupt, stage << 24, b);
                J.npend[ir.slot] = 1;  // per-item status of a parse-only job
            }
            __syncthreads();
            continue;
        }

        uint32_t npend = 0, pbytes = 0;
        if (!bad) {
            // ---- literal placement: a thread copies a tiny run (<= kLaneBytes)
            //      by itself, all threads at once; a warp copies each longer one ----
            for (uint32_t i = tid; i < n; i += kLocThreads) {
                const uint32_t ll = tll[i];
                if (ll <= kLaneBytes) {
                    const uint32_t la = tlit[i], lb = tpos[i];
                    for (uint32_t k = 0; k < ll; k++) sout[lb + k] = slit[la + k];
                }
            }
            for (uint32_t i = warp; i < n; i += kLocWarps)
                if (tll[i] > kLaneBytes) copy_run(sout, slit, tlit[i], tpos[i], tll[i], lane);
            // ---- every match byte starts unresolved; external sources are pending for good ----
            for (uint32_t i = tid; i < n; i += kLocThreads) {
                const uint32_t ml = tml[i];
                uint8_t st = 0;  // 0: none/done, 1: unresolved in-block, 2: pending
                if (ml) {
                    const uint32_t s = tpos[i] + tll[i];
                    pend_update_smem(pend, s, s + ml, true);
                    st = tsrc[i] >= B ? 1 : 2;
                }
                tstat[i] = st;
            }
            __syncthreads();
            // ---- the stream buffers are free from here on: start the next item's
            //      copies, so that they land while this block finishes ----
            if (cleft == 0) {
                if (tid == 0) misc[0] = atomicAdd(&job.counters[1], chunk);
                __syncthreads();
                cnext = misc[0];
                cleft = chunk;
            }
            pf_item = cnext++;
            cleft--;
            if (tid == 0 && pf_item < job.n_items) stage_streams(job, pf_item, tcmd, lenb, soff, slit, bar);
            // ---- in-block matches: rounds of ready periodic fills; each warp
            //      works on four matches at once, eight lanes per match ----
            for (;;) {
                bool progress = false, left = false;
                const uint32_t g = lane >> 3, sl = lane & 7;
                const uint32_t gmask = 0xffu << (8 * g);
                for (uint32_t base = warp * 4; base < n; base += kLocWarps * 4) {
                    const uint32_t i = base + g;
                    const bool act = i < n && tstat[i] == 1;  // the same for the group's lanes
                    uint32_t ml = 0, o = 0, so = 0, d = 1, we = 0;
                    bool busy = false;
                    if (act) {
                        ml = tml[i];
                        o = tpos[i] + tll[i];
                        so = (uint32_t)(tsrc[i] - B);
                        d = o - so;
                        we = so + min(d, ml);  // periodic source window [so, we)
                        for (uint32_t w = (so >> 5) + sl; w <= ((we - 1) >> 5); w += 8)
                            busy |= (((volatile uint32_t*)pend)[w] & range_mask(w, so, we)) != 0;
                    }
                    const uint32_t bm = __ballot_sync(ACX_FULL, busy);  // every lane, active or not
                    const bool ready = act && (bm & gmask) == 0;
                    if (act && !ready) left = true;
                    __threadfence_block();  // source reads after the readiness reads
                    if (ready) {
                        if (d >= ml) {
                            for (uint32_t k = sl; k < ml; k += 8) sout[o + k] = sout[so + k];
                        } else {
                            // out[o+k] = out[so + (k mod d)]: the source window only, so lanes are independent
                            uint32_t r = sl % d;
                            const uint32_t step = 8 % d;
                            for (uint32_t k = sl; k < ml; k += 8) {
                                sout[o + k] = sout[so + r];
                                r += step;
                                if (r >= d) r -= d;
                            }
                        }
                    }
                    __syncwarp();
                    __threadfence_block();
                    if (ready) {
                        for (uint32_t w = (o >> 5) + sl; w <= ((o + ml - 1) >> 5); w += 8)
                            atomicAnd(&pend[w], ~range_mask(w, o, o + ml));
                        if (sl == 0) tstat[i] = 0;
                        progress = true;
                    }
                }
                const int any_left = __syncthreads_or(left);
                const int any_prog = __syncthreads_or(progress);
                if (!any_left || !any_prog) break;
            }
            // ---- whatever is still unresolved becomes pending pieces (for a
            //      partial item: the wanted matches only) ----
            if (partial)
                for (uint32_t i = i0; i < i1; i++)
                    if (tstat[i] && !wanted(need, tpos[i] + tll[i], tml[i])) tstat[i] = 0;
            uint32_t cnt = 0, nbytes = 0;
            for (uint32_t i = i0; i < i1; i++)
                if (tstat[i]) {
                    cnt += pieces_of(tml[i]);
                    nbytes += tml[i];
                }
            v3[0] = cnt; v3[1] = nbytes; v3[2] = 0;
            block_scan3(v3, tot3, scanbuf);
            npend = tot3[0];
            pbytes = tot3[1];
            uint32_t k = v3[0];
            for (uint32_t i = i0; i < i1; i++) {
                if (!tstat[i]) continue;
                const uint32_t o = tpos[i] + tll[i];
                k += emit_pieces(J.spans + ir.span_base + k, o, tsrc[i], tml[i], B + o - tsrc[i]);
            }
        }
        __syncthreads();
        if (bad) {
            if (tid == 0) set_err_arc(job, a, kErrCorrupt, stage << 24, b);
            npend = 0;
        }
        // ---- write the block (pending bytes are filled by the cross-block pass) ----
        uint8_t* gout = J.out + (uint64_t)ir.slot * kBlock;
        const uint32_t nv = R / 16;
        for (uint32_t i = tid; i < nv; i += kLocThreads) reinterpret_cast<uint4*>(gout)[i] = reinterpret_cast<uint4*>(sout)[i];
        for (uint32_t x = 16 * nv + tid; x < R; x += kLocThreads) gout[x] = sout[x];
        {
            // the pending bitmap is written for every block (all clear when nothing
            // is pending, a corrupt block included), so readers need no second
            // lookup and never wait on a corrupt block
            uint4* gp = reinterpret_cast<uint4*>(J.pmap + (uint64_t)ir.slot * (kBlock / 32));
            const uint4* sp = reinterpret_cast<const uint4*>(pend);
            const uint4* np4 = reinterpret_cast<const uint4*>(need);
            for (uint32_t i = tid; i < kBlock / 128; i += kLocThreads) {
                uint4 v = npend ? sp[i] : make_uint4(0, 0, 0, 0);
                if (partial) {  // unwanted bytes are never read: leave them out of the bitmap
                    const uint4 m = np4[i];
                    v.x &= m.x; v.y &= m.y; v.z &= m.z; v.w &= m.w;
                }
                gp[i] = v;
            }
        }
        if (tid == 0) {
            J.npend[ir.slot] = npend;
            if (npend) {
                atomicAdd(&job.counters[kStatPending], npend);
                atomicAdd(reinterpret_cast<unsigned long long*>(job.counters + kStatPendBytes), (unsigned long long)pbytes);
            }
        }
        __syncthreads();
    }
}

// ---- cross-block pass --------------------------------------------------------------------
// Are the bytes [s, e) (absolute) final?  The local pass writes every
// block's pending-byte bitmap; a clear bit means a final byte.  The loads are
// relaxed: a caller that goes on to read the bytes issues one fence first
// (strong read + fence = acquire pattern), so a failed poll costs no fence.
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
        if (p0 == p1) return (ld_relaxed_u32(p0) & lo0 & hi1) == 0;
        const uint32_t w0 = ld_relaxed_u32(p0), w1 = ld_relaxed_u32(p1);
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
            if (ld_relaxed_u32(pm + w) & range_mask(w, lo, hi)) return false;  // pairs with the fenced clears
    }
    return true;
}

constexpr int kExtThreads = 1024;  // one CTA per SM: grid barriers stay cheap
constexpr uint32_t kRound0WaitNs = 4000;  // wait of a round-0 piece for its sources when they are many
constexpr uint32_t kWaitAllPerLane = 16;   // pieces per grid lane up to which round 0 waits without limit

// Are the bytes a piece reads final?  (period 0: [src, src+len); otherwise the
// residues phase.. of the period window [src, src+period), one or two ranges.)
__device__ __forceinline__ bool piece_final(const ArcJob& L, uint64_t src, uint32_t phase, uint32_t period,
                                            uint32_t len) {
    if (period == 0) return src_final(L, src, src + len);
    if (len >= period) return src_final(L, src, src + period);
    if (phase + len <= period) return src_final(L, src + phase, src + phase + len);
    return src_final(L, src + phase, src + period) && src_final(L, src, src + (phase + len - period));
}

// A warp's attempt at its lanes' pieces (lane `has` a piece `rec` of the
// block in output slot `dslot`, all of archive L).  Each lane checks its own
// piece; the ready pieces are then copied by the whole warp, lane i moving
// byte i (one coalesced request per piece), eight pieces' loads in flight
// before their stores; after one fence (the release) the owners clear the
// pieces' pending bits with relaxed atomic ANDs.  Returns true on the lanes
// whose piece is done.
constexpr int kCopyBatch = 8;
__device__ bool try_pieces(bool has, const ArcJob& L, uint32_t dslot, SpanRec rec, SpanRec* wrec, uint64_t* wdst,
                           int lane) {
    const uint64_t src = (uint64_t)rec.x | ((uint64_t)(rec.y & 0xff) << 32);
    const uint32_t phase = rec.y >> 8, period = rec.w, o = rec.z & 0xffff, len = rec.z >> 16;
    const bool ready = has && piece_final(L, src, phase, period, len);
    const uint32_t rmask = __ballot_sync(ACX_FULL, ready);
    if (!rmask) return false;
    __threadfence();  // acquire: the bitmap reads above are ordered before the source reads below
    wrec[lane] = rec;
    wdst[lane] = (uint64_t)dslot * kBlock + o;
    __syncwarp();
    uint8_t* g = L.out;
    uint32_t m = rmask;
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
                    const uint64_t q = rp ? rs + ((r.y >> 8) + (uint32_t)lane) % rp : rs + lane;
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
    __threadfence();  // release: every lane's stores are visible before any bit is cleared
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

// One pass over work list `in` (n entries) by warps w0, w0 + nw, ...: every
// piece is attempted once; the unfinished ones go to list `out`.
__device__ void round_pass(const JobDev& job, uint32_t in, uint32_t out, uint32_t n, uint32_t w0, uint32_t nw,
                           SpanRec* wrec, uint64_t* wdst, ListEnt* sbuf, int lane) {
    uint32_t sn = 0;
    for (uint32_t i0 = w0 * 32; i0 < n; i0 += nw * 32) {
        const uint32_t i = i0 + lane;
        const bool has = i < n;
        ListEnt e{0, 0};
        if (has) e = job.lists[in][i];
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
        round_pass(job, in, out, n, warp, nw, wrec, wdst, sbuf, lane);
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
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t t = gtimer();
        job.counters[kTrace] = 0;
        job.counters[kTrace + 1] = (uint32_t)t;
        job.counters[kTrace + 2] = (uint32_t)(t >> 32);
    }
    // round 0: pieces handed out in ascending order (the warp takes blocks from
    // a ticket, its idle lanes take the block's next pieces); a lane waits a
    // short while for sources that are about to be finished by lower pieces,
    // then defers its piece to the rounds below.
    {
        // wait_ns 0 (automatic): in output order, waiting pieces cost little
        // while pieces are few per lane of the grid; with many (long, wide
        // chains, e.g. text) waiting lanes would clog the hand-out, so a piece
        // that waited kRound0WaitNs goes to the rounds
        uint64_t wait_ns;
        if (job.wait_ns == 0) {
            const uint64_t pieces = *((volatile uint32_t*)&job.counters[kStatPending]);
            wait_ns = pieces <= kWaitAllPerLane * (uint64_t)gridDim.x * blockDim.x ? ~0ull : kRound0WaitNs;
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
                    if (lane == 0) item = atomicAdd(&job.counters[2], 1u);
                    item = __shfl_sync(ACX_FULL, item, 0);
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
                    l_span = base + next + r;
                    rec = J.spans[l_span];
                    l_blk = blk;
                    l_dsl = dsl;
                    l_item = item;
                    l_arc = arc;
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
        round_pass(job, in, out, n, gwarp, nwarps, wrec, wdst, sbuf, lane);
    }
}

size_t local_smem_bytes(uint32_t T, uint32_t LB, bool need) { return loc_layout(T, LB, need).total; }

cudaError_t launch_local(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = local_smem_bytes(job.max_tok, job.max_lenb, (job.flags & kJobNeed) != 0);
    cudaError_t e = cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // a small job (a seek, a serving tick) needs no more CTAs than ticket runs
    const uint64_t runs = (job.n_items + (uint64_t)(job.chunk ? job.chunk : 1) - 1) / (job.chunk ? job.chunk : 1);
    grid = job_grid(grid, runs);
    k_local<<<grid, kLocThreads, sm, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_external(const JobDev& job, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kExtThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_external, job);
}

int local_occupancy(size_t smem) {
    cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
