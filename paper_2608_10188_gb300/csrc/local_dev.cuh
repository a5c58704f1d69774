// Device code of the local pass of the decode (paper: "parse" and the
// in-block part of "copy"), shared by k_local and the fused decode kernel.
// See assemble.cu for the pass as a whole.
#pragma once
#include "common.cuh"

namespace acx {

constexpr int kLocThreads = 128;
constexpr int kLocWarps = kLocThreads / 32;

struct LocLayout {
    uint32_t out, pend, tsrc, tpos, tll, tml, tlit, tcmd, tstat, lenb, soff, slit, scan, bar, misc, need, tlvl, tlvk,
        lhist, total;
};

// Shared-memory workspace of one local group for blocks of up to T tokens
// and LB length bytes; need: jobs with wanted-byte intervals; lvl: jobs that
// sort pieces by level (the token levels and a level histogram).
__host__ __device__ inline LocLayout loc_layout(uint32_t T, uint32_t LB, bool need, bool lvl = false) {
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
    L.tlvl = lvl ? take(T16 + 16, 16) : 0;       // token levels as staged (jobs with kJobLevels)
    L.tlvk = lvl ? take(T16, 16) : 0;            // the block's token levels, kept past the next block's staging
    L.lhist = lvl ? take(4 * (kMaxLevel + 2), 16) : 0;
    L.total = (o + 127) & ~127u;
    return L;
}

// Literal runs up to this many bytes are copied by one thread (a byte at a
// time, every thread of the CTA on its own run); longer ones by eight lanes.
constexpr uint32_t kLaneBytes = 32;

// Does the match at [o, o + ml) of a block touch a wanted byte?
__device__ __forceinline__ bool wanted(const uint32_t* need, uint32_t o, uint32_t ml) {
    for (uint32_t w = o >> 5; w <= ((o + ml - 1) >> 5); w++)
        if (need[w] & range_mask(w, o, o + ml)) return true;
    return false;
}

// Barriers of one 128-thread group: named barrier `bid` (0 in k_local, where
// the group is the whole CTA; 1.. for the groups of a fused CTA).
__device__ __forceinline__ void grp_sync(uint32_t bid) {
    asm volatile("bar.sync %0, %1;" ::"r"(bid), "n"(kLocThreads) : "memory");
}
__device__ __forceinline__ int grp_or(uint32_t bid, int v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.cta.red.or.pred p, %2, %3, q;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(bid), "n"(kLocThreads)
        : "memory");
    return (int)r;
}

// Group-wide exclusive scan of three u32 values per thread (tid: the thread
// in its group).
__device__ __forceinline__ void block_scan3(uint32_t v[3], uint32_t tot[3], uint32_t* buf, uint32_t bid, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
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
    grp_sync(bid);
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
    grp_sync(bid);
}

// The four-entry distance history ("The Last Sequential Element") as a map
// from the history before a run of tokens to the history after it, packed in
// 64 bits: entry k (bits 16k..16k+15) is kHRef | j, "entry j of the history
// before the run", or the index in the block of the NEW token whose distance
// it holds (a block that passes the token checks has at most kBlock / 4 + 1
// tokens, so an index never reaches kHRef).  Maps compose associatively,
// which makes the history a prefix scan.
typedef uint64_t HMap;
constexpr uint32_t kHRef = 0x8000;
constexpr HMap kHIdentity = 0x8003800280018000ull;

// The map followed by token i with command cmd: a NEW token pushes its own
// distance in front; a repeat of entry j moves that entry to the front.
__device__ __forceinline__ HMap hmap_step(HMap m, uint8_t cmd, uint32_t i) {
    if (cmd == kNew) return (m << 16) | i;
    if (cmd >= 2 && cmd <= 4) {  // entry j = cmd - 1 >= 1 (a repeat of entry 0 changes nothing)
        const uint32_t s = 16 * (cmd - 1);
        const uint64_t low = m & ((1ull << s) - 1);   // entries 0 .. j-1
        const uint64_t e = (m >> s) & 0xffff;          // entry j
        const uint64_t high = s == 48 ? 0ull : m & (~0ull << (s + 16));
        return high | (low << 16) | e;
    }
    return m;
}
// (first f, then g): an entry of g that names entry j of its input takes f's entry j
__device__ __forceinline__ HMap hmap_compose(HMap f, HMap g) {
    const uint32_t flo = (uint32_t)f, fhi = (uint32_t)(f >> 32);
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t x = (uint32_t)(g >> (16 * k)) & 0xffff;
        const uint32_t j = x & 3;
        const uint32_t fj = (j & 2 ? fhi : flo) >> (16 * (j & 1));
        v[k] = (x & kHRef) ? fj & 0xffff : x;
    }
    return (uint64_t)(v[0] | (v[1] << 16)) | ((uint64_t)(v[2] | (v[3] << 16)) << 32);
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

// Run copy out[b, b+L) = src[a, a+L) (both in shared memory, the two ranges
// disjoint: a literal run, or an in-block match at distance >= L), by the
// eight lanes sl = 0..7 of a lane group: 16-byte stores in the middle, each
// from five funnel-shifted source words, bytes at the ragged ends.  Source
// words may reach 3 bytes past the run, still inside the buffer (the literal
// buffer is padded; a match source ends at or before its destination, which
// holds at least 4 bytes); those bytes are shifted out unused.
__device__ __forceinline__ void copy_run8(uint8_t* sout, const uint8_t* lit, uint32_t a, uint32_t b, uint32_t L,
                                          uint32_t sl) {
    const uint32_t e = b + L;
    const uint32_t q0 = (b + 15) >> 4, q1 = e >> 4;  // whole 16-byte chunks [q0, q1)
    if (q0 >= q1) {
        for (uint32_t x = b + sl; x < e; x += 8) sout[x] = lit[a + (x - b)];
        return;
    }
    for (uint32_t x = b + sl; x < 16 * q0; x += 8) sout[x] = lit[a + (x - b)];
    for (uint32_t x = 16 * q1 + sl; x < e; x += 8) sout[x] = lit[a + (x - b)];
    const uint32_t* lw = reinterpret_cast<const uint32_t*>(lit);
    const uint32_t s0 = a + 16 * q0 - b;  // source of chunk q0
    const uint32_t sh = 8 * (s0 & 3);
    for (uint32_t q = q0 + sl; q < q1; q += 8) {
        const uint32_t w = (s0 >> 2) + 4 * (q - q0);
        const uint32_t x0 = lw[w], x1 = lw[w + 1], x2 = lw[w + 2], x3 = lw[w + 3], x4 = lw[w + 4];
        reinterpret_cast<uint4*>(sout)[q] = make_uint4(__funnelshift_r(x0, x1, sh), __funnelshift_r(x1, x2, sh),
                                                       __funnelshift_r(x2, x3, sh), __funnelshift_r(x3, x4, sh));
    }
}

// Issue the 1-D TMA copies of an item's four decoded streams (16-aligned,
// padded) into the stream buffers (one thread).  Nothing is issued for a
// block beyond the job's shared-memory limits (the caller treats it as bad).
__device__ __forceinline__ void stage_streams(const JobDev& job, uint32_t item, uint8_t* tcmd, uint8_t* lenb, uint8_t* soff,
                              uint8_t* slit, uint8_t* tlvl, uint64_t* bar) {
    const ArcJob J = load_arc(job, find_arc(job, item));
    const ItemRef ir = item_ref(J, item - J.item_base);
    const BlockDev& bd = J.blk[ir.blk];
    const uint32_t n = bd.n_tok, LB = bd.s_raw[kLen], n_new = bd.n_new, n_lit = bd.s_raw[kLit];
    if (n > job.max_tok || LB > job.max_lenb || n_new > job.max_tok || n_lit > kBlock) return;
    const uint8_t* scr = J.scratch + ir.scratch;
    const uint32_t sz[4] = {(n + 15) & ~15u, (LB + 15) & ~15u, (5 * n_new + 15) & ~15u, (n_lit + 15) & ~15u};
    uint8_t* dsts[4] = {tcmd, lenb, soff, slit};
    // the level body (stored in the payload, 16-aligned and padded) beside them
    const uint32_t lsz = (job.flags & kJobLevels) && bd.lvl_body ? sz[0] : 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic use of the buffers
    mbar_arrive_tx(bar, sz[0] + sz[1] + sz[2] + sz[3] + lsz);
    for (int q = 0; q < 4; q++)
        if (sz[q]) tma_load_1d(dsts[q], scr + bd.s_off[q], sz[q], bar);
    if (lsz) tma_load_1d(tlvl, J.arc + bd.payload + bd.lvl_body, lsz, bar);
}

// Item -> ticket order of the local pass: tickets are items, except in a
// fused decode, where the local groups follow the entropy warps' hand-out
// order (most symbols first) so that a ticket's streams are decoded early.
__device__ __forceinline__ uint32_t ticket_item(const JobDev& job, uint32_t t) {
    if (t >= job.n_items || !job.ready || !job.one.order) return t;
    return job.one.order[t];
}

// Wait (bounded) until the entropy stage of a fused decode has published
// item's streams; then generic-proxy writes of other SMs are visible to this
// thread's bulk copies.
__device__ __forceinline__ bool wait_ready(const uint32_t* ready, uint32_t item, uint64_t deadline) {
    uint32_t spins = 0;
    while (ld_acquire_u32(ready + item) == 0) {
        __nanosleep(64);
        if ((++spins & 63) == 0 && gtimer() > deadline) return false;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// The local pass of one 128-thread group (k_local: a whole CTA; k_fused: a
// group of a fused CTA) over the job's tickets, with its workspace at sm and
// named barrier bid; tid is the thread's index in its group.
__device__ __forceinline__ void local_worker(const JobDev& job, uint8_t* sm, uint32_t bid, int tid) {
    const bool lvl = (job.flags & kJobLevels) != 0;
    const LocLayout L = loc_layout(job.max_tok, job.max_lenb, (job.flags & kJobNeed) != 0, lvl);
    uint8_t* tlvl = sm + L.tlvl;                                      // valid in kJobLevels jobs
    uint8_t* tlvk = sm + L.tlvk;
    uint32_t* lhist = reinterpret_cast<uint32_t*>(sm + L.lhist);
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
    const int lane = tid & 31, warp = tid >> 5;
    const uint64_t deadline = gtimer() + job.timeout_ns;       // waits on published blocks (fused decodes)
    const uint64_t copy_deadline = gtimer() + kCopyWaitNs;    // waits on this group's own bulk copies
    if (tid == 0) mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    grp_sync(bid);
    uint32_t phase = 0;
    const uint32_t chunk = job.chunk ? job.chunk : 1u;
    uint32_t cnext = 0, cleft = 0;  // the group's current run of `chunk` tickets
    uint32_t pf_item = 0xffffffffu;  // the next item, claimed early (group-uniform)

    for (;;) {
        uint32_t item;
        bool prefetched = false;  // its streams are already in flight
        if (pf_item != 0xffffffffu) {
            item = pf_item;
            prefetched = misc[2] != 0;  // written by the thread that issued the item's copies
            pf_item = 0xffffffffu;
        } else {
            if (cleft == 0) {
                if (tid == 0) misc[0] = atomicAdd(&job.counters[1], chunk);
                grp_sync(bid);
                cnext = misc[0];
                cleft = chunk;
            }
            item = ticket_item(job, cnext++);
            cleft--;
        }
        // the next block's ticket: its atomic goes out now and is read at the
        // prefetch point, so its latency hides behind this block's work
        uint32_t pre_claim = 0;
        bool claimed = cleft == 0;  // group-uniform
        if (claimed && tid == 0) pre_claim = atomicAdd(&job.counters[1], chunk);
        // a block that ends before the prefetch point (corrupt, or a parse-only
        // job) hands the claimed tickets on to the next iteration
        auto settle_claim = [&]() {
            if (!claimed) return;
            if (tid == 0) misc[0] = pre_claim;
            grp_sync(bid);
            cnext = misc[0];
            cleft = chunk;
            claimed = false;
        };
        if (item >= job.n_items) return;
        const int a = find_arc(job, item);
        const ArcJob J = load_arc(job, a);
        const ItemRef ir = item_ref(J, item - J.item_base);
        const uint32_t b = ir.blk;
        const BlockDev& bd = J.blk[b];
        const uint64_t B = (uint64_t)b * kBlock;
        const uint32_t R = bd.raw_len, n = bd.n_tok, LB = bd.s_raw[kLen], n_lit = bd.s_raw[kLit];
        const uint32_t n_new = bd.n_new;
        bool bad = n > job.max_tok || LB > job.max_lenb || n_new > job.max_tok || n_lit > kBlock;
        int stage = bad ? kStageLimits : 0;
        auto mark = [&](bool cond, int st) {
            if (cond && !bad) { bad = true; stage = st; }
        };

        // ---- stage the four decoded streams with 1-D TMA bulk copies (unless
        //      they were prefetched during the previous block) ----
        if (!bad && tid == 0 && !prefetched && (!job.ready || wait_ready(job.ready, item, deadline)))
            stage_streams(job, item, tcmd, lenb, soff, slit, tlvl, bar);
        for (uint32_t i = tid; i < kBlock / 32; i += kLocThreads) pend[i] = 0;
        if (tid == 0) misc[1] = 0;
        // wanted bytes of this item (all when it names none)
        const bool partial = (job.flags & kJobNeed) && ir.need_n != 0;
        if (partial) {
            for (uint32_t i = tid; i < kBlock / 32; i += kLocThreads) need[i] = 0;
            grp_sync(bid);
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
                if ((++spins & 1023) == 0 && gtimer() > copy_deadline) { timed_out = true; break; }
            phase++;
        }
        if (grp_or(bid, timed_out)) {
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
            block_scan3(v3, tot3, scanbuf, bid, tid);
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
        grp_sync(bid);
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
            block_scan3(v3, tot3, scanbuf, bid, tid);
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
        any_rep = grp_or(bid, any_rep && !bad);
        mark(misc[1] != 0, kStageSources);

        // ---- the four-entry history (blocks with repeat codes only) as a
        //      warp-level scan of packed maps by warp 0, while the other warps
        //      place the literals, which need positions only (a parse-only job
        //      places none) ----
        const bool place = !bad && !(job.flags & kJobIndex);
        if (!bad && (any_rep || place)) {
            if (any_rep && warp == 0) {
                const uint32_t per = (n + 31) / 32;
                const uint32_t j0 = min(n, lane * per), j1 = min(n, j0 + per);
                HMap agg = kHIdentity;
                for (uint32_t i = j0; i < j1; i++) agg = hmap_step(agg, tcmd[i], i);
                // inclusive scan of the lanes' maps (earlier maps act first)
                HMap inc = agg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const HMap prev = __shfl_up_sync(ACX_FULL, inc, o);
                    if (lane >= o) inc = hmap_compose(prev, inc);
                }
                const HMap ex = __shfl_up_sync(ACX_FULL, inc, 1);
                const HMap pre = lane > 0 ? ex : kHIdentity;
                // the history before this lane's tokens: the block starts from
                // (1, 2, 3, 4); a NEW token's entry is its distance
                auto entry = [&](int k) -> uint64_t {
                    const uint32_t x = (uint32_t)(pre >> (16 * k)) & 0xffff;
                    return (x & kHRef) ? (uint64_t)((x & 3) + 1) : B + tpos[x] + tll[x] - tsrc[x];
                };
                // the lane's history in four registers (selects, no indexed array)
                uint64_t h0 = entry(0), h1 = entry(1), h2 = entry(2), h3 = entry(3);
                for (uint32_t i = j0; i < j1; i++) {
                    const uint8_t c = tcmd[i];
                    const uint64_t dst = B + tpos[i] + tll[i];
                    if (c == kNew) {
                        h3 = h2; h2 = h1; h1 = h0; h0 = dst - tsrc[i];
                    } else if (c >= 1 && c <= 4) {
                        const uint32_t j = c - 1u;
                        const uint64_t d = j == 0 ? h0 : j == 1 ? h1 : j == 2 ? h2 : h3;
                        if (d < 1 || d > dst) misc[1] = 1;
                        tsrc[i] = dst - d;
                        h3 = j >= 3 ? h2 : h3;
                        h2 = j >= 2 ? h1 : h2;
                        h1 = j >= 1 ? h0 : h1;
                        h0 = d;
                    }
                }
            }
            if (place && (warp > 0 || !any_rep)) {
                // literal placement: a thread copies a tiny run (<= kLaneBytes)
                // by itself, all threads at once; eight lanes copy each longer one
                const int w0 = any_rep ? 1 : 0, nw = kLocWarps - w0;
                for (uint32_t i = tid - 32 * w0; i < n; i += 32 * nw) {
                    const uint32_t ll = tll[i];
                    if (ll <= kLaneBytes) {
                        const uint32_t la = tlit[i], lb = tpos[i];
                        for (uint32_t k = 0; k < ll; k++) sout[lb + k] = slit[la + k];
                    }
                }
                for (uint32_t i = (warp - w0) * 4 + (lane >> 3); i < n; i += nw * 4)
                    if (tll[i] > kLaneBytes) copy_run8(sout, slit, tlit[i], tpos[i], tll[i], lane & 7);
            }
            grp_sync(bid);
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
            grp_sync(bid);
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
            grp_sync(bid);
            settle_claim();
            continue;
        }

        uint32_t npend = 0, pbytes = 0;
        if (!bad) {
            // ---- every match byte starts unresolved; external sources are pending for good;
            //      the in-block matches are listed (the literal positions are dead now) ----
            uint16_t* act_list = tlit;
            if (tid == 0) misc[3] = 0;
            grp_sync(bid);
            for (uint32_t i = tid; i < n; i += kLocThreads) {
                const uint32_t ml = tml[i];
                uint8_t st = 0;  // 0: none/done, 1: unresolved in-block, 2: pending
                if (ml) {
                    const uint32_t s = tpos[i] + tll[i];
                    pend_update_smem(pend, s, s + ml, true);
                    st = tsrc[i] >= B ? 1 : 2;
                    if (st == 1) act_list[atomicAdd((uint32_t*)&misc[3], 1u)] = (uint16_t)i;
                }
                tstat[i] = st;
                if (lvl) tlvk[i] = tlvl[i];  // the staging buffer takes the next block's levels below
            }
            grp_sync(bid);
            // ---- the stream buffers are free from here on: start the next item's
            //      copies, so that they land while this block finishes ----
            settle_claim();
            pf_item = ticket_item(job, cnext++);
            cleft--;
            // (issued by the last warp, which takes the fewest in-block matches
            // below, so that its loads of the next block's descriptor delay the
            // rounds least)
            if (tid == kLocThreads - 32) {
                // in a fused decode, only streams that are already published
                const bool go = pf_item < job.n_items && (!job.ready || ld_acquire_u32(job.ready + pf_item) != 0);
                if (go) {
                    if (job.ready) asm volatile("fence.proxy.async.global;" ::: "memory");
                    stage_streams(job, pf_item, tcmd, lenb, soff, slit, tlvl, bar);
                }
                misc[2] = go;
            }
            // ---- in-block matches: rounds of ready periodic fills over the
            //      listed matches; each warp works on four matches at once,
            //      eight lanes per match ----
            const uint32_t n_act = misc[3];
            for (;;) {
                bool progress = false, left = false;
                const uint32_t g = lane >> 3, sl = lane & 7;
                const uint32_t gmask = 0xffu << (8 * g);
                for (uint32_t base = warp * 4; base < n_act; base += kLocWarps * 4) {
                    const uint32_t i = base + g < n_act ? act_list[base + g] : n;
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
                            copy_run8(sout, sout, so, o, ml, sl);
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
                const int any_left = grp_or(bid, left);
                const int any_prog = grp_or(bid, progress);
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
            block_scan3(v3, tot3, scanbuf, bid, tid);
            npend = tot3[0];
            pbytes = tot3[1];
            if (lvl) {
                // the block's row of the level table (pieces of level <= l,
                // a piece's level being its token's level byte clamped to
                // [1, n_levels]); the pieces themselves stay in output order
                // and carry their level, and the level list is built from
                // them (k_level_fill)
                const uint32_t Lg = job.n_levels;
                for (uint32_t l = tid; l <= Lg; l += kLocThreads) lhist[l] = 0;
                grp_sync(bid);
                for (uint32_t i = i0; i < i1; i++)
                    if (tstat[i]) atomicAdd(&lhist[min(max((uint32_t)tlvk[i], 1u), Lg)], pieces_of(tml[i]));
                grp_sync(bid);
                if (warp == 0) {
                    uint32_t carry = 0;
                    uint32_t* row = job.lvl_tab + (uint64_t)ir.slot * (Lg + 1);
                    for (uint32_t l0 = 0; l0 <= Lg; l0 += 32) {
                        const uint32_t l = l0 + lane;
                        uint32_t inc = l <= Lg ? lhist[l] : 0;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(ACX_FULL, inc, o);
                            if (lane >= o) inc += y;
                        }
                        if (l <= Lg) row[l] = carry + inc;
                        carry += __shfl_sync(ACX_FULL, inc, 31);
                    }
                }
            }
            {
                uint32_t k = v3[0];
                for (uint32_t i = i0; i < i1; i++) {
                    if (!tstat[i]) continue;
                    const uint32_t o = tpos[i] + tll[i];
                    const uint32_t lv = lvl ? min(max((uint32_t)tlvk[i], 1u), job.n_levels) : 0u;
                    k += emit_pieces(J.spans + ir.span_base + k, o, tsrc[i], tml[i], B + o - tsrc[i], lv);
                }
            }
        }
        grp_sync(bid);
        if (bad) {
            if (tid == 0) set_err_arc(job, a, kErrCorrupt, stage << 24, b);
            npend = 0;
            if (lvl)  // an empty row: the level rounds take nothing from this block
                for (uint32_t l = tid; l <= job.n_levels; l += kLocThreads)
                    job.lvl_tab[(uint64_t)ir.slot * (job.n_levels + 1) + l] = 0;
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
        grp_sync(bid);
        settle_claim();
    }
}

}  // namespace acx
