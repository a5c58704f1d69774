// Device code of the entropy stage of the decode (paper, Table 1/2: "ANS"): interleaved-rANS
// lane decoders for the four per-block streams, one warp per block.
//
// Stream layout (format v1): K initial 32-bit states (padded to 16 B), then
// 16-bit renormalisation words in decode order.  Symbol i belongs to lane
// i mod K; a step decodes one symbol per lane; lanes whose state fell below
// 2^16 take the next words in lane order (ballot + popc gives each its rank).
//
// GB300 mapping:
//  * decode tables of the four stream types (4 x 4096 u32 entries:
//    sym | (f-1) << 8 | (slot-c) << 20) live in shared memory, shared by the
//    16 warps of a CTA;
//  * each warp streams its words through a 2 KiB shared-memory ring filled
//    by 512-byte 1-D TMA bulk copies (cp.async.bulk + mbarrier), kept up to
//    three chunks ahead of the decoder;
//  * K = 64 / 128 lanes run as 2 / 4 independent states per warp lane (ILP);
//  * ring residency is checked once per 8 steps (of 32 symbols), not per step;
//  * the tables and rings are read at 32-bit shared-window addresses, and the
//    renormalisation is branch-free (every lane reads its candidate word).
// Every wait is bounded by %globaltimer.
#pragma once
#include "common.cuh"

namespace acx {

constexpr int kRansWarps = 16;
constexpr int kRingWords = 1024;   // 2 KiB of 16-bit words per warp
constexpr int kRingMask = 2 * kRingWords - 1;  // byte offset within a ring
constexpr int kChunkWords = 256;   // one TMA chunk = 512 B
constexpr int kSlots = kRingWords / kChunkWords;
constexpr int kGroupSyms = 16;     // full steps between ring checks, times the states per lane
constexpr int kStageBytes = 32 * kGroupSyms;  // a warp's symbols of one group, staged for 16-byte stores

struct RansSmem {
    uint32_t tab[4][kM];                               // 64 KiB
    uint16_t ringspace[(kRansWarps + 1) * kRingWords];  // the warps' rings, 2 KiB-aligned in the shared window
    uint64_t bar[kRansWarps][kSlots];
    alignas(16) uint8_t stage[kRansWarps][kStageBytes];
    uint64_t sbar[kRansWarps];                         // short-stream staging barrier of each warp
    int arc;                                           // archive whose tables are loaded
    int next_arc;
};

// Shared-window address of warp w's ring: 2 KiB-aligned, so that a wrapped
// byte offset is OR-ed onto it.
__device__ __forceinline__ uint32_t ring_addr(RansSmem& S, int w) {
    return ((smem_u32(S.ringspace) + kRingMask) & ~(uint32_t)kRingMask) + (uint32_t)w * (2 * kRingWords);
}

__device__ __forceinline__ bool wait_chunk(uint64_t* bar, uint32_t q, uint64_t deadline) {
    uint32_t spins = 0;
    bool ok = true;
    while (!mbar_try_wait(&bar[q % kSlots], (q / kSlots) & 1)) {
        if ((++spins & 1023) == 0 && gtimer() > deadline) { ok = false; break; }
    }
    return __all_sync(ACX_FULL, ok);
}

__device__ __forceinline__ void issue_chunk(uint32_t ring_s, uint64_t* bar, const uint8_t* words, uint32_t q,
                                            uint32_t c, uint32_t wbytes, int lane) {
    if (lane == 0) {
        const uint32_t slot = q % kSlots;
        const uint32_t bytes = min(512u, wbytes - 512 * c);
        mbar_arrive_tx(&bar[slot], bytes);
        tma_load_1d_s(ring_s + slot * 2 * kChunkWords, words + 512 * c, bytes, &bar[slot]);
    }
}

// One rANS symbol of state x with the decode table at shared address tab_s:
// returns the table entry (its low byte is the symbol) and updates x to
// f * (x >> 12) + (x & 4095) - c, stored as (f-1) << 8 and (slot-c) << 20.
__device__ __forceinline__ uint32_t rans_sym(uint32_t tab_s, uint32_t& x) {
    const uint32_t e = lds_u32(tab_s + ((x & (kM - 1)) << 2));
    const uint32_t q = x >> kProbBits;
    x = ((e >> 8) & 0xfffu) * q + q + (e >> 20);
    return e;
}

// Renormalisation of one state per lane, words taken in lane order from the
// ring position rb (byte offset): every lane reads its candidate word and only
// the lanes below 2^16 keep it, so no lane branches.
__device__ __forceinline__ void rans_renorm(uint32_t& x, uint32_t& rb, uint32_t ring_s, uint32_t lt_mask,
                                            uint32_t& p) {
    const bool need = x < kL;
    const uint32_t b = __ballot_sync(ACX_FULL, need);
    const uint32_t w = lds_u16(ring_s | ((rb + 2 * __popc(b & lt_mask)) & (kRingMask - 1)));
    x = need ? (x << 16) | w : x;
    const uint32_t c = __popc(b);
    rb += 2 * c;
    p += c;
}

// Decode one stream with one warp; S states per lane (S = 1 for K <= 32,
// else K / 32).  `seq` counts the TMA chunks this warp has used (slot and
// mbarrier phase bookkeeping across streams).  Returns false on a format
// violation (word overrun, end states != 2^16) or an expired wait.
template <int S>
__device__ __forceinline__ bool rans_stream(uint32_t tab_s, const uint8_t* __restrict__ body, uint32_t enc,
                                            uint32_t n, uint32_t K, uint8_t* __restrict__ out, uint32_t ring_s,
                                            uint32_t stage_s, uint64_t* bar, uint32_t& seq, int lane,
                                            uint64_t deadline) {
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
    // stream sits at byte ((rbase + w) * 2) & kRingMask of the ring
    const uint32_t rbase = (seq0 % kSlots) * kChunkWords;
    uint32_t issued = 0, ready = 0;
    for (; issued < nchunks && issued < (uint32_t)kSlots; issued++)
        issue_chunk(ring_s, bar, words, seq0 + issued, issued, wbytes, lane);
    const uint32_t lt_mask = (1u << lane) - 1;
    uint32_t p = 0;
    const uint32_t steps = ok ? (n + K - 1) / K : 0;
    uint32_t t0 = 0;
    // make words [p, p + need_words) resident, and refill the slots whose chunk
    // lies wholly below p
    auto advance = [&](uint32_t need_words) {
        while (ready < nchunks && ready * kChunkWords < p + need_words) {
            if (!wait_chunk(bar, seq0 + ready, deadline)) { ok = false; return; }
            ready++;
        }
        if (issued < nchunks && kChunkWords * (issued + 1) <= p + kChunkWords * kSlots) {
            __syncwarp();
            do {
                issue_chunk(ring_s, bar, words, seq0 + issued, issued, wbytes, lane);
                issued++;
            } while (issued < nchunks && kChunkWords * (issued + 1) <= p + kChunkWords * kSlots);
        }
    };
    if (K == 32 * S) {
        // Fast path: groups of full steps (every lane valid); a group reads
        // at most 32 * kGroupSyms words.  Its symbols (kStageBytes
        // consecutive bytes of the stream) are staged in shared memory and
        // go out as one 16-byte store per lane.
        constexpr int U = kGroupSyms / S;
        const uint32_t full_groups = ok ? (n / K) / U : 0;
        const uint32_t st_lane = stage_s + lane;
        for (uint32_t g = 0; g < full_groups; g++, t0 += U) {
            advance(32 * kGroupSyms);
            if (!ok) break;
            uint32_t rb = ((rbase + p) * 2) & kRingMask;
#pragma unroll
            for (int u = 0; u < U; u++) {
#pragma unroll
                for (int s = 0; s < S; s++) sts_u8(st_lane + (u * S + s) * 32, rans_sym(tab_s, x[s]));
#pragma unroll
                for (int s = 0; s < S; s++) rans_renorm(x[s], rb, ring_s, lt_mask, p);
            }
            __syncwarp();
            const uint4 v = lds_u128(stage_s + 16 * lane);
            reinterpret_cast<uint4*>(out + (size_t)t0 * (32 * S))[lane] = v;  // (out is 16-aligned)
            __syncwarp();
            if (p > W) { ok = false; break; }
        }
    }
    for (; t0 < steps && ok; t0 += kGroupSyms / S) {
        // the next steps read at most 32 * kGroupSyms words from p on
        advance(32 * kGroupSyms);
        if (!ok) break;
        uint32_t rb = ((rbase + p) * 2) & kRingMask;
#pragma unroll
        for (int u = 0; u < kGroupSyms / S; u++) {
            const uint32_t t = t0 + u;
#pragma unroll
            for (int s = 0; s < S; s++) {
                const uint32_t j = 32 * s + lane, i = t * K + j;
                const bool act = j < K && i < n;
                uint32_t xs = act ? x[s] : kL;  // an idle lane neither decodes nor takes a word
                const uint32_t e = rans_sym(tab_s, xs);
                if (act) {
                    out[i] = (uint8_t)e;
                    x[s] = xs;
                }
            }
            // words are taken in stream-lane order j = 0..K-1 within the step
#pragma unroll
            for (int s = 0; s < S; s++) {
                const uint32_t j = 32 * s + lane;
                const bool act = j < K && t * K + j < n;
                uint32_t xs = act ? x[s] : kL;
                rans_renorm(xs, rb, ring_s, lt_mask, p);
                if (act) x[s] = xs;
            }
        }
        if (p > W) { ok = false; break; }
    }
    // drain chunks still in flight so the barrier phases stay in step
    while (ready < issued) {
        if (!wait_chunk(bar, seq0 + ready, deadline)) { ok = false; break; }
        ready++;
    }
    seq = seq0 + issued;
    ok = ok && p == W;
    bool fin = true;
#pragma unroll
    for (int s = 0; s < S; s++) fin = fin && (32 * s + lane >= K || x[s] == kL);
    return __all_sync(ACX_FULL, ok && fin);
}

// The wide-lane variants are rare (archives encoded with more than 32
// lanes): out of line, so that they do not raise the kernel's register
// pressure.
static __device__ __noinline__ bool rans_stream2(uint32_t tab_s, const uint8_t* body, uint32_t enc, uint32_t n, uint32_t K,
                                          uint8_t* out, uint32_t ring_s, uint32_t stage_s, uint64_t* bar,
                                          uint32_t& seq, int lane, uint64_t deadline) {
    return rans_stream<2>(tab_s, body, enc, n, K, out, ring_s, stage_s, bar, seq, lane, deadline);
}
static __device__ __noinline__ bool rans_stream4(uint32_t tab_s, const uint8_t* body, uint32_t enc, uint32_t n, uint32_t K,
                                          uint8_t* out, uint32_t ring_s, uint32_t stage_s, uint64_t* bar,
                                          uint32_t& seq, int lane, uint64_t deadline) {
    return rans_stream<4>(tab_s, body, enc, n, K, out, ring_s, stage_s, bar, seq, lane, deadline);
}

// The short streams of a block (cmd, len, off) decoded concurrently by one
// warp: stream g runs on lanes [lo_g, lo_g + K_g) with its own word pointer;
// their words are staged whole into the warp's ring by TMA.  Returns 0 on
// success, 1 when the layout does not fit (caller decodes them one by one),
// -1 on a format violation or an expired wait.
__device__ __forceinline__ int rans_short3(uint32_t tab0_s, const BlockDev& bd, const uint8_t* pay, uint8_t* scr,
                                           uint32_t ring_s, uint64_t* sbar, uint32_t& sphase, int lane,
                                           uint64_t deadline) {
    uint32_t lo[3], K[3], W[3], hdr[3], roff[3], nw_bytes[3];
    uint32_t lanes = 0, bytes = 0;
    for (int g = 0; g < 3; g++) {
        K[g] = 0;
        if (!bd.s_raw[g] || !(bd.rans_mask & (1u << g))) continue;
        K[g] = bd.s_K[g];
        if (K[g] > 32) return 1;
        hdr[g] = (4 * K[g] + 15) & ~15u;
        const uint32_t enc = bd.s_enc[g];
        if (enc < hdr[g] || ((enc - hdr[g]) & 1)) return -1;
        W[g] = (enc - hdr[g]) >> 1;
        nw_bytes[g] = (2 * W[g] + 15) & ~15u;
        lo[g] = lanes;
        lanes += K[g];
        roff[g] = bytes;
        bytes += nw_bytes[g];
    }
    if (lanes > 32 || bytes > 2 * kRingWords) return 1;
    if (lanes == 0) return 0;
    // stage every short stream's words
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_tx(sbar, bytes);
        for (int g = 0; g < 3; g++)
            if (K[g] && nw_bytes[g]) tma_load_1d_s(ring_s + roff[g], pay + bd.s_body[g] + hdr[g], nw_bytes[g], sbar);
    }
    int my = -1;
    for (int g = 0; g < 3; g++)
        if (K[g] && lane >= (int)lo[g] && lane < (int)(lo[g] + K[g])) my = g;
    uint32_t x = kL, n = 0, Kg = 1, Wg = 0, gmask = 0, steps = 0, tb_s = tab0_s;
    uint8_t* o = scr;
    const uint32_t j = my >= 0 ? lane - lo[my] : 0;
    bool ok = true;
    uint32_t rb = 0;  // byte position of the group's next word in the ring
    for (int g = 0; g < 3; g++)
        if (K[g]) steps = max(steps, (bd.s_raw[g] + K[g] - 1) / K[g]);
    if (my >= 0) {
        n = bd.s_raw[my];
        Kg = K[my];
        Wg = W[my];
        rb = roff[my];
        gmask = (Kg == 32 ? 0xffffffffu : ((1u << Kg) - 1)) << lo[my];
        o = scr + bd.s_off[my];
        tb_s = tab0_s + my * kM * 4;
        x = *reinterpret_cast<const uint32_t*>(pay + bd.s_body[my] + 4 * j);
        ok = x >= kL;
    }
    {
        uint32_t spins = 0;
        bool w = true;
        while (!mbar_try_wait(sbar, sphase & 1))
            if ((++spins & 1023) == 0 && gtimer() > deadline) { w = false; break; }
        sphase++;
        if (!__all_sync(ACX_FULL, w)) return -1;
    }
    ok = __all_sync(ACX_FULL, ok);
    const uint32_t lt_mask = (1u << lane) - 1;
    uint32_t p = 0;
    // The word pointer p is per stream group, so an overrun (a corrupt
    // stream) is noticed by one group first: the loop ends only on the
    // warp-uniform flag, refreshed every 8 steps, and ring reads stay inside
    // this warp's ring until then.
    bool okw = ok;
    uint32_t i = j;
    for (uint32_t t = 0; t < steps && okw; t++, i += Kg) {
        const bool act = i < n;  // idle lanes (n = 0) never decode
        uint32_t xs = act ? x : kL;
        const uint32_t e = rans_sym(tb_s, xs);
        if (act) o[i] = (uint8_t)e;
        const bool need = act && xs < kL;
        const uint32_t b = __ballot_sync(ACX_FULL, need) & gmask;
        const uint32_t w = lds_u16(ring_s | ((rb + 2 * __popc(b & lt_mask)) & (kRingMask - 1)));
        if (act) x = need ? (xs << 16) | w : xs;
        const uint32_t c = __popc(b);
        rb += 2 * c;
        p += c;
        if ((t & 7) == 7) {
            if (p > Wg) ok = false;
            okw = __all_sync(ACX_FULL, ok);
        }
    }
    if (p > Wg) ok = false;
    ok = __all_sync(ACX_FULL, ok);
    const bool fin = my < 0 || (p == Wg && x == kL);
    __syncwarp();  // the ring is free again for the next stream's copies
    return __all_sync(ACX_FULL, ok && fin) ? 0 : -1;
}

__device__ __forceinline__ void copy_stored(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n, int lane) {
    const uint32_t nv = (n + 15) / 16;  // bodies and scratch streams are 16-aligned and padded
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = lane; i < nv; i += 32) d[i] = s[i];
}

// Entropy-decode one work item's streams (one warp) into its decoded-stream
// scratch: the three short streams together when they fit the warp, then the
// rest one by one (the literal stream is skipped by a parse-only job).
// tab0_s is the shared address of the four decode tables; bar (kSlots
// barriers), sbar, the ring and the symbol stage (kStageBytes, 16-aligned)
// are the warp's own.  A corrupt stream sets the
// job's (and the archive's) error status.
__device__ __forceinline__ void rans_block(const JobDev& job, int a, const ArcJob& J, const ItemRef& ir,
                                           uint32_t tab0_s, uint32_t ring_s, uint32_t stage_s, uint64_t* bar,
                                           uint64_t* sbar, uint32_t& seq, uint32_t& sphase, int lane,
                                           uint64_t deadline) {
    const uint32_t b = ir.blk;
    if (J.items && J.slot && lane == 0) J.slot[b] = ir.slot;  // read by the cross-block pass
    const BlockDev& bd = J.blk[b];
    const uint8_t* pay = J.arc + bd.payload;
    uint8_t* scr = J.scratch + ir.scratch;
    bool ok = true;
    int fs = 0;
    const int sh = rans_short3(tab0_s, bd, pay, scr, ring_s, sbar, sphase, lane, deadline);
    if (sh < 0) ok = false;
    const int n_streams = (job.flags & kJobIndex) ? 3 : 4;  // a parse needs no literals
    for (int s = 0; s < n_streams && ok; s++) {
        if (sh == 0 && s < 3 && (bd.rans_mask & (1u << s))) continue;  // decoded above
        fs = s;
        const uint32_t n = bd.s_raw[s];
        if (n == 0) continue;
        uint8_t* o = scr + bd.s_off[s];
        const uint8_t* body = pay + bd.s_body[s];
        if (bd.rans_mask & (1u << s)) {
            const uint32_t K = bd.s_K[s];
            const uint32_t tb = tab0_s + s * kM * 4;
            if (K <= 32) ok = rans_stream<1>(tb, body, bd.s_enc[s], n, K, o, ring_s, stage_s, bar, seq, lane, deadline);
            else if (K == 64) ok = rans_stream2(tb, body, bd.s_enc[s], n, K, o, ring_s, stage_s, bar, seq, lane, deadline);
            else ok = rans_stream4(tb, body, bd.s_enc[s], n, K, o, ring_s, stage_s, bar, seq, lane, deadline);
        } else {
            copy_stored(body, o, n, lane);
        }
    }
    if (!ok && lane == 0) {
        // a stream fails on a format violation, or on a copy that never landed
        set_err_arc(job, a, gtimer() > deadline ? kErrTimeout : kErrCorrupt, (kStageRans << 24) | fs, b);
        if (job.flags & kJobIndex) J.npend[ir.slot] = 1;  // per-item status of a parse-only job
    }
}

}  // namespace acx
