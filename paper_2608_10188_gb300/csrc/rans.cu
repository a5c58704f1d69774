// Entropy stage of the decode (paper, Table 1/2: "ANS"): interleaved-rANS
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
//  * ring residency is checked once per 4 steps, not per step.
// Every wait is bounded by %globaltimer.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "launch.h"

namespace acx {

constexpr int kRansWarps = 16;
constexpr int kRingWords = 1024;   // 2 KiB of 16-bit words per warp
constexpr int kChunkWords = 256;   // one TMA chunk = 512 B
constexpr int kSlots = kRingWords / kChunkWords;
constexpr int kStepGroup = 4;      // steps between ring checks

struct RansSmem {
    uint32_t tab[4][kM];                     // 64 KiB
    uint16_t ring[kRansWarps][kRingWords];   // 32 KiB
    uint64_t bar[kRansWarps][kSlots];
    uint64_t sbar[kRansWarps];               // short-stream staging barrier of each warp
    int arc;                                 // archive whose tables are loaded
    int next_arc;
};

__device__ __forceinline__ bool wait_chunk(uint64_t* bar, uint32_t q, uint64_t deadline) {
    uint32_t spins = 0;
    bool ok = true;
    while (!mbar_try_wait(&bar[q % kSlots], (q / kSlots) & 1)) {
        if ((++spins & 1023) == 0 && gtimer() > deadline) { ok = false; break; }
    }
    return __all_sync(ACX_FULL, ok);
}

__device__ __forceinline__ void issue_chunk(uint16_t* ring, uint64_t* bar, const uint8_t* words, uint32_t q,
                                            uint32_t c, uint32_t wbytes, int lane) {
    if (lane == 0) {
        const uint32_t slot = q % kSlots;
        const uint32_t bytes = min(512u, wbytes - 512 * c);
        mbar_arrive_tx(&bar[slot], bytes);
        tma_load_1d(ring + slot * kChunkWords, words + 512 * c, bytes, &bar[slot]);
    }
}

// Decode one stream with one warp; S states per lane (S = 1 for K <= 32,
// else K / 32).  `seq` counts the TMA chunks this warp has used (slot and
// mbarrier phase bookkeeping across streams).  Returns false on a format
// violation (word overrun, end states != 2^16) or an expired wait.
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
    for (; issued < nchunks && issued < (uint32_t)kSlots; issued++)
        issue_chunk(ring, bar, words, seq0 + issued, issued, wbytes, lane);
    const uint32_t lt_mask = (1u << lane) - 1;
    uint32_t p = 0;
    const uint32_t steps = ok ? (n + K - 1) / K : 0;
    uint32_t t0 = 0;
    if (K == 32 * S) {
        // Fast path: whole groups of full steps (every lane valid), with
        // immediate store offsets and the ring position kept in one register.
        const uint32_t full_groups = ok ? (n / K) / kStepGroup : 0;
        uint8_t* op = out + lane;
        for (uint32_t g = 0; g < full_groups; g++, t0 += kStepGroup) {
            while (ready < nchunks && ready * kChunkWords < p + kStepGroup * 32 * S) {
                if (!wait_chunk(bar, seq0 + ready, deadline)) { ok = false; break; }
                ready++;
            }
            if (!ok) break;
            if (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots) {
                __syncwarp();
                do {
                    issue_chunk(ring, bar, words, seq0 + issued, issued, wbytes, lane);
                    issued++;
                } while (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots);
            }
            uint8_t* og = op + t0 * (32 * S);
            uint32_t rp = rbase + p;
#pragma unroll
            for (int u = 0; u < kStepGroup; u++) {
#pragma unroll
                for (int s = 0; s < S; s++) {
                    const uint32_t e = tab[x[s] & (kM - 1)];
                    og[(u * S + s) * 32] = (uint8_t)e;
                    const uint32_t q = x[s] >> kProbBits;
                    x[s] = ((e >> 8) & 0xfffu) * q + q + (e >> 20);
                }
#pragma unroll
                for (int s = 0; s < S; s++) {
                    const bool need = x[s] < kL;
                    const uint32_t b = __ballot_sync(ACX_FULL, need);
                    if (need) x[s] = (x[s] << 16) | ring[(rp + __popc(b & lt_mask)) & (kRingWords - 1)];
                    rp += __popc(b);
                }
            }
            p = rp - rbase;
            if (p > W) { ok = false; break; }
        }
    }
    for (; t0 < steps; t0 += kStepGroup) {
        // the next kStepGroup steps read at most kStepGroup * 32 * S words from p on
        while (ready < nchunks && ready * kChunkWords < p + kStepGroup * 32 * S) {
            if (!wait_chunk(bar, seq0 + ready, deadline)) { ok = false; break; }
            ready++;
        }
        if (!ok) break;
        // refill slots whose previous chunk lies wholly below p
        if (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots) {
            __syncwarp();
            do {
                issue_chunk(ring, bar, words, seq0 + issued, issued, wbytes, lane);
                issued++;
            } while (issued < nchunks && 256 * (issued + 1) <= p + 256 * kSlots);
        }
#pragma unroll
        for (int u = 0; u < kStepGroup; u++) {
            const uint32_t t = t0 + u;
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
#pragma unroll
            for (int s = 0; s < S; s++) {
                const uint32_t b = __ballot_sync(ACX_FULL, need[s]);
                if (need[s]) x[s] = (x[s] << 16) | ring[(rbase + p + __popc(b & lt_mask)) & (kRingWords - 1)];
                p += __popc(b);
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

// The short streams of a block (cmd, len, off) decoded concurrently by one
// warp: stream g runs on lanes [lo_g, lo_g + K_g) with its own word pointer;
// their words are staged whole into the warp's ring by TMA.  Returns 0 on
// success, 1 when the layout does not fit (caller decodes them one by one),
// -1 on a format violation or an expired wait.
__device__ int rans_short3(const uint32_t* __restrict__ tab, const BlockDev& bd, const uint8_t* pay, uint8_t* scr,
                           uint16_t* ring, uint64_t* sbar, uint32_t& sphase, int lane, uint64_t deadline) {
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
            if (K[g] && nw_bytes[g])
                tma_load_1d(reinterpret_cast<uint8_t*>(ring) + roff[g], pay + bd.s_body[g] + hdr[g], nw_bytes[g], sbar);
    }
    int my = -1;
    for (int g = 0; g < 3; g++)
        if (K[g] && lane >= (int)lo[g] && lane < (int)(lo[g] + K[g])) my = g;
    uint32_t x = 0, n = 0, Kg = 1, Wg = 0, ro = 0, gmask = 0, steps = 0;
    uint8_t* o = nullptr;
    const uint32_t* tb = tab;
    const uint32_t j = my >= 0 ? lane - lo[my] : 0;
    bool ok = true;
    for (int g = 0; g < 3; g++)
        if (K[g]) steps = max(steps, (bd.s_raw[g] + K[g] - 1) / K[g]);
    if (my >= 0) {
        n = bd.s_raw[my];
        Kg = K[my];
        Wg = W[my];
        ro = roff[my] / 2;
        gmask = (Kg == 32 ? 0xffffffffu : ((1u << Kg) - 1)) << lo[my];
        o = scr + bd.s_off[my];
        tb = tab + my * kM;
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
    for (uint32_t t = 0; t < steps && okw; t++) {
        const uint32_t i = t * Kg + j;
        bool need = false;
        if (my >= 0 && i < n) {
            const uint32_t e = tb[x & (kM - 1)];
            o[i] = (uint8_t)e;
            const uint32_t q = x >> kProbBits;
            x = ((e >> 8) & 0xfffu) * q + q + (e >> 20);
            need = x < kL;
        }
        const uint32_t b = __ballot_sync(ACX_FULL, need) & gmask;
        if (need) x = (x << 16) | ring[(ro + p + __popc(b & lt_mask)) & (kRingWords - 1)];
        p += __popc(b);
        if (p > Wg) ok = false;
        if ((t & 7) == 7) okw = __all_sync(ACX_FULL, ok);
    }
    ok = __all_sync(ACX_FULL, ok);
    const bool fin = my < 0 || (p == Wg && x == kL);
    __syncwarp();  // the ring is free again for the next stream's copies
    return __all_sync(ACX_FULL, ok && fin) ? 0 : -1;
}

__device__ void copy_stored(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n, int lane) {
    const uint32_t nv = (n + 15) / 16;  // bodies and scratch streams are 16-aligned and padded
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = lane; i < nv; i += 32) d[i] = s[i];
}

// Start of a decode call: every ticket and statistic restarts at zero.
__global__ void k_prologue(uint32_t* counters, uint32_t n_counters, int* errs, uint32_t n_errs) {
    for (uint32_t i = threadIdx.x; i < n_counters; i += blockDim.x) counters[i] = 0;
    for (uint32_t i = threadIdx.x; i < n_errs; i += blockDim.x) errs[i] = 0;
    if (threadIdx.x == 0) {
        counters[kStatPending] = 0;
        counters[kStatPolls] = 0;
        counters[kListCnt] = 0;
        counters[kListCnt + 1] = 0;
        counters[kBarCount] = 0;
        counters[kStatPendBytes] = 0;
        counters[kStatPendBytes + 1] = 0;
    }
}

// Each CTA works on one archive at a time (its tables in shared memory);
// its warps take blocks of that archive from the archive's ticket, and when
// the archive is exhausted the CTA moves to the archive with the most blocks
// left.
__global__ void __launch_bounds__(kRansWarps * 32) k_rans(JobDev job) {
    extern __shared__ __align__(128) uint8_t smraw[];
    RansSmem& S = *reinterpret_cast<RansSmem*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kSlots) mbar_init(&S.bar[warp][lane], 1);
    if (lane == kSlots) mbar_init(&S.sbar[warp], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (threadIdx.x == 0) {
        const uint64_t target = (uint64_t)blockIdx.x * job.n_items / gridDim.x;
        S.next_arc = job.n_arcs > 1 ? find_arc(job, (uint32_t)target) : 0;
        S.arc = -1;
    }
    __syncthreads();
    const uint64_t deadline = gtimer() + job.timeout_ns;
    uint32_t seq = 0, sphase = 0;
    uint32_t* tickets = job.counters + 3;
    for (;;) {
        const int a = S.next_arc;
        if (a < 0) break;
        const ArcJob J = load_arc(job, a);
        if (S.arc != a) {
            const uint4* src = reinterpret_cast<const uint4*>(J.dtab);
            uint4* dst = reinterpret_cast<uint4*>(&S.tab[0][0]);
            for (int i = threadIdx.x; i < (int)(4 * kM / 4); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) S.arc = a;
        }
        const uint32_t n_a = J.hi - J.lo;
        const uint32_t chunk = job.chunk ? job.chunk : 1u;
        uint32_t cnext = 0, cleft = 0;  // this warp's current run of `chunk` tickets
        for (;;) {
            if (cleft == 0) {
                uint32_t t0 = 0;
                if (lane == 0) t0 = atomicAdd(&tickets[a], chunk);
                cnext = __shfl_sync(ACX_FULL, t0, 0);
                cleft = chunk;
            }
            const uint32_t tk = cnext++;
            cleft--;
            if (tk >= n_a) break;
            const ItemRef ir = item_ref(J, J.order ? J.order[tk] : tk);
            const uint32_t b = ir.blk;
            if (J.items && J.slot && lane == 0) J.slot[b] = ir.slot;  // read by the cross-block pass
            const BlockDev& bd = J.blk[b];
            const uint8_t* pay = J.arc + bd.payload;
            uint8_t* scr = J.scratch + ir.scratch;
            bool ok = true;
            int fs = 0;
            // the three short streams together when they fit one warp
            const int sh = rans_short3(&S.tab[0][0], bd, pay, scr, &S.ring[warp][0], &S.sbar[warp], sphase, lane,
                                       deadline);
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
                    const uint32_t* tb = &S.tab[s][0];
                    uint16_t* ring = &S.ring[warp][0];
                    uint64_t* bar = &S.bar[warp][0];
                    if (K <= 32) ok = rans_stream<1>(tb, body, bd.s_enc[s], n, K, o, ring, bar, seq, lane, deadline);
                    else if (K == 64) ok = rans_stream<2>(tb, body, bd.s_enc[s], n, K, o, ring, bar, seq, lane, deadline);
                    else ok = rans_stream<4>(tb, body, bd.s_enc[s], n, K, o, ring, bar, seq, lane, deadline);
                } else {
                    copy_stored(body, o, n, lane);
                }
            }
            if (!ok && lane == 0) {
                set_err_arc(job, a, kErrCorrupt, (kStageRans << 24) | fs, b);
                if (job.flags & kJobIndex) J.npend[ir.slot] = 1;  // per-item status of a parse-only job
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int best = -1;
            uint32_t best_left = 0;
            for (uint32_t k = 0; k < job.n_arcs; k++) {
                const ArcJob Jk = load_arc(job, (int)k);
                const uint32_t taken = *((volatile uint32_t*)&tickets[k]);
                const uint32_t n_k = Jk.hi - Jk.lo;
                const uint32_t left = taken < n_k ? n_k - taken : 0;
                if (left > best_left) { best_left = left; best = (int)k; }
            }
            S.next_arc = best;
        }
        __syncthreads();
    }
}

size_t rans_smem_bytes() { return sizeof(RansSmem); }

static std::atomic<int> g_sm_count{0};

void note_sm_count(int n_sms) { g_sm_count.store(n_sms); }

int job_grid(int full, uint64_t need) {
    const int n_sms = std::max(g_sm_count.load(), 1);
    const uint64_t g = std::max<uint64_t>(need, (uint64_t)n_sms);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)full, g));
}

cudaError_t launch_prologue(uint32_t* counters, uint32_t n_counters, cudaStream_t st, int* errs, uint32_t n_errs) {
    k_prologue<<<1, 128, 0, st>>>(counters, n_counters, errs, n_errs);
    return cudaGetLastError();
}

cudaError_t launch_rans(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = rans_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // a small job needs no more CTAs than its warps can take ticket runs
    const uint64_t per_cta = (uint64_t)kRansWarps * (job.chunk ? job.chunk : 1);
    grid = job_grid(grid, (job.n_items + per_cta - 1) / per_cta);
    k_rans<<<grid, kRansWarps * 32, sm, st>>>(job);
    return cudaGetLastError();
}

int rans_occupancy() {
    const size_t sm = rans_smem_bytes();
    cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rans, kRansWarps * 32, sm) != cudaSuccess) return 0;
    return n;
}

}  // namespace acx
