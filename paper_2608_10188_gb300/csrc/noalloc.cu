// Decode entry point that allocates nothing (aceapex_decode_noalloc).
//
// Some callers cannot allocate device memory when they decode: allocators
// that hand the whole device to a framework pool at start-up, or real-time
// paths where an allocation's latency or failure is not acceptable.  For
// small archives they get this entry point: every byte of scratch it needs
// (the decode plan, the dependency lists, the decoded streams, the pending
// bitmaps and pieces, the work lists, the tickets and the error word) lives
// in one file-scope device array, and the archive's plan is built on the
// device by a small kernel, so neither device nor host memory is allocated.
// The call reads the plan summary and the status back to the host and
// synchronises its stream twice, so it cannot be recorded into a CUDA graph.
//
// Limits: at most kNaMaxBlocks blocks (1 MiB of output) and the per-region
// capacities below; valid archives beyond them are rejected with
// ACEAPEX_E_ARG, archives the regular entry point finds corrupt with
// ACEAPEX_E_CORRUPT.  The array is shared by every call in the process on a
// given device: calls that overlap on the GPU (other streams, other host
// threads) race on it.
#include <algorithm>
#include <mutex>

#include "../../include/aceapex.h"
#include "common.cuh"
#include "launch.h"

namespace acx {

namespace {

constexpr uint32_t kNaMaxBlocks = 64;
constexpr size_t kNaStreamBytes = 2u << 20;     // decoded streams
constexpr uint32_t kNaSpanSlots = 96u * 1024;   // pending pieces (and each work list)

// Layout of the static scratch (byte offsets, 256-aligned regions).
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffSummary = 0;
constexpr size_t kOffErr = al(kOffSummary + 64);
constexpr size_t kOffCounters = al(kOffErr + 16);
constexpr size_t kOffPlan = al(kOffCounters + kCounterWords * 4);
constexpr size_t kOffTab = al(kOffPlan + kNaMaxBlocks * sizeof(BlockDev));
constexpr size_t kOffNpend = al(kOffTab + 4 * kM * 4);
constexpr size_t kOffPmap = al(kOffNpend + kNaMaxBlocks * 4);
// dependency lists, copied out of the archive: block b's (at most b ids) at
// [b(b-1)/2, b(b-1)/2 + b), so the kernels read aligned words
constexpr size_t kNaDepWords = (size_t)kNaMaxBlocks * (kNaMaxBlocks - 1) / 2;
constexpr size_t kOffDeps = al(kOffPmap + (size_t)kNaMaxBlocks * (kBlock / 8));
constexpr size_t kOffSpans = al(kOffDeps + kNaDepWords * 4);
constexpr size_t kOffLists = al(kOffSpans + (size_t)kNaSpanSlots * sizeof(SpanRec));
constexpr size_t kOffStreams = al(kOffLists + 2 * (size_t)kNaSpanSlots * sizeof(JobDev::ListEnt));
constexpr size_t kNaBytes = al(kOffStreams + kNaStreamBytes + 64);

}  // namespace

// The scratch of aceapex_decode_noalloc (about 5.3 MiB per device).
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNaBytes];

namespace {

// Plan summary written by k_plan_small and read back by the host.
struct NaSummary {
    int32_t status;       // 0 ok, -2 corrupt, -1 beyond the static limits
    uint32_t n_blocks, min_match, max_tok, max_lenb, has_deps;
    uint64_t total, span_slots, stream_bytes;
};
static_assert(sizeof(NaSummary) <= 64, "summary");

__device__ __forceinline__ uint16_t rd16d(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
__device__ __forceinline__ uint32_t rd32d(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ uint64_t rd64d(const uint8_t* p) { return (uint64_t)rd32d(p) | ((uint64_t)rd32d(p + 4) << 32); }

// Validate a format v1 archive held in device memory and build its decode
// plan in the static scratch (one CTA).  The checks are the host plan
// builder's: header, tables, index entries, payload descriptors.
__global__ void __launch_bounds__(256) k_plan_small(const uint8_t* a, uint64_t len, uint8_t* base) {
    NaSummary* S = reinterpret_cast<NaSummary*>(base + kOffSummary);
    BlockDev* blk = reinterpret_cast<BlockDev*>(base + kOffPlan);
    uint32_t* tab = reinterpret_cast<uint32_t*>(base + kOffTab);
    uint32_t* deps = reinterpret_cast<uint32_t*>(base + kOffDeps);
    __shared__ int bad;            // 0 ok, -2 corrupt, -1 too large
    __shared__ uint64_t off_tab, off_idx, off_deps, total;
    __shared__ uint32_t nb, min_match, flags;
    __shared__ uint16_t freq[4][256];
    __shared__ uint32_t ok_tab[4];
    const int tid = threadIdx.x;
    if (tid == 0) {
        bad = 0;
        if (len < 64 || a[0] != 'A' || a[1] != 'C' || a[2] != 'X' || a[3] != '1' || rd16d(a + 4) != 1 ||
            rd32d(a + 8) != kBlock) {
            bad = -2;
        } else {
            flags = rd16d(a + 6);
            min_match = rd32d(a + 12);
            total = rd64d(a + 16);
            nb = rd32d(a + 24);
            off_tab = rd64d(a + 32);
            off_idx = rd64d(a + 40);
            off_deps = rd64d(a + 48);
            if (min_match < 4 || min_match > kBlock || (uint64_t)nb != (total + kBlock - 1) / kBlock) bad = -2;
            else if (off_tab > len || len - off_tab < 2048) bad = -2;
            else if (off_idx > len || (len - off_idx) / 40 < nb) bad = -2;
            else if (nb > kNaMaxBlocks) bad = -1;
        }
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) S->status = bad;
        return;
    }
    for (uint32_t i = tid; i < 4 * 256; i += blockDim.x) freq[i >> 8][i & 255] = rd16d(a + off_tab + 2 * i);
    __syncthreads();
    if (tid < 4) {
        uint32_t sum = 0;
        for (int k = 0; k < 256; k++) sum += freq[tid][k];
        ok_tab[tid] = sum == kM;
        if (sum != 0 && sum != kM) bad = -2;
    }
    __syncthreads();
    if (tid < 4 && ok_tab[tid]) {  // decode entries sym | (f-1) << 8 | (slot-c) << 20
        uint32_t c = 0;
        for (int k = 0; k < 256; k++) {
            const uint32_t f = freq[tid][k];
            for (uint32_t r = 0; r < f; r++) tab[tid * kM + c + r] = (uint32_t)k | ((f - 1) << 8) | (r << 20);
            c += f;
        }
    }
    for (uint32_t b = tid; b < nb; b += blockDim.x) {
        const uint8_t* e = a + off_idx + 40 * (uint64_t)b;
        const uint64_t poff = rd64d(e);
        const uint32_t plen = rd32d(e + 8), n_tok = rd32d(e + 12), raw = rd32d(e + 16);
        const uint32_t dep_off = rd32d(e + 20), n_deps = rd32d(e + 24);
        const uint64_t B = (uint64_t)b * kBlock;
        const uint64_t R = total - B < kBlock ? total - B : kBlock;
        bool ok = raw == R && !(off_deps == 0 && (dep_off || n_deps));
        // an ascending list of distinct ids below b has at most b entries
        const uint32_t dslot = b * (b - 1) / 2;
        if (ok && off_deps) {
            ok = off_deps <= len && (len - off_deps) / 4 >= (uint64_t)dep_off + n_deps && n_deps <= b;
            uint32_t prev = 0;
            for (uint32_t k = 0; ok && k < n_deps; k++) {
                const uint32_t id = rd32d(a + off_deps + 4 * ((uint64_t)dep_off + k));
                if (id >= b || (k && id <= prev)) ok = false;
                prev = id;
                deps[dslot + k] = id;
            }
        }
        ok = ok && !(poff & 15) && !(plen & 15) && plen >= 48 && poff <= len && len - poff >= plen;
        BlockDev bd{};
        if (ok) {
            const uint8_t* pay = a + poff;
            bd.payload = poff;
            bd.raw_len = raw;
            bd.n_tok = n_tok;
            if (off_deps) {
                bd.dep_off = dslot;
                bd.n_deps = n_deps;
            }
            uint64_t off = 48, soff = 0;
            for (int s = 0; s < 4 && ok; s++) {
                const uint8_t* d = pay + 12 * s;
                const uint32_t sraw = rd32d(d), enc = rd32d(d + 4);
                const uint8_t mode = d[8], K = d[9];
                if (rd16d(d + 10) != 0 || sraw > kMaxStreamRaw || off + enc > plen) { ok = false; break; }
                if (mode == 0) {
                    if (enc != sraw || K != 0) ok = false;
                } else if (mode == 1) {
                    const bool lanes_ok = K >= 1 && K <= kMaxLanes && (K & (K - 1)) == 0;
                    const uint32_t hdr = (4u * K + 15) & ~15u;
                    if (sraw == 0 || !lanes_ok || !ok_tab[s] || enc < hdr || ((enc - hdr) & 1)) ok = false;
                    bd.rans_mask |= 1u << s;
                } else {
                    ok = false;
                }
                bd.s_raw[s] = sraw;
                bd.s_body[s] = (uint32_t)off;
                bd.s_enc[s] = enc;
                bd.s_K[s] = K;
                bd.s_off[s] = (uint32_t)soff;
                soff = (soff + sraw + 15) & ~(uint64_t)15;
                off = (off + enc + 15) & ~(uint64_t)15;
            }
            if (flags & 2) {  // the level body (one stored byte per token) after the four streams
                ok = ok && off + n_tok <= plen;
                off = (off + n_tok + 15) & ~(uint64_t)15;
            }
            ok = ok && off == plen && bd.s_raw[kCmd] == n_tok && bd.s_raw[kOff] % 5 == 0 && bd.s_raw[kLit] <= raw;
            // every token but a closing literal run has a match of at least
            // min_match bytes: more tokens than that cannot sum to the block
            // (the regular decode finds such a block corrupt too)
            ok = ok && n_tok <= raw / min_match + 1;
            bd.n_new = bd.s_raw[kOff] / 5;
            bd.scratch = soff;  // this block's stream bytes; offsets are assigned below
        }
        if (!ok) bad = -2;
        blk[b] = bd;
    }
    __syncthreads();
    if (tid == 0) {
        int st = bad;
        uint64_t scratch = 0, slots = 0;
        uint32_t max_tok = 1, max_lenb = 1;
        for (uint32_t b = 0; b < nb && !st; b++) {
            BlockDev& bd = blk[b];
            const uint64_t sz = bd.scratch;
            bd.scratch = scratch;
            bd.span_base = (uint32_t)slots;
            scratch += sz;
            slots += bd.n_tok + kSpanSlack;
            max_tok = max(max_tok, bd.n_tok);
            max_lenb = max(max_lenb, bd.s_raw[kLen]);
        }
        if (!st && (scratch + 64 > kNaStreamBytes || slots > kNaSpanSlots)) st = -1;
        S->status = st;
        S->n_blocks = nb;
        S->min_match = min_match;
        S->max_tok = max_tok;
        S->max_lenb = max_lenb;
        S->total = total;
        S->has_deps = off_deps != 0;
        S->span_slots = slots;
        S->stream_bytes = scratch;
    }
}

// Device address of the static scratch, looked up once per device.
std::mutex g_na_mutex;
uint8_t* g_na_base[64];

}  // namespace
}  // namespace acx

using namespace acx;

extern "C" int aceapex_decode_noalloc(const void* d_arc, uint64_t arc_len, void* d_out, uint64_t out_cap,
                                      void* stream) {
    if (!d_arc || !d_out) return ACEAPEX_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ACEAPEX_E_CUDA;
    uint8_t* base = nullptr;
    {
        // set-up on the first call on this device (with that device current):
        // the host-side name of the array is not a device address
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_base[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ACEAPEX_E_CUDA;
            g_na_base[dev] = static_cast<uint8_t*>(p);
        }
        base = g_na_base[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_plan_small<<<1, 256, 0, st>>>((const uint8_t*)d_arc, arc_len, base);
    if (cudaGetLastError() != cudaSuccess) return ACEAPEX_E_CUDA;
    NaSummary S;
    if (cudaMemcpyAsync(&S, base + kOffSummary, sizeof S, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACEAPEX_E_CUDA;
    if (S.status == -1) return ACEAPEX_E_ARG;  // beyond the static scratch limits
    if (S.status != 0) return ACEAPEX_E_CORRUPT;
    if (out_cap < S.total) return ACEAPEX_E_ARG;
    if (S.n_blocks == 0) return ACEAPEX_OK;
    const size_t lsm = local_smem_bytes(S.max_tok, S.max_lenb);
    if (lsm > 227 * 1024) return ACEAPEX_E_CORRUPT;  // as the regular plan: no valid block needs that much
    JobDev job{};
    ArcJob& J = job.one;
    J.arc = (const uint8_t*)d_arc;
    J.blk = reinterpret_cast<const BlockDev*>(base + kOffPlan);
    J.dtab = reinterpret_cast<const uint32_t*>(base + kOffTab);
    J.scratch = base + kOffStreams;
    J.out = (uint8_t*)d_out;
    J.npend = reinterpret_cast<uint32_t*>(base + kOffNpend);
    J.pmap = reinterpret_cast<uint32_t*>(base + kOffPmap);
    J.spans = reinterpret_cast<SpanRec*>(base + kOffSpans);
    J.total = S.total;
    J.n_blocks = S.n_blocks;
    J.lo = 0;
    J.hi = S.n_blocks;
    J.min_match = S.min_match;
    J.deps = S.has_deps ? reinterpret_cast<const uint32_t*>(base + kOffDeps) : nullptr;
    job.n_arcs = 1;
    job.n_items = S.n_blocks;
    job.counters = reinterpret_cast<uint32_t*>(base + kOffCounters);
    job.err = reinterpret_cast<int*>(base + kOffErr);
    job.timeout_ns = 2000000000ull;
    job.max_tok = S.max_tok;
    job.max_lenb = S.max_lenb;
    job.lists[0] = reinterpret_cast<JobDev::ListEnt*>(base + kOffLists);
    job.lists[1] = job.lists[0] + kNaSpanSlots;
    int n_sms = 0;
    if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ACEAPEX_E_CUDA;
    note_sm_count(n_sms);
    // the array keeps the previous call's contents: clear the error word; the
    // prologue kernel clears the tickets and statistics
    if (cudaMemsetAsync(job.err, 0, 16, st) != cudaSuccess) return ACEAPEX_E_CUDA;
    if (launch_prologue(job.counters, 3 + 1, st) != cudaSuccess) return ACEAPEX_E_CUDA;
    if (launch_rans(job, std::max(1, rans_occupancy()) * n_sms, st) != cudaSuccess) return ACEAPEX_E_CUDA;
    if (launch_local(job, std::max(1, local_occupancy(lsm)) * n_sms, st) != cudaSuccess) return ACEAPEX_E_CUDA;
    if (launch_external(job, std::max(1, external_occupancy()) * n_sms, st) != cudaSuccess) return ACEAPEX_E_CUDA;
    int err[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(err, job.err, sizeof err, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ACEAPEX_E_CUDA;
    return err[0];
}
