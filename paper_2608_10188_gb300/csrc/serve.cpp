// Serving (aceapex_server_*): a request loop over one archive held compressed
// in device memory, with a bounded cache of decoded blocks.
//
// Requests (byte regions) arrive at any time.  A worker thread forms ticks:
// it admits the requests that have arrived, in arrival order, while the
// cache can hold what they need, walks each one's byte-level dependency
// closure minus what the cache already holds (paper, Random Access at Scale),
// and decodes the union with one launch sequence: the block decodes write
// into cache slots, then one gather copies every admitted region to its
// destination.  Ticks go to K lanes, each a stream with its own context,
// scratch and staging, up to two ticks deep; a new tick takes the lane with
// the fewest ticks in flight.  Ticks on different lanes run on the device at
// the same time unless one reads or writes a block that the other decodes,
// or decodes a block that the other reads: then the later one waits for the
// earlier one's completion event.  Requests that arrive while ticks run join
// the next tick (continuous batching); the host prepares it while they run.
//
// Cache: slots of 16 KiB (cache_bytes / 16 KiB of them), each with its
// pending count and bitmap.  A block's kept bytes are the wanted bytes of its
// last decode; a block decoded again keeps them (they are wanted again).
// Blocks read by a tick that has not completed are pinned; the others are
// evicted least recently used first.  Admission is by memory: a request
// waits while its closure needs more slots (or more blocks per tick) than are
// free or evictable, and is refused (ACEAPEX_E_BUSY) if it could never fit.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <queue>
#include <thread>
#include <vector>

#include "host.h"

using namespace acx;

namespace {

struct Req {
    uint64_t id = 0, start = 0, len = 0;
    uint8_t* dst = nullptr;
    int64_t at_ns = 0, admit_ns = 0;
    uint32_t closure = 0, decoded = 0;
};
struct ReqLater {  // min-heap on (arrival, id)
    bool operator()(const Req& a, const Req& b) const { return a.at_ns != b.at_ns ? a.at_ns > b.at_ns : a.id > b.id; }
};

// Host staging and device copies of one tick's tables (two sets per lane:
// the host fills one while the other's copies may still be pending).
struct TickBufs {
    ItemDev* h_items = nullptr;
    uint32_t* h_need = nullptr;
    GatherReq* h_gather = nullptr;
    int* h_err = nullptr;
    size_t cap_items = 0, cap_need = 0, cap_gather = 0;
    DevBuf d_items, d_need, d_gather;
};

// A stream of ticks with its own context (counters, error words), scratch
// and staging.
struct Lane {
    aceapex_ctx* c = nullptr;
    cudaStream_t st = nullptr;
    DevBuf streams, spans, lists;
    TickBufs bufs[2];
    uint64_t formed = 0;  // ticks formed on this lane (their staging alternates)
    int inflight = 0;
};

struct Tick {
    int lane = 0, set = 0;
    uint64_t seq = 0;
    cudaEvent_t start = nullptr, done = nullptr;
    std::vector<Req> reqs;
    std::vector<uint32_t> used;       // pinned blocks (sorted)
    std::vector<uint32_t> decoded;    // blocks written by this tick (sorted)
    std::vector<uint64_t> after;      // ticks in flight at launch that this one reads or writes after
};

bool sorted_meet(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
    size_t i = 0, j = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] == b[j]) return true;
        if (a[i] < b[j]) i++; else j++;
    }
    return false;
}

cudaError_t host_grow(void** p, size_t* cap, size_t need, size_t elem) {
    if (need <= *cap) return cudaSuccess;
    size_t n = std::max(need, *cap * 2 + 64);
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaHostAlloc(p, n * elem, cudaHostAllocDefault);
    if (e == cudaSuccess) *cap = n;
    return e;
}

}  // namespace

struct aceapex_server {
    aceapex_ctx* c = nullptr;  // own context (the worker thread's)
    aceapex_archive* A = nullptr;
    aceapex_server_params prm{};
    uint32_t n_slots = 0;
    std::chrono::steady_clock::time_point t0;
    // device
    uint8_t* cache = nullptr;
    uint32_t* npend = nullptr;
    uint32_t* pmap = nullptr;
    uint32_t* d_slot = nullptr;
    std::vector<Lane> lanes;
    std::deque<Tick> inflight;
    std::vector<cudaEvent_t> free_events;
    cudaEvent_t t0_ev = nullptr;               // the device clock's origin (recorded at creation)
    std::deque<std::pair<float, float>> spans_ms;  // device intervals of the last completed ticks
    std::deque<std::pair<uint64_t, int>> failed;   // recent failed ticks (seq, status)
    uint64_t seq_next = 1;
    // host cache state
    std::vector<uint32_t> slot_of;   // block -> slot or kNoSlot
    std::vector<Ivs> valid;          // block -> kept bytes (resident blocks)
    std::vector<uint32_t> pins;
    std::list<uint32_t> lru;         // unpinned resident blocks, most recent first
    std::vector<std::list<uint32_t>::iterator> lru_it;
    std::vector<uint8_t> in_lru;
    std::vector<uint32_t> free_slots;
    TickState walk;                  // the tick being formed: blocks to decode, wanted bytes, blocks read
    // closure walks of a tick's candidate requests run in parallel on these
    // threads (plus the worker); each walk sees the cache, not the tick
    struct WalkOut {
        std::vector<uint32_t> sched, used;
        std::vector<Ivs> need;  // wanted bytes of sched[i]
        bool bad = false;       // depends on a block the parse found corrupt
    };
    static constexpr int64_t kSpinNs = 250000;  // the worker yields instead of sleeping this close to an arrival
    static constexpr size_t kInlineWalks = 2;  // ticks of at most this many candidates walk on the worker alone
    std::vector<std::thread> pool;
    std::vector<TickState> pool_ts;
    std::mutex pool_mu;
    std::condition_variable pool_cv, pool_done_cv;
    uint64_t pool_gen = 0;
    int pool_busy = 0;
    bool pool_stop = false;
    std::atomic<size_t> pool_next{0};
    size_t pool_n = 0;
    const std::vector<Req>* pool_reqs = nullptr;
    std::vector<WalkOut>* pool_outs = nullptr;
    void walk_items(int ti);
    void walk_all(const std::vector<Req>& reqs, std::vector<WalkOut>& outs);
    // requests
    std::mutex mu;
    std::condition_variable cv;
    std::priority_queue<Req, std::vector<Req>, ReqLater> queue;
    std::vector<aceapex_completion> done;
    uint64_t next_id = 1, submitted = 0, finished = 0;
    std::thread worker;
    std::atomic<bool> stop{false};
    int fatal = 0;
    std::string fatal_msg;
    // statistics (under mu)
    std::vector<double> lat_us;
    std::vector<uint32_t> closures;
    uint64_t n_ok = 0, n_err = 0, n_busy = 0, bytes = 0, ticks = 0, blk_decoded = 0, blk_hit = 0;
    uint64_t tick_overlaps = 0, tick_waits = 0;
    int64_t form_ns = 0, walk_ns = 0, launch_ns = 0;  // host time forming the launched ticks; in their walks; in their launches
    int64_t first_arrival = -1, last_done = 0;

    int64_t now() const {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
    }
    void touch(uint32_t b) {  // most recently used
        if (in_lru[b]) lru.erase(lru_it[b]);
        lru.push_front(b);
        lru_it[b] = lru.begin();
        in_lru[b] = 1;
    }
    void pin(uint32_t b) {
        if (pins[b]++ == 0 && in_lru[b]) {
            lru.erase(lru_it[b]);
            in_lru[b] = 0;
        }
    }
    void unpin(uint32_t b) {
        if (--pins[b] == 0 && slot_of[b] != kNoSlot) touch(b);
    }
    void drop(uint32_t b) {  // forget a resident block, free its slot
        if (slot_of[b] == kNoSlot) return;
        if (in_lru[b]) {
            lru.erase(lru_it[b]);
            in_lru[b] = 0;
        }
        free_slots.push_back(slot_of[b]);
        slot_of[b] = kNoSlot;
        valid[b].clear();
    }
    static const Ivs* valid_fn(void* self, uint32_t b) {
        aceapex_server* s = (aceapex_server*)self;
        return s->slot_of[b] != kNoSlot ? &s->valid[b] : nullptr;
    }
    void run();
    bool form_tick(int li);
    void finish_tick(Tick& t, int status);
    cudaEvent_t take_event(cudaError_t* e);
    void complete(const Req& r, int status, int64_t t_done);
};

void aceapex_server::complete(const Req& r, int status, int64_t t_done) {
    aceapex_completion cpl{};
    cpl.id = r.id;
    cpl.status = status;
    cpl.closure_blocks = r.closure;
    cpl.decoded_blocks = r.decoded;
    cpl.latency_us = (double)(t_done - r.at_ns) / 1e3;
    cpl.queue_us = r.admit_ns ? (double)(r.admit_ns - r.at_ns) / 1e3 : 0.0;
    std::lock_guard<std::mutex> g(mu);
    done.push_back(cpl);
    finished++;
    if (status == ACEAPEX_OK) {
        n_ok++;
        bytes += r.len;
        lat_us.push_back(cpl.latency_us);
        closures.push_back(r.closure);
        if (first_arrival < 0 || r.at_ns < first_arrival) first_arrival = r.at_ns;
        last_done = std::max(last_done, t_done);
    } else if (status == ACEAPEX_E_BUSY) {
        n_busy++;
    } else {
        n_err++;
    }
    cv.notify_all();
}

void aceapex_server::finish_tick(Tick& t, int status) {
    const int64_t tn = now();
    // a tick that read or rewrote blocks after a failed one fails with it
    for (uint64_t q : t.after)
        for (const auto& f : failed)
            if (f.first == q && status == ACEAPEX_OK) status = f.second;
    if (status != ACEAPEX_OK) {
        failed.emplace_back(t.seq, status);
        if (failed.size() > 64) failed.pop_front();
    }
    for (uint32_t b : t.used) unpin(b);
    if (status != ACEAPEX_OK)
        for (uint32_t b : t.decoded)
            if (pins[b] == 0) drop(b);
    // device intervals: pairs of ticks (on different lanes) that ran at the same time
    float s_ms = 0, e_ms = 0;
    if (t.start && t.done && cudaEventElapsedTime(&s_ms, t0_ev, t.start) == cudaSuccess &&
        cudaEventElapsedTime(&e_ms, t0_ev, t.done) == cudaSuccess) {
        uint64_t ov = 0;
        for (const auto& iv : spans_ms) ov += s_ms < iv.second && iv.first < e_ms;
        spans_ms.emplace_back(s_ms, e_ms);
        if (spans_ms.size() > 16) spans_ms.pop_front();
        std::lock_guard<std::mutex> g(mu);
        tick_overlaps += ov;
    }
    for (const Req& r : t.reqs) complete(r, status, tn);
    if (t.start) free_events.push_back(t.start);
    if (t.done) free_events.push_back(t.done);
    lanes[t.lane].inflight--;
}

cudaEvent_t aceapex_server::take_event(cudaError_t* e) {
    if (free_events.empty()) {
        cudaEvent_t ev = nullptr;
        *e = cudaEventCreate(&ev);
        return *e == cudaSuccess ? ev : nullptr;
    }
    cudaEvent_t ev = free_events.back();
    free_events.pop_back();
    *e = cudaSuccess;
    return ev;
}

// One closure walk per request, against the cache only (thread ti's state).
void aceapex_server::walk_items(int ti) {
    TickState& ts = pool_ts[ti];
    WalkJournal j;
    const Plan& P = A->plan;
    for (;;) {
        const size_t i = pool_next.fetch_add(1);
        if (i >= pool_n) break;
        const Req& r = (*pool_reqs)[i];
        WalkOut& o = (*pool_outs)[i];
        ts.begin(P.n_blocks);
        span_walk(P, *A->midx, r.start, r.len, &aceapex_server::valid_fn, this, &ts, &j);
        o.bad = j.bad;
        o.sched.assign(ts.sched.begin(), ts.sched.end());
        o.used.assign(ts.used.begin(), ts.used.end());
        o.need.resize(o.sched.size());
        for (size_t k = 0; k < o.sched.size(); k++) o.need[k].swap(ts.need[o.sched[k]]);
    }
}

void aceapex_server::walk_all(const std::vector<Req>& reqs, std::vector<WalkOut>& outs) {
    outs.resize(reqs.size());
    pool_reqs = &reqs;
    pool_outs = &outs;
    pool_n = reqs.size();
    pool_next.store(0);
    if (reqs.size() <= kInlineWalks || pool.empty()) {
        // a lone request (an unloaded server): waking the pool threads would
        // cost more than the walk itself
        walk_items(0);
        return;
    }
    {
        std::lock_guard<std::mutex> g(pool_mu);
        pool_busy = (int)pool.size();
        pool_gen++;
    }
    pool_cv.notify_all();
    walk_items(0);
    std::unique_lock<std::mutex> g(pool_mu);
    pool_done_cv.wait(g, [this] { return pool_busy == 0; });
}

// Admit the arrived requests that fit and launch one tick on lane li; false
// if nothing was launched.
bool aceapex_server::form_tick(int li) {
    const Plan& P = A->plan;
    Lane& Ln = lanes[li];
    aceapex_ctx* c = Ln.c;
    cudaStream_t st = Ln.st;
    const int set = (int)(Ln.formed & 1);
    TickBufs& B = Ln.bufs[set];
    DevBuf& streams = Ln.streams;
    DevBuf& spans = Ln.spans;
    DevBuf& lists = Ln.lists;
    TickState& T = walk;
    T.begin(P.n_blocks);
    std::vector<Req> admitted, cand;
    std::vector<uint32_t> new_blocks;  // scheduled and not resident: need a slot
    const int64_t tn = now();
    {
        std::lock_guard<std::mutex> g(mu);
        while (!queue.empty() && queue.top().at_ns <= tn && cand.size() < prm.max_tick_requests) {
            cand.push_back(queue.top());
            queue.pop();
        }
    }
    if (cand.empty()) return false;
    std::vector<WalkOut> outs;
    walk_all(cand, outs);
    const int64_t t_walked = now();
    // admission in arrival order: a request joins while the cache can hold its
    // closure next to those admitted before it
    uint32_t avail = (uint32_t)(free_slots.size() + lru.size());
    size_t k = 0;
    for (; k < cand.size(); k++) {
        Req& r = cand[k];
        WalkOut& o = outs[k];
        if (o.bad) {  // a corrupt block: this request fails alone
            complete(r, ACEAPEX_E_CORRUPT, now());
            continue;
        }
        uint32_t need_slots = 0, new_sched = 0;
        for (uint32_t b : o.sched)
            if (!T.scheduled(b)) {
                new_sched++;
                if (slot_of[b] == kNoSlot) need_slots++;
            }
        // blocks kept by the cache that this request reads must stay: they are
        // pinned below, so they leave the evictable count
        uint32_t newly_pinned = 0;
        for (uint32_t b : o.used)
            if (T.used_mark[b] != T.epoch && slot_of[b] != kNoSlot && pins[b] == 0 && in_lru[b]) newly_pinned++;
        const bool fits = need_slots + newly_pinned <= avail && T.sched.size() + new_sched <= prm.max_tick_blocks;
        if (!fits) {
            if (!admitted.empty() || !inflight.empty()) break;  // wait for slots to free up
            // nothing else holds the cache: this request can never fit
            complete(r, ACEAPEX_E_BUSY, now());
            continue;
        }
        avail -= need_slots + newly_pinned;
        for (size_t q = 0; q < o.sched.size(); q++) {
            const uint32_t b = o.sched[q];
            if (!T.scheduled(b)) {
                T.sched_mark[b] = T.epoch;
                T.sched.push_back(b);
                T.need[b].swap(o.need[q]);  // (o is not read again)
                if (slot_of[b] == kNoSlot) new_blocks.push_back(b);
            } else {
                for (const auto& iv : o.need[q]) iv_union(T.need[b], iv.first, iv.second);
            }
        }
        for (uint32_t b : o.used)
            if (T.used_mark[b] != T.epoch) {
                T.used_mark[b] = T.epoch;
                T.used.push_back(b);
                pin(b);
            }
        r.admit_ns = tn;
        r.closure = (uint32_t)o.used.size();
        r.decoded = (uint32_t)o.sched.size();
        admitted.push_back(r);
    }
    if (k < cand.size()) {  // not admitted now: back to the queue (arrival order is kept)
        std::lock_guard<std::mutex> g(mu);
        for (; k < cand.size(); k++) queue.push(cand[k]);
    }
    if (admitted.empty()) return false;
    // slots for the new blocks: free ones first, then the least recently used
    for (uint32_t b : new_blocks) {
        uint32_t s;
        if (!free_slots.empty()) {
            s = free_slots.back();
            free_slots.pop_back();
        } else {
            const uint32_t victim = lru.back();
            lru.pop_back();
            in_lru[victim] = 0;
            s = slot_of[victim];
            slot_of[victim] = kNoSlot;
            valid[victim].clear();
        }
        slot_of[b] = s;
    }
    // work items: the blocks to decode, in block order, with their wanted bytes
    std::vector<uint32_t> blocks(T.sched.begin(), T.sched.end());
    std::sort(blocks.begin(), blocks.end());
    std::vector<uint32_t> slots(blocks.size());
    for (size_t i = 0; i < blocks.size(); i++) slots[i] = slot_of[blocks[i]];
    SubsetPlan S;
    subset_plan(P, blocks.data(), slots.data(), blocks.size(), &S);
    std::vector<uint32_t> need, iv;
    for (size_t i = 0; i < blocks.size(); i++) {
        Ivs& nb = T.need[blocks[i]];
        need_intervals(nb, P.blk[blocks[i]].raw_len, &iv);
        S.items[i].need_off = (uint32_t)need.size();
        S.items[i].need_n = (uint32_t)iv.size();
        need.insert(need.end(), iv.begin(), iv.end());
        valid[blocks[i]].swap(nb);  // kept once this tick has run (later ticks are ordered after it)
    }
    cudaError_t e;
    int rc = ACEAPEX_OK;
    const size_t nblk = blocks.size(), nreq = admitted.size();
    const int64_t t_launch = now();
    if ((e = host_grow((void**)&B.h_items, &B.cap_items, std::max<size_t>(nblk, 1), sizeof(ItemDev))) != cudaSuccess ||
        (e = host_grow((void**)&B.h_need, &B.cap_need, std::max<size_t>(need.size(), 1), sizeof(uint32_t))) != cudaSuccess ||
        (e = host_grow((void**)&B.h_gather, &B.cap_gather, nreq, sizeof(GatherReq))) != cudaSuccess ||
        (e = B.d_items.ensure(std::max<size_t>(nblk, 1) * sizeof(ItemDev))) != cudaSuccess ||
        (e = B.d_need.ensure(std::max<size_t>(need.size(), 1) * sizeof(uint32_t))) != cudaSuccess ||
        (e = B.d_gather.ensure(nreq * sizeof(GatherReq))) != cudaSuccess ||
        (e = streams.ensure(S.scratch_bytes)) != cudaSuccess ||
        (e = spans.ensure(std::max<uint64_t>(S.span_slots, 1) * sizeof(SpanRec))) != cudaSuccess ||
        (e = lists.ensure(2 * std::max<uint64_t>(S.span_slots, 1) * sizeof(JobDev::ListEnt))) != cudaSuccess)
        rc = cuda_fail(c, e, "server: tick buffers");
    uint64_t max_len = 0;
    if (rc == ACEAPEX_OK) {
        if (nblk) memcpy(B.h_items, S.items.data(), nblk * sizeof(ItemDev));
        if (!need.empty()) memcpy(B.h_need, need.data(), need.size() * sizeof(uint32_t));
        for (size_t i = 0; i < nreq; i++) {
            B.h_gather[i] = GatherReq{admitted[i].dst, admitted[i].start, admitted[i].len};
            max_len = std::max(max_len, admitted[i].len);
        }
        if ((nblk && (e = cudaMemcpyAsync(B.d_items.p, B.h_items, nblk * sizeof(ItemDev), cudaMemcpyHostToDevice, st)) !=
                         cudaSuccess) ||
            (!need.empty() && (e = cudaMemcpyAsync(B.d_need.p, B.h_need, need.size() * sizeof(uint32_t),
                                                   cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(B.d_gather.p, B.h_gather, nreq * sizeof(GatherReq), cudaMemcpyHostToDevice, st)) !=
                cudaSuccess)
            rc = cuda_fail(c, e, "server: tick upload");
    }
    // order after the ticks in flight that decode a block this tick reads, or
    // read a block this tick decodes (the same lane's are ordered by its stream)
    Tick t;
    t.lane = li;
    t.set = set;
    t.seq = seq_next++;
    t.used.assign(T.used.begin(), T.used.end());
    std::sort(t.used.begin(), t.used.end());
    t.decoded = blocks;  // sorted
    bool waited = false;
    for (const Tick& u : inflight) {
        if (!sorted_meet(t.used, u.decoded) && !sorted_meet(t.decoded, u.used)) continue;
        t.after.push_back(u.seq);
        if (u.lane != li && rc == ACEAPEX_OK) {
            if ((e = cudaStreamWaitEvent(st, u.done, 0)) != cudaSuccess) rc = cuda_fail(c, e, "server: tick order");
            waited = true;
        }
    }
    if (rc == ACEAPEX_OK && (t.start = take_event(&e)) == nullptr) rc = cuda_fail(c, e, "event");
    if (rc == ACEAPEX_OK && (e = cudaEventRecord(t.start, st)) != cudaSuccess) rc = cuda_fail(c, e, "event");
    if (rc == ACEAPEX_OK && nblk) {
        JobDev job{};
        ArcJob& Jb = job.one;
        Jb.arc = (const uint8_t*)A->d_arc;
        Jb.blk = A->d_blk;
        Jb.dtab = A->d_dtab;
        Jb.scratch = (uint8_t*)streams.p;
        Jb.out = cache;
        Jb.npend = npend;
        Jb.pmap = pmap;
        Jb.spans = (SpanRec*)spans.p;
        Jb.total = P.total;
        Jb.n_blocks = P.n_blocks;
        Jb.lo = 0;
        Jb.hi = (uint32_t)nblk;
        Jb.min_match = P.min_match;
        Jb.deps = A->d_deps;
        Jb.items = (const ItemDev*)B.d_items.p;
        Jb.need = (const uint32_t*)B.d_need.p;
        Jb.slot = d_slot;
        job.n_arcs = 1;
        job.n_items = (uint32_t)nblk;
        job.counters = c->counters;
        job.err = c->d_err;
        job.timeout_ns = (uint64_t)c->params.timeout_us * 1000ull;
        job.max_tok = S.max_tok;
        job.max_lenb = S.max_lenb;
        job.flags = need.empty() ? 0 : kJobNeed;
        job.lists[0] = (JobDev::ListEnt*)lists.p;
        job.lists[1] = job.lists[0] + std::max<uint64_t>(S.span_slots, 1);
        LaunchPlan lp;
        rc = launch_plan(c, c->params, S.max_tok, S.max_lenb, &lp, job.flags);
        // the cross-block pass of a tick holds a 1024-thread CTA per 32 blocks
        // at most, so that ticks on other lanes find SMs beside it
        lp.grid_ext = std::min<int>(lp.grid_ext, (int)std::max<size_t>(1, (nblk + 31) / 32));
        if (rc == ACEAPEX_OK) rc = enqueue_job(c, job, lp, 4, c->d_err, 4, st, nullptr);
    } else if (rc == ACEAPEX_OK) {
        if ((e = cudaMemsetAsync(c->d_err, 0, 4 * sizeof(int), st)) != cudaSuccess) rc = cuda_fail(c, e, "server");
    }
    if (rc == ACEAPEX_OK && (e = launch_gather(nullptr, (const GatherReq*)B.d_gather.p, (uint32_t)nreq, max_len, cache,
                                               d_slot, st)) != cudaSuccess)
        rc = cuda_fail(c, e, "server: gather launch");
    if (rc == ACEAPEX_OK &&
        (e = cudaMemcpyAsync(B.h_err, c->d_err, 4 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        rc = cuda_fail(c, e, "server: status copy");
    t.reqs.swap(admitted);
    if (rc == ACEAPEX_OK && (t.done = take_event(&e)) == nullptr) rc = cuda_fail(c, e, "event");
    if (rc == ACEAPEX_OK && (e = cudaEventRecord(t.done, st)) != cudaSuccess) rc = cuda_fail(c, e, "event");
    Ln.formed++;
    Ln.inflight++;
    {
        const int64_t t_end = now();
        std::lock_guard<std::mutex> g(mu);
        form_ns += t_end - tn;
        walk_ns += t_walked - tn;
        launch_ns += t_end - t_launch;
        ticks++;
        tick_waits += waited;
        blk_decoded += nblk;
        blk_hit += T.used.size() - T.sched.size();
    }
    if (rc != ACEAPEX_OK) {
        // the launch failed: nothing more is launched; the server stops
        cudaDeviceSynchronize();
        if (t.start) free_events.push_back(t.start);
        if (t.done) free_events.push_back(t.done);
        t.start = t.done = nullptr;
        finish_tick(t, rc);
        std::lock_guard<std::mutex> g(mu);
        fatal = rc;
        fatal_msg = c->err;
        return true;
    }
    inflight.push_back(std::move(t));
    return true;
}

void aceapex_server::run() {
    cudaSetDevice(c->device);
    while (!stop.load()) {
        // completed ticks, on any lane
        for (auto it = inflight.begin(); it != inflight.end();) {
            const cudaError_t q = cudaEventQuery(it->done);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            int status = ACEAPEX_OK;
            if (q != cudaSuccess) {
                status = ACEAPEX_E_CUDA;
            } else if (lanes[it->lane].bufs[it->set].h_err[0]) {
                status = lanes[it->lane].bufs[it->set].h_err[0];
            }
            finish_tick(*it, status);
            it = inflight.erase(it);
        }
        // the lane with the fewest ticks in flight, two at most
        int li = 0;
        for (int k = 1; k < (int)lanes.size(); k++)
            if (lanes[k].inflight < lanes[li].inflight) li = k;
        bool launched = false;
        if (lanes[li].inflight < 2 && !fatal) launched = form_tick(li);
        if (launched) continue;
        // nothing to launch: wait briefly for a completion or an arrival
        int64_t next_at = -1;
        {
            std::lock_guard<std::mutex> g(mu);
            if (!queue.empty()) next_at = queue.top().at_ns;
        }
        if (!inflight.empty()) {
            std::this_thread::yield();
        } else {
            std::unique_lock<std::mutex> g(mu);
            const int64_t tn = now();
            int64_t wait_ns = 2000000;
            if (next_at >= 0) wait_ns = std::max<int64_t>(0, std::min<int64_t>(wait_ns, next_at - tn));
            // a timed sleep may end tens of microseconds late (timer slack):
            // sleep until shortly before the next arrival, then yield
            if (wait_ns > kSpinNs)
                cv.wait_for(g, std::chrono::nanoseconds(wait_ns - kSpinNs));
            else if (wait_ns > 0) {
                g.unlock();
                std::this_thread::yield();
            }
        }
    }
    // drain what is on the GPU
    for (Lane& L : lanes) cudaStreamSynchronize(L.st);
    while (!inflight.empty()) {
        Tick& t = inflight.front();
        finish_tick(t, cudaEventQuery(t.done) == cudaSuccess ? lanes[t.lane].bufs[t.set].h_err[0] : ACEAPEX_E_CUDA);
        inflight.pop_front();
    }
}

static void server_free(aceapex_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        s->stop.store(true);
        s->cv.notify_all();
        s->worker.join();
    }
    {
        std::lock_guard<std::mutex> g(s->pool_mu);
        s->pool_stop = true;
    }
    s->pool_cv.notify_all();
    for (auto& t : s->pool) t.join();
    if (s->c) cudaSetDevice(s->c->device);
    for (Lane& L : s->lanes)
        if (L.st) cudaStreamSynchronize(L.st);
    for (auto& ev : s->free_events) cudaEventDestroy(ev);
    if (s->t0_ev) cudaEventDestroy(s->t0_ev);
    for (size_t k = 0; k < s->lanes.size(); k++) {
        Lane& L = s->lanes[k];
        for (auto& B : L.bufs) {
            if (B.h_items) cudaFreeHost(B.h_items);
            if (B.h_need) cudaFreeHost(B.h_need);
            if (B.h_gather) cudaFreeHost(B.h_gather);
            if (B.h_err) cudaFreeHost(B.h_err);
            B.d_items.release();
            B.d_need.release();
            B.d_gather.release();
        }
        L.streams.release();
        L.spans.release();
        L.lists.release();
        if (L.st) cudaStreamDestroy(L.st);
        if (k > 0 && L.c) aceapex_ctx_destroy(L.c);  // lane 0 runs on the server's own context
    }
    if (s->cache) cudaFree(s->cache);
    if (s->npend) cudaFree(s->npend);
    if (s->pmap) cudaFree(s->pmap);
    if (s->d_slot) cudaFree(s->d_slot);
    if (s->c) aceapex_ctx_destroy(s->c);
    delete s;
}

extern "C" {

int aceapex_server_create(aceapex_ctx* ctx, aceapex_archive* A, const aceapex_server_params* p,
                          aceapex_server** out) {
    if (!ctx || !A || !out) return fail(ctx, ACEAPEX_E_ARG, "server_create: null argument");
    *out = nullptr;
    aceapex_server* s = new (std::nothrow) aceapex_server();
    if (!s) return fail(ctx, ACEAPEX_E_NOMEM, "server_create: host allocation");
    if (p) s->prm = *p;
    if (!s->prm.cache_bytes) s->prm.cache_bytes = 4ull << 30;
    if (!s->prm.max_tick_blocks) s->prm.max_tick_blocks = 16384;
    if (!s->prm.max_tick_requests) s->prm.max_tick_requests = 4096;
    if (!s->prm.streams) s->prm.streams = 2;
    if (s->prm.streams > 16) {
        delete s;
        return fail(ctx, ACEAPEX_E_ARG, "server_create: more than 16 tick streams");
    }
    s->A = A;
    const uint32_t nb = A->plan.n_blocks;
    s->n_slots = (uint32_t)std::min<uint64_t>(s->prm.cache_bytes / kBlock, 0xfffffff0u);
    int rc = aceapex_ctx_create(ctx->device, &ctx->params, &s->c);
    if (rc) {
        delete s;
        return fail(ctx, rc, "server_create: context");
    }
    if (s->n_slots == 0) {
        server_free(s);
        return fail(ctx, ACEAPEX_E_ARG, "server_create: cache smaller than one block");
    }
    // the byte-level closure needs the archive's match index
    if ((rc = build_match_index(ctx, A))) {
        server_free(s);
        return rc;
    }
    s->lanes.resize(s->prm.streams);
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < s->lanes.size() && e == cudaSuccess && rc == 0; k++) {
        Lane& L = s->lanes[k];
        if (k == 0) L.c = s->c;
        else rc = aceapex_ctx_create(ctx->device, &ctx->params, &L.c);
        if (rc == 0) e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking);
        for (auto& B : L.bufs)
            if (rc == 0 && e == cudaSuccess) e = cudaHostAlloc((void**)&B.h_err, 4 * sizeof(int), cudaHostAllocDefault);
    }
    if (rc) {
        server_free(s);
        return fail(ctx, rc, "server_create: lane context");
    }
    if (e == cudaSuccess) e = cudaEventCreate(&s->t0_ev);
    if (e == cudaSuccess) e = cudaEventRecord(s->t0_ev, s->lanes[0].st);
    if (e == cudaSuccess) e = cudaMalloc(&s->cache, (size_t)s->n_slots * kBlock);
    if (e == cudaSuccess) e = cudaMalloc(&s->npend, (size_t)s->n_slots * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->pmap, (size_t)s->n_slots * (kBlock / 8));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_slot, (size_t)std::max<uint32_t>(nb, 1) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->d_slot, 0xff, (size_t)std::max<uint32_t>(nb, 1) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->pmap, 0, (size_t)s->n_slots * (kBlock / 8));
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        server_free(s);
        return oom ? fail(ctx, ACEAPEX_E_NOMEM, "server_create: device memory for the cache")
                   : cuda_fail(ctx, e, "server_create");
    }
    s->slot_of.assign(nb, kNoSlot);
    s->valid.assign(nb, Ivs());
    s->pins.assign(nb, 0);
    s->lru_it.resize(nb);
    s->in_lru.assign(nb, 0);
    s->free_slots.resize(s->n_slots);
    for (uint32_t i = 0; i < s->n_slots; i++) s->free_slots[i] = s->n_slots - 1 - i;
    s->t0 = std::chrono::steady_clock::now();
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int n_walk = (int)std::min(8u, std::max(1u, hw / 2));  // walkers, the worker included
    s->pool_ts.resize(n_walk);
    for (int t = 1; t < n_walk; t++)
        s->pool.emplace_back([s, t] {
            uint64_t seen = 0;
            for (;;) {
                {
                    std::unique_lock<std::mutex> g(s->pool_mu);
                    s->pool_cv.wait(g, [s, seen] { return s->pool_stop || s->pool_gen != seen; });
                    if (s->pool_stop) return;
                    seen = s->pool_gen;
                }
                s->walk_items(t);
                std::lock_guard<std::mutex> g(s->pool_mu);
                if (--s->pool_busy == 0) s->pool_done_cv.notify_all();
            }
        });
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return ACEAPEX_OK;
}

int64_t aceapex_server_now_ns(const aceapex_server* s) { return s ? s->now() : -1; }

int aceapex_server_submit_many(aceapex_server* s, int n, const uint64_t* start, const uint64_t* len, void* const* d_out,
                               const int64_t* at_ns, uint64_t* ids) {
    if (!s || n < 0 || (n && (!start || !len || !d_out))) return ACEAPEX_E_ARG;
    const uint64_t total = s->A->plan.total;
    for (int i = 0; i < n; i++)
        if (start[i] > total || len[i] > total - start[i] || (len[i] && !d_out[i])) return ACEAPEX_E_RANGE;
    const int64_t tn = s->now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->fatal) return s->fatal;
        for (int i = 0; i < n; i++) {
            Req r;
            r.id = s->next_id++;
            r.start = start[i];
            r.len = len[i];
            r.dst = (uint8_t*)d_out[i];
            r.at_ns = at_ns && at_ns[i] >= 0 ? at_ns[i] : tn;
            if (ids) ids[i] = r.id;
            s->queue.push(r);
            s->submitted++;
        }
    }
    s->cv.notify_all();
    return ACEAPEX_OK;
}

int aceapex_server_submit(aceapex_server* s, uint64_t start, uint64_t len, void* d_out, int64_t at_ns, uint64_t* id) {
    return aceapex_server_submit_many(s, 1, &start, &len, &d_out, &at_ns, id);
}

int aceapex_server_poll(aceapex_server* s, aceapex_completion* out, int max, int wait_ms) {
    if (!s || max < 0 || (max && !out)) return ACEAPEX_E_ARG;
    std::unique_lock<std::mutex> g(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv.wait_for(g, std::chrono::milliseconds(wait_ms), [s] { return !s->done.empty() || s->fatal; });
    const int n = (int)std::min<size_t>(s->done.size(), (size_t)max);
    for (int i = 0; i < n; i++) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    return n;
}

int aceapex_server_drain(aceapex_server* s, int timeout_ms) {
    if (!s) return ACEAPEX_E_ARG;
    std::unique_lock<std::mutex> g(s->mu);
    const bool ok = s->cv.wait_for(g, std::chrono::milliseconds(timeout_ms),
                                   [s] { return s->finished == s->submitted || s->fatal; });
    if (s->fatal) return s->fatal;
    return ok ? ACEAPEX_OK : ACEAPEX_E_TIMEOUT;
}

int aceapex_server_get_stats(aceapex_server* s, int reset, aceapex_server_stats* out) {
    if (!s || !out) return ACEAPEX_E_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    out->completed = s->n_ok;
    out->failed = s->n_err;
    out->refused = s->n_busy;
    out->bytes = s->bytes;
    out->ticks = s->ticks;
    out->blocks_decoded = s->blk_decoded;
    out->blocks_hit = s->blk_hit;
    out->tick_overlaps = s->tick_overlaps;
    out->tick_waits = s->tick_waits;
    out->tick_host_ms = (double)s->form_ns / 1e6;
    out->walk_ms = (double)s->walk_ns / 1e6;
    out->launch_ms = (double)s->launch_ns / 1e6;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_us = sum / v.size();
        std::vector<uint32_t> cl = s->closures;
        std::sort(cl.begin(), cl.end());
        double cs = 0;
        for (uint32_t x : cl) cs += x;
        out->closure_mean = cs / cl.size();
        out->closure_p50 = cl[(cl.size() - 1) / 2];
        out->closure_p99 = cl[std::min(cl.size() - 1, (size_t)(0.99 * (cl.size() - 1) + 0.5))];
        const double span_s = (double)(s->last_done - s->first_arrival) / 1e9;
        out->seconds = span_s;
        out->gbs = span_s > 0 ? (double)s->bytes / span_s / 1e9 : 0.0;
    }
    if (reset) {
        s->lat_us.clear();
        s->closures.clear();
        s->n_ok = s->n_err = s->n_busy = s->bytes = s->ticks = s->blk_decoded = s->blk_hit = 0;
        s->tick_overlaps = s->tick_waits = 0;
        s->form_ns = s->walk_ns = s->launch_ns = 0;
        s->first_arrival = -1;
        s->last_done = 0;
    }
    return ACEAPEX_OK;
}

const char* aceapex_server_last_error(const aceapex_server* s) { return s ? s->fatal_msg.c_str() : "null server"; }

int aceapex_server_destroy(aceapex_server* s) {
    if (!s) return ACEAPEX_E_ARG;
    server_free(s);
    return ACEAPEX_OK;
}

}  // extern "C"
