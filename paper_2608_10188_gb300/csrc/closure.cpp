// Byte-level dependency closures: the archive's match index (built by a
// parse-only pass on the device) and the walk from wanted byte ranges back
// through the matches that write them.
//
// Paper, Random Access at Scale and "The byte-level refutation": what a
// region needs is not every block its blocks reference but the bytes its
// bytes were copied from.  With sources anywhere in the output (absolute
// offsets), a block-level closure grows to a large part of the archive,
// while the byte-level one stays near the region: each copied byte has one
// source, and chains end at literals after a few steps (the encoder caps the
// chain depth).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "host.h"

using namespace acx;

namespace {

// Is [s, e) inside the union of v?
bool iv_covers(const Ivs& v, uint32_t s, uint32_t e) {
    auto it = std::upper_bound(v.begin(), v.end(), std::make_pair(s, 0xffffffffu));
    if (it == v.begin()) return false;
    --it;
    return it->first <= s && it->second >= e;
}

// The parts of [s, e) outside v.
void iv_minus(uint32_t s, uint32_t e, const Ivs& v, Ivs* out) {
    out->clear();
    auto it = std::upper_bound(v.begin(), v.end(), std::make_pair(s, 0xffffffffu));
    if (it != v.begin() && std::prev(it)->second > s) s = std::prev(it)->second;
    for (; s < e && it != v.end() && it->first < e; ++it) {
        if (it->first > s) out->push_back({s, it->first});
        s = std::max(s, it->second);
    }
    if (s < e) out->push_back({s, e});
}

// Does [s, e) meet the union of v?
bool iv_meets(const Ivs& v, uint32_t s, uint32_t e) {
    auto it = std::upper_bound(v.begin(), v.end(), std::make_pair(s, 0xffffffffu));
    if (it != v.begin() && std::prev(it)->second > s) return true;
    return it != v.end() && it->first < e;
}

// v |= [s, e)
void iv_add(Ivs& v, uint32_t s, uint32_t e) {
    auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(s, 0u));
    if (it != v.begin() && std::prev(it)->second >= s) --it;
    auto jt = it;
    while (jt != v.end() && jt->first <= e) {
        s = std::min(s, jt->first);
        e = std::max(e, jt->second);
        ++jt;
    }
    it = v.erase(it, jt);
    v.insert(it, {s, e});
}

}  // namespace

namespace {

// Count one parsed block into the parse statistics (paper, The Last
// Sequential Element).  Its token records, in token order, hold the source
// (x, y bits 0..7), the destination offset and match length (z) and the
// command (w).  A token's literal run is its destination minus the previous
// token's end; a repeat-coded token ends a dependency-free run, and the block
// end ends the last one (the history resets per block).
void count_block(const SpanRec* h, uint32_t n, uint64_t B, aceapex_parse_stats& S, std::vector<uint32_t>& runs) {
    S.blocks++;
    S.tokens += n;
    S.values += 2ull * n;
    S.max_tokens_block = std::max<uint64_t>(S.max_tokens_block, n);
    uint32_t end = 0, run = 0;
    for (uint32_t q = 0; q < n; q++) {
        const SpanRec& r = h[q];
        const uint32_t ml = r.z >> 16, o = r.z & 0xffff, ll = o - end;
        const uint64_t src = (uint64_t)r.x | ((uint64_t)(r.y & 0xff) << 32);
        end = o + ml;
        S.literal_bytes += ll;
        S.match_bytes += ml;
        S.multibyte_values += (ll >= 128) + (ml >= 128);
        if (r.w == kLitOnly) {
            S.lit_only++;
            run++;
        } else {
            if (B + o - src < ml) S.overlap_matches++;
            if (src < B) S.external_matches++;
            if (r.w == kNew) {
                S.new_matches++;
                run++;
            } else {
                S.rep_matches[r.w - kRep0]++;
                runs.push_back(run);
                run = 0;
            }
        }
    }
    runs.push_back(run);
}

// Sum, maximum and median (rank floor(runs / 2)) of the run lengths.
void finish_runs(aceapex_parse_stats& S, std::vector<uint32_t>& runs) {
    if (runs.empty()) return;
    for (uint32_t v : runs) {
        S.run_len_sum += v;
        S.max_run = std::max<uint64_t>(S.max_run, v);
    }
    S.runs = runs.size();
    std::nth_element(runs.begin(), runs.begin() + runs.size() / 2, runs.end());
    S.median_run = runs[runs.size() / 2];
}

}  // namespace

int acx::build_match_index(aceapex_ctx* c, aceapex_archive* A) {
    if (A->midx) return ACEAPEX_OK;
    const Plan& P = A->plan;
    MatchIndex* M = new (std::nothrow) MatchIndex();
    if (!M) return fail(c, ACEAPEX_E_NOMEM, "match index: host allocation");
    M->first.assign((size_t)P.n_blocks + 1, 0);
    cudaSetDevice(c->device);
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete M;
        return cuda_fail(c, e, "match index: stream");
    }
    DevBuf items, recs, scratch, status;
    M->bad.assign(P.n_blocks, 0);
    std::vector<uint32_t> st_h;
    std::vector<SpanRec> h;
    std::vector<ItemDev> it;
    std::vector<uint32_t> runs;
    aceapex_parse_stats S{};
    int rc = ACEAPEX_OK;
    constexpr uint32_t kChunk = 16384;  // blocks per parse-only job
    for (uint32_t c0 = 0; c0 < P.n_blocks && rc == ACEAPEX_OK; c0 += kChunk) {
        const uint32_t c1 = std::min(P.n_blocks, c0 + kChunk), k = c1 - c0;
        it.assign(k, ItemDev{});
        uint64_t toks = 0, sb = 0;
        uint32_t max_tok = 1, max_lenb = 1;
        for (uint32_t i = 0; i < k; i++) {
            const BlockDev& bd = P.blk[c0 + i];
            it[i].block = c0 + i;
            it[i].slot = i;  // index of the item's status word
            it[i].span_base = (uint32_t)toks;  // token records, packed
            it[i].scratch = sb;
            toks += bd.n_tok;
            sb += (bd.s_off[3] + bd.s_raw[3] + 15) & ~15ull;
            max_tok = std::max(max_tok, bd.n_tok);
            max_lenb = std::max(max_lenb, bd.s_raw[kLen]);
        }
        sb += 64;
        if ((e = items.ensure(k * sizeof(ItemDev))) != cudaSuccess ||
            (e = recs.ensure(std::max<uint64_t>(toks, 1) * sizeof(SpanRec))) != cudaSuccess ||
            (e = scratch.ensure(sb)) != cudaSuccess || (e = status.ensure(k * sizeof(uint32_t))) != cudaSuccess ||
            (e = cudaMemsetAsync(status.p, 0, k * sizeof(uint32_t), st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(items.p, it.data(), k * sizeof(ItemDev), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            rc = cuda_fail(c, e, "match index: scratch");
            break;
        }
        JobDev job{};
        ArcJob& J = job.one;
        J.arc = (const uint8_t*)A->d_arc;
        J.blk = A->d_blk;
        J.dtab = A->d_dtab;
        J.scratch = (uint8_t*)scratch.p;
        J.spans = (SpanRec*)recs.p;
        J.total = P.total;
        J.n_blocks = P.n_blocks;
        J.lo = 0;
        J.hi = k;
        J.min_match = P.min_match;
        J.deps = A->d_deps;
        J.items = (const ItemDev*)items.p;
        J.npend = (uint32_t*)status.p;
        job.n_arcs = 1;
        job.n_items = k;
        job.counters = c->counters;
        job.err = c->d_err;
        job.timeout_ns = (uint64_t)c->params.timeout_us * 1000ull;
        job.max_tok = max_tok;
        job.max_lenb = max_lenb;
        job.flags = kJobIndex;
        LaunchPlan lp;
        if ((rc = launch_plan(c, c->params, max_tok, max_lenb, &lp, kJobIndex))) break;
        if ((rc = enqueue_job(c, job, lp, 4, nullptr, 0, st, nullptr))) break;
        // a corrupt block is recorded in its status word and the index goes on
        if ((rc = ctx_read_status(c, st)) && rc != ACEAPEX_E_CORRUPT) break;
        rc = ACEAPEX_OK;
        st_h.resize(k);
        if ((e = cudaMemcpy(st_h.data(), status.p, k * sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            rc = cuda_fail(c, e, "match index: status");
            break;
        }
        h.resize(toks);
        if (toks && (e = cudaMemcpy(h.data(), recs.p, toks * sizeof(SpanRec), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            rc = cuda_fail(c, e, "match index: records");
            break;
        }
        uint64_t t = 0;
        for (uint32_t i = 0; i < k; i++) {
            const uint32_t b = c0 + i, n = P.blk[b].n_tok;
            M->first[b] = M->o.size();
            if (st_h[i]) {
                M->bad[b] = 1;
                S.bad_blocks++;
                t += n;
                continue;
            }
            count_block(h.data() + t, n, (uint64_t)b * kBlock, S, runs);
            for (uint32_t q = 0; q < n; q++, t++) {
                const SpanRec& r = h[t];
                const uint32_t ml = r.z >> 16;
                if (!ml) continue;
                M->o.push_back((uint16_t)(r.z & 0xffff));
                M->ml.push_back((uint16_t)ml);
                M->src.push_back((uint64_t)r.x | ((uint64_t)(r.y & 0xff) << 32));
            }
        }
    }
    M->first[P.n_blocks] = M->o.size();
    finish_runs(S, runs);
    M->stats = S;
    cudaStreamDestroy(st);
    items.release();
    recs.release();
    scratch.release();
    status.release();
    if (rc) {
        delete M;
        return rc;
    }
    A->midx = M;
    return ACEAPEX_OK;
}

void acx::TickState::begin(uint32_t n_blocks) {
    if (sched_mark.size() != n_blocks) {
        sched_mark.assign(n_blocks, 0);
        used_mark.assign(n_blocks, 0);
        touch_req.assign(n_blocks, 0);
        need.assign(n_blocks, Ivs());
        epoch = 0;
    }
    if (++epoch == 0) {  // the stamps wrapped: clear them once
        std::fill(sched_mark.begin(), sched_mark.end(), 0);
        std::fill(used_mark.begin(), used_mark.end(), 0);
        epoch = 1;
    }
    sched.clear();
    used.clear();
}

void acx::span_walk(const Plan& P, const MatchIndex& M, uint64_t start, uint64_t len, ValidFn valid, void* self,
                    TickState* T, WalkJournal* J) {
    (void)P;
    const uint32_t ep = T->epoch;
    if (++T->req == 0) {
        std::fill(T->touch_req.begin(), T->touch_req.end(), 0);
        T->req = 1;
    }
    const uint32_t rq = T->req;
    J->saved.clear();
    J->bad = false;
    J->sched0 = T->sched.size();
    J->used0 = T->used.size();
    auto& stack = T->stack;
    Ivs& parts = T->parts;
    stack.clear();
    auto push_abs = [&](uint64_t s, uint64_t e) {  // absolute [s, e), split by block
        for (uint64_t a = s / kBlock; a <= (e - 1) / kBlock; a++) {
            const uint64_t A0 = a * kBlock;
            stack.push_back({(uint32_t)a, (uint32_t)(std::max(s, A0) - A0), (uint32_t)(std::min(e, A0 + kBlock) - A0)});
        }
    };
    if (len) push_abs(start, start + len);
    while (!stack.empty()) {
        const TickState::R r = stack.back();
        stack.pop_back();
        if (r.s >= r.e) continue;
        const uint32_t X = r.b;
        if (!M.bad.empty() && M.bad[X]) {  // no matches are known there: the region cannot be decoded
            J->bad = true;
            continue;
        }
        if (T->used_mark[X] != ep) {
            T->used_mark[X] = ep;
            T->used.push_back(X);
        }
        Ivs& nX = T->need[X];
        if (T->sched_mark[X] != ep) {
            const Ivs* V = valid(self, X);
            if (V && iv_covers(*V, r.s, r.e)) continue;  // kept from an earlier decode
            T->sched_mark[X] = ep;
            T->touch_req[X] = rq;
            T->sched.push_back(X);
            nX.clear();
            // a block decoded again keeps what it held: its kept bytes are wanted too
            if (V)
                for (const auto& iv : *V) stack.push_back({X, iv.first, iv.second});
        }
        iv_minus(r.s, r.e, nX, &parts);
        if (parts.empty()) continue;
        if (T->touch_req[X] != rq) {  // scheduled by an earlier request: keep its need for an undo
            T->touch_req[X] = rq;
            J->saved.push_back({X, nX});
        }
        const uint64_t lo = M.first[X], hi = M.first[X + 1];
        // Every byte enters the wanted set together with all matches that
        // touch it, so a match touching the wanted set is already followed.
        for (const auto& p : parts) {
            // matches of X overlapping p (matches are disjoint and in order)
            uint64_t a = lo, z = hi;
            while (a < z) {
                const uint64_t m = (a + z) / 2;
                if ((uint32_t)M.o[m] + M.ml[m] <= p.first) a = m + 1; else z = m;
            }
            for (uint64_t k = a; k < hi && M.o[k] < p.second; k++) {
                const uint32_t o = M.o[k], ml = M.ml[k];
                if (iv_meets(nX, o, o + ml)) continue;
                stack.push_back({X, o, o + ml});  // the whole match is decoded
                const uint64_t dst = (uint64_t)X * kBlock + o, src = M.src[k];
                const uint64_t d = dst - src;
                push_abs(src, src + std::min<uint64_t>(d, ml));  // its source window (one period if it overlaps)
            }
            iv_add(nX, p.first, p.second);
        }
    }
}

void acx::span_undo(TickState* T, const WalkJournal& J) {
    for (size_t i = J.sched0; i < T->sched.size(); i++) {
        T->sched_mark[T->sched[i]] = 0;
        T->need[T->sched[i]].clear();
    }
    T->sched.resize(J.sched0);
    for (const auto& sv : J.saved) T->need[sv.first] = sv.second;
    for (size_t i = J.used0; i < T->used.size(); i++) T->used_mark[T->used[i]] = 0;
    T->used.resize(J.used0);
}

void acx::iv_union(Ivs& v, uint32_t s, uint32_t e) { iv_add(v, s, e); }

void acx::need_intervals(const Ivs& need, uint32_t raw_len, std::vector<uint32_t>* out) {
    out->clear();
    if (need.size() == 1 && need[0].first == 0 && need[0].second >= raw_len) return;
    for (const auto& iv : need) out->push_back(iv.first | (std::min(iv.second, kBlock) << 16));
}

extern "C" int aceapex_archive_index(aceapex_ctx* c, aceapex_archive* A) {
    if (!c || !A) return fail(c, ACEAPEX_E_ARG, "archive_index: null argument");
    return build_match_index(c, A);
}

extern "C" int aceapex_archive_parse_stats(aceapex_ctx* c, aceapex_archive* A, aceapex_parse_stats* stats) {
    if (!c || !A || !stats) return fail(c, ACEAPEX_E_ARG, "archive_parse_stats: null argument");
    const int rc = build_match_index(c, A);
    if (rc) return rc;
    *stats = A->midx->stats;
    return ACEAPEX_OK;
}

// Diagnostics (not part of the documented ABI; host only): the parse
// statistics of token records given on the host — recs[4 * t .. 4 * t + 4)
// is token t's record (as the parse-only pass writes it), blocks in order,
// n_tok[b] tokens each.
extern "C" int acx_debug_parse_stats(const uint32_t* recs, const uint32_t* n_tok, uint32_t n_blocks,
                                     aceapex_parse_stats* out) {
    if (!recs || !n_tok || !out) return -1;
    aceapex_parse_stats S{};
    std::vector<uint32_t> runs;
    const SpanRec* h = reinterpret_cast<const SpanRec*>(recs);
    uint64_t t = 0;
    for (uint32_t b = 0; b < n_blocks; b++) {
        count_block(h + t, n_tok[b], (uint64_t)b * kBlock, S, runs);
        t += n_tok[b];
    }
    finish_runs(S, runs);
    *out = S;
    return 0;
}

// Diagnostics (not part of the documented ABI; host only): the byte-level
// closure of [start, start + len) of an archive given as host bytes, under a
// match index given as arrays (first[n_blocks + 1], o/ml/src[n_match]).
// Writes the closure's blocks in ascending order to blocks[], each block's
// interval count to iv_count[] and its wanted intervals (start | end << 16)
// to ivs[]; *n_blocks gets the block count.  Returns 0, -1 when a capacity is
// too small, -2 for a corrupt archive.
extern "C" int acx_debug_closure(const uint8_t* h_arc, uint64_t arc_len, const uint64_t* first, uint64_t n_match,
                                 const uint16_t* o, const uint16_t* ml, const uint64_t* src, uint64_t start,
                                 uint64_t len, uint32_t* blocks, uint32_t* iv_count, uint32_t* ivs,
                                 uint32_t cap_blocks, uint32_t cap_ivs, uint32_t* n_blocks) {
    Plan P;
    std::string why;
    if (build_plan(h_arc, arc_len, &P, &why) != 0) return -2;
    if (start > P.total || len > P.total - start) return -1;
    MatchIndex M;
    M.first.assign(first, first + P.n_blocks + 1);
    M.o.assign(o, o + n_match);
    M.ml.assign(ml, ml + n_match);
    M.src.assign(src, src + n_match);
    TickState T;
    WalkJournal J;
    T.begin(P.n_blocks);
    span_walk(P, M, start, len, [](void*, uint32_t) -> const Ivs* { return nullptr; }, nullptr, &T, &J);
    std::vector<uint32_t> bl(T.sched.begin(), T.sched.end());
    std::sort(bl.begin(), bl.end());
    if (bl.size() > cap_blocks) return -1;
    uint32_t k = 0;
    for (size_t i = 0; i < bl.size(); i++) {
        blocks[i] = bl[i];
        const Ivs& v = T.need[bl[i]];
        iv_count[i] = (uint32_t)v.size();
        for (const auto& iv : v) {
            if (k >= cap_ivs) return -1;
            ivs[k++] = iv.first | (iv.second << 16);
        }
    }
    *n_blocks = (uint32_t)bl.size();
    return 0;
}

// Diagnostics (not part of the documented ABI): copy an archive's match index
// to host arrays (first[n_blocks + 1], o/ml/src[cap], bad[n_blocks]); returns
// the number of matches, or -1 (no index, or cap too small).
extern "C" int64_t acx_debug_match_index(const aceapex_archive* A, uint64_t* first, uint16_t* o, uint16_t* ml,
                                         uint64_t* src, uint8_t* bad, uint64_t cap) {
    if (!A || !A->midx) return -1;
    const MatchIndex& M = *A->midx;
    if (M.o.size() > cap) return -1;
    std::copy(M.first.begin(), M.first.end(), first);
    std::copy(M.o.begin(), M.o.end(), o);
    std::copy(M.ml.begin(), M.ml.end(), ml);
    std::copy(M.src.begin(), M.src.end(), src);
    std::copy(M.bad.begin(), M.bad.end(), bad);
    return (int64_t)M.o.size();
}
