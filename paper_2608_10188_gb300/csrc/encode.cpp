// Library encoder for format v1 (host, C++).
//
// Paper, Setup: the encoder performs a global match search and stores every
// back-reference as an absolute position in the output, cut into 16 KiB
// blocks.  "The Last Sequential Element": with no_rep the repeat codes are
// suppressed and every match goes out with an explicit offset, keeping the
// same matches (so the history-free archive differs only in coding).
//
// Match search: a long-window hash (16 bytes, any distance) finds copies
// anywhere earlier; by default it keeps the FIRST occurrence of a window, so a
// copy of a copy points at the original bytes (with absolute offsets this
// costs no offset bits, and it keeps cross-block dependency chains short);
// the short-window hash likewise keeps the oldest occurrence inside its 4 MiB
// window; every output byte's chain depth is tracked and a match whose
// source bytes are already at the depth cap is not taken (paper, "Depth Does
// Not Govern Latency": a depth bound is an encode-time choice, nearly free); a short-window hash (6 bytes,
// recent positions) finds local repeats; the four history distances and
// distances 1..4 are always tried.  A match is taken when its estimated
// saving in bits (length x literal cost - token cost) is positive, which
// keeps chance k-mer hits out of the token stream.  The parse is sequential;
// stream construction, frequency counting and rANS coding run on threads.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace acx {

uint64_t fnv1a64(const uint8_t* p, uint64_t n) {
    uint64_t h = 0xcbf29ce484222325ULL;
    for (uint64_t i = 0; i < n; i++) h = (h ^ p[i]) * 0x100000001b3ULL;
    return h;
}

namespace {

// Default chain-depth cap.  At 16 it costs nothing measurable on the genome
// and 0.02% on text, while bounding the dependency chains the cross-block
// pass must follow.
constexpr uint32_t kDefaultMaxDepth = 16;

struct BlockStreams {
    std::vector<uint8_t> s[4];
    std::vector<uint8_t> lvl;  // per token: its cross-block level (archives with level bodies)
};

inline uint64_t load64(const uint8_t* p) {
    uint64_t v;
    memcpy(&v, p, 8);
    return v;
}

inline uint32_t common_len(const uint8_t* a, const uint8_t* b, uint64_t limit) {
    uint64_t L = 0;
    while (L + 8 <= limit) {
        uint64_t x = load64(a + L) ^ load64(b + L);
        if (x) return (uint32_t)(L + (__builtin_ctzll(x) >> 3));
        L += 8;
    }
    while (L < limit && a[L] == b[L]) L++;
    return (uint32_t)L;
}

// Byte-serial match length allowing overlap (source may run into the destination).
inline uint32_t overlap_len(const uint8_t* s, uint64_t pos, uint64_t src, uint64_t limit) {
    if (pos - src >= 8) return common_len(s + pos, s + src, limit);
    uint64_t L = 0;
    while (L < limit && s[src + L] == s[pos + L]) L++;
    return (uint32_t)L;
}

void put_varint(std::vector<uint8_t>& v, uint32_t x) {
    while (x >= 0x80) {
        v.push_back((uint8_t)(x | 0x80));
        x >>= 7;
    }
    v.push_back((uint8_t)x);
}

// Largest-remainder normalisation of counts to 4096 with every present symbol >= 1.
void normalise(const uint64_t cnt[256], uint16_t f[256]) {
    uint64_t tot = 0;
    for (int s = 0; s < 256; s++) tot += cnt[s];
    memset(f, 0, 512);
    if (!tot) return;
    double rem[256];
    int sum = 0;
    for (int s = 0; s < 256; s++) {
        if (!cnt[s]) { rem[s] = -1; continue; }
        double ideal = (double)cnt[s] * kM / (double)tot;
        int v = (int)ideal;
        if (v < 1) v = 1;
        f[s] = (uint16_t)v;
        rem[s] = ideal - v;
        sum += v;
    }
    while (sum < (int)kM) {  // hand out the remainder by largest fractional part
        int best = -1;
        for (int s = 0; s < 256; s++)
            if (cnt[s] && (best < 0 || rem[s] > rem[best])) best = s;
        f[best]++;
        rem[best] -= 1.0;
        sum++;
    }
    while (sum > (int)kM) {  // too many forced ones: take from the largest entries
        int best = -1;
        for (int s = 0; s < 256; s++)
            if (f[s] > 1 && (best < 0 || f[s] > f[best])) best = s;
        f[best]--;
        sum--;
    }
}

// Interleaved rANS encoder, K lanes; returns body bytes (states padded to 16, then words).
std::vector<uint8_t> rans_encode(const uint8_t* sym, uint32_t n, uint32_t K, const uint16_t f[256]) {
    uint32_t c[256], acc = 0;
    for (int s = 0; s < 256; s++) { c[s] = acc; acc += f[s]; }
    std::vector<uint32_t> x(K, kL);
    std::vector<uint16_t> w;
    w.reserve(n / 2 + 16);
    for (uint32_t i = n; i-- > 0;) {
        uint32_t& st = x[i & (K - 1)];
        const uint32_t fs = f[sym[i]];
        if (st >= (fs << 20)) {
            w.push_back((uint16_t)st);
            st >>= 16;
        }
        st = (st / fs) * kM + st % fs + c[sym[i]];
    }
    const uint32_t hdr = (4 * K + 15) & ~15u;
    std::vector<uint8_t> body(hdr + 2 * w.size(), 0);
    for (uint32_t j = 0; j < K; j++) memcpy(&body[4 * j], &x[j], 4);
    for (size_t k = 0; k < w.size(); k++) memcpy(&body[hdr + 2 * k], &w[w.size() - 1 - k], 2);
    return body;
}

struct Parser {
    const uint8_t* s;
    uint64_t n;
    bool no_rep;
    bool oldest;         // long-window table keeps the first occurrence instead of the latest
    bool short_oldest;   // short-window table keeps the oldest occurrence inside its window
    uint32_t max_depth;  // chain-depth cap (0 = none)
    uint32_t min_match;
    double lit_bits;
    int lbits, sbits;
    std::vector<uint64_t> hl;  // 16-byte window -> most recent position + 1
    std::vector<uint32_t> hs;  // 6-byte window  -> position + 1 (low 32 bits)
    std::vector<uint8_t> depth;  // chain depth of every output byte (0 = literal), saturating
    // every match emitted so far, in output order, and the index of each
    // block's first match (for source forwarding)
    struct Emitted {
        uint64_t dst, src;
        uint32_t len;
    };
    std::vector<Emitted> emitted;
    std::vector<uint64_t> block_first;
    // the parse covers [base, n): sources stay inside it (a segment of a
    // segmented encode), depth[] and block_first[] are indexed from it
    uint64_t base = 0;

    // Follow a non-periodic source window [s, s + w) back through the
    // non-periodic matches that produced it: their bytes equal their sources,
    // so the window can be read at its root instead.  The output is the same;
    // the decoder's cross-block dependency chains become short.
    uint64_t forward(uint64_t s, uint32_t w) const {
        for (int hop = 0; hop < 64; hop++) {
            if (s < base) break;
            const uint64_t b = (s - base) / kBlock;
            if (b >= block_first.size()) break;
            const uint64_t lo = block_first[b];
            const uint64_t hi = b + 1 < block_first.size() ? block_first[b + 1] : emitted.size();
            // last match of the block starting at or before s
            uint64_t a = lo, z = hi;
            while (a < z) {
                const uint64_t m = (a + z) / 2;
                if (emitted[m].dst <= s) a = m + 1; else z = m;
            }
            if (a == lo) break;
            const Emitted& M = emitted[a - 1];
            if (s + w > M.dst + M.len || M.dst - M.src < M.len) break;  // not inside, or periodic
            s = M.src + (s - M.dst);
        }
        return s;
    }

    static inline uint32_t hash_long(const uint8_t* p, int bits) {
        const uint64_t a = load64(p), b = load64(p + 8);
        return (uint32_t)(((a * 0x9E3779B97F4A7C15ULL) ^ (b * 0xC2B2AE3D27D4EB4FULL)) >> (64 - bits));
    }
    static inline uint32_t hash_short(const uint8_t* p, int bits) {
        const uint64_t a = load64(p) & 0xFFFFFFFFFFFFULL;
        return (uint32_t)((a * 0xCF1BBCDCB7A56463ULL) >> (64 - bits));
    }
    void insert(uint64_t p) {
        if (p + 16 <= n) {
            uint64_t& slot = hl[hash_long(s + p, lbits)];
            if (!oldest || !slot) slot = p + 1;
        }
        if (p + 8 <= n) {
            // 32-bit entries: position + 1 modulo 2^32 (only distances below
            // the short window are used, so the high bits are never needed)
            uint32_t& slot = hs[hash_short(s + p, sbits)];
            if (!short_oldest || !slot || (uint32_t)((uint32_t)p - (slot - 1)) >= kShortWindow) slot = (uint32_t)(p + 1);
        }
    }
    static constexpr uint64_t kShortWindow = 1u << 22;
    // deepest chain among the bytes a match would read (its periodic source window)
    uint32_t window_depth(uint64_t pos, uint64_t d, uint32_t L) const {
        const uint64_t w = d < L ? d : L;
        uint32_t m = 0;
        const uint8_t* dp = &depth[pos - d - base];
        for (uint64_t k = 0; k < w; k++) m = m > dp[k] ? m : dp[k];
        return m;
    }
    // cost in bits of a NEW token (cmd + two varints + absolute offset)
    double new_cost(uint64_t src) const {
        int bits = 1;
        while (bits < 40 && (src >> bits)) bits++;
        return 18.0 + bits;
    }

    void parse_block(uint64_t B, uint64_t E, BlockStreams& out, uint64_t& ins) {
        block_first.push_back(emitted.size());
        std::vector<uint8_t>& cmd = out.s[kCmd];
        std::vector<uint8_t>& len = out.s[kLen];
        std::vector<uint8_t>& lit = out.s[kLit];
        std::vector<uint64_t> srcs;
        uint64_t hist[4] = {1, 2, 3, 4};
        uint64_t pos = B, lit0 = B;
        while (pos < E) {
            while (ins < pos) insert(ins++);
            if (pos + 24 <= n) __builtin_prefetch(&hl[hash_long(s + pos + 8, lbits)]);
            const uint64_t limit = E - pos;
            uint32_t bestL = 0, bestDepth = 0;
            uint64_t bestD = 0;
            int bestRep = -1;
            double bestGain = 0.0;
            auto consider = [&](uint64_t d, int rep_idx) {
                if (d == 0 || d > pos - base) return;
                const uint32_t L = overlap_len(s, pos, pos - d, limit);
                if (L < min_match) return;
                int ri = rep_idx;
                if (ri < 0)
                    for (int j = 0; j < 4; j++)
                        if (hist[j] == d) { ri = j; break; }
                // costs in history-mode terms in both modes, so the history-free
                // archive keeps exactly the same matches
                const double cost = ri >= 0 ? 14.0 : new_cost(pos - d);
                const double gain = L * lit_bits - cost;
                if (gain <= bestGain) return;
                const uint32_t sd = window_depth(pos, d, L);
                if (max_depth && sd + 1 > max_depth) return;  // would exceed the chain-depth cap
                bestGain = gain; bestL = L; bestD = d; bestRep = ri; bestDepth = sd + 1;
            };
            for (int j = 0; j < 4; j++) consider(hist[j], j);
            for (uint64_t d = 1; d <= 4; d++) consider(d, -1);
            if (pos + 16 <= n) {
                const uint64_t q = hl[hash_long(s + pos, lbits)];
                if (q) consider(pos - (q - 1), -1);
            }
            if (pos + 8 <= n) {
                const uint32_t q = hs[hash_short(s + pos, sbits)];
                const uint64_t back = (uint32_t)((uint32_t)pos - (q - 1));
                if (q && back > 0 && back < kShortWindow) consider(back, -1);
            }
            if (!bestL) { pos++; continue; }
            if (bestRep < 0 && bestD >= bestL) {
                // an explicit offset: read the same bytes at their root (decided in
                // history-mode terms, so both modes keep identical matches)
                const uint64_t s0 = forward(pos - bestD, bestL);
                if (s0 != pos - bestD) {
                    const uint32_t sd = window_depth(pos, pos - s0, bestL);
                    if (!max_depth || sd + 1 <= max_depth) {
                        bestD = pos - s0;
                        bestDepth = sd + 1;
                        bestRep = -1;
                        for (int j = 0; j < 4; j++)
                            if (hist[j] == bestD) { bestRep = j; break; }
                    }
                }
            }
            memset(&depth[pos - base], bestDepth > 255 ? 255 : (int)bestDepth, bestL);
            emitted.push_back({pos, pos - bestD, bestL});
            const uint32_t LL = (uint32_t)(pos - lit0);
            const bool rep_code = bestRep >= 0 && !no_rep;
            cmd.push_back(rep_code ? (uint8_t)(1 + bestRep) : kNew);
            put_varint(len, LL);
            put_varint(len, bestL);
            lit.insert(lit.end(), s + lit0, s + pos);
            if (!rep_code) srcs.push_back(pos - bestD);
            // the history follows the history-mode rules in both modes
            if (bestRep >= 0) {
                const uint64_t d = hist[bestRep];
                for (int j = bestRep; j > 0; j--) hist[j] = hist[j - 1];
                hist[0] = d;
            } else {
                hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = bestD;
            }
            pos += bestL;
            lit0 = pos;
        }
        if (lit0 < E) {
            cmd.push_back(kLitOnly);
            put_varint(len, (uint32_t)(E - lit0));
            put_varint(len, 0);
            lit.insert(lit.end(), s + lit0, s + E);
        }
        std::vector<uint8_t>& off = out.s[kOff];
        off.resize(5 * srcs.size());
        for (int p = 0; p < 5; p++)
            for (size_t i = 0; i < srcs.size(); i++) off[p * srcs.size() + i] = (uint8_t)(srcs[i] >> (8 * p));
    }
};

template <class F>
void parallel_for(uint32_t n, int threads, F fn) {
    std::atomic<uint32_t> next(0);
    auto work = [&]() {
        for (;;) {
            uint32_t i = next.fetch_add(1);
            if (i >= n) break;
            fn(i);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < threads; t++) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

}  // namespace

int encode_archive(const uint8_t* src, uint64_t n, int no_rep, uint32_t min_match, uint32_t max_lanes, int threads,
                   int latest, uint32_t max_depth, int short_latest, int deps, uint64_t segment, int levels,
                   uint8_t** out, uint64_t* out_len, EncDepthStats* stats) {
    if (segment % kBlock) return -1;
    if (!out || !out_len || (n && !src)) return -1;
    if (min_match == 0) min_match = 4;
    if (max_lanes == 0) max_lanes = 32;
    if (min_match < 4 || min_match > kBlock || max_lanes > kMaxLanes || (max_lanes & (max_lanes - 1))) return -1;
    if (n >= (1ull << 40)) return -1;  // absolute offsets are 40-bit
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    const uint32_t nb = (uint32_t)((n + kBlock - 1) / kBlock);
    std::vector<BlockStreams> blocks(nb);
    // dependency lists: per block, the ascending ids of the earlier blocks
    // holding bytes that its matches read
    std::vector<uint32_t> dep_ids, dep_off(nb, 0), dep_n(nb, 0);
    // chain-depth statistics: each block's deepest byte, each segment's match histogram
    std::vector<uint8_t> blk_depth(stats ? nb : 0, 0);
    try {
        // order-0 literal cost estimate
        uint64_t hist[256] = {0};
        for (uint64_t i = 0; i < n; i++) hist[src[i]]++;
        double H = 0.0;
        for (int c = 0; c < 256; c++)
            if (hist[c]) {
                const double p = (double)hist[c] / (double)n;
                H -= p * log2(p);
            }
        // the parse: one segment, or segments of `segment` bytes parsed in
        // parallel, each with sources inside itself (a genome's chromosomes)
        const uint64_t seg = segment ? segment : std::max<uint64_t>(n, 1);
        const uint32_t n_seg = (uint32_t)((n + seg - 1) / seg);
        std::vector<std::vector<uint32_t>> seg_deps(deps ? nb : 0);
        std::vector<std::vector<uint64_t>> seg_hist(stats ? n_seg : 0);  // per segment: 3 x 256 counts
        std::atomic<int> failed(0);
        auto parse_segment = [&](uint32_t g) {
            try {
                const uint64_t s0 = (uint64_t)g * seg, s1 = std::min<uint64_t>(n, s0 + seg);
                Parser P;
                P.s = src;
                P.n = s1;
                P.base = s0;
                P.no_rep = no_rep != 0;
                P.oldest = latest == 0;
                P.short_oldest = short_latest == 0;
                P.max_depth = max_depth == 0 ? kDefaultMaxDepth : max_depth;
                P.depth.assign(s1 - s0, 0);
                P.min_match = min_match;
                P.lit_bits = std::max(H, 1.0) + 0.1;
                P.lbits = 16;
                while (P.lbits < 27 && (1ull << P.lbits) < s1 - s0) P.lbits++;
                P.sbits = std::min(P.lbits, 22);
                P.hl.assign(1ull << P.lbits, 0);
                P.hs.assign(1ull << P.sbits, 0);
                uint64_t ins = s0;
                const uint32_t b0 = (uint32_t)(s0 / kBlock), b1 = (uint32_t)((s1 + kBlock - 1) / kBlock);
                for (uint32_t b = b0; b < b1; b++) {
                    const uint64_t B = (uint64_t)b * kBlock, E = std::min<uint64_t>(s1, B + kBlock);
                    P.parse_block(B, E, blocks[b], ins);
                }
                // cross-block levels, matches in output order: a match whose
                // source window lies in its own block and holds only level-0
                // bytes is finished by the decoder's local pass (level 0);
                // any other match has 1 + the highest level in its window
                std::vector<uint8_t> mlev;  // per emitted match
                if (stats || levels) {
                    std::vector<uint8_t> lvl(s1 - s0, 0);
                    mlev.resize(P.emitted.size());
                    for (size_t m = 0; m < P.emitted.size(); m++) {
                        const Parser::Emitted& M = P.emitted[m];
                        const uint64_t B = M.dst / kBlock * kBlock, d = M.dst - M.src, w = d < M.len ? d : M.len;
                        uint32_t mx = 0;
                        for (uint64_t q = M.src; q < M.src + w; q++) mx = std::max<uint32_t>(mx, lvl[q - s0]);
                        const uint32_t l = (M.src >= B && mx == 0) ? 0 : std::min<uint32_t>(mx + 1, 255);
                        memset(&lvl[M.dst - s0], (int)l, M.len);
                        mlev[m] = (uint8_t)l;
                    }
                }
                if (levels) {
                    // one level byte per token: the block's matches in order,
                    // then 0 for a closing literal-only token
                    for (uint32_t b = b0; b < b1; b++) {
                        const uint64_t lo = P.block_first[b - b0];
                        const uint64_t hi = b + 1 < b1 ? P.block_first[b + 1 - b0] : P.emitted.size();
                        std::vector<uint8_t>& L = blocks[b].lvl;
                        L.assign(mlev.begin() + lo, mlev.begin() + hi);
                        L.resize(blocks[b].s[kCmd].size(), 0);
                    }
                }
                if (stats) {
                    for (uint32_t b = b0; b < b1; b++) {
                        const uint64_t B = (uint64_t)b * kBlock, E = std::min<uint64_t>(s1, B + kBlock);
                        uint8_t m = 0;
                        for (uint64_t q = B; q < E; q++) m = std::max(m, P.depth[q - s0]);
                        blk_depth[b] = m;
                    }
                    std::vector<uint64_t>& hh = seg_hist[g];
                    hh.assign(3 * 256, 0);
                    for (size_t m = 0; m < P.emitted.size(); m++) {
                        const Parser::Emitted& M = P.emitted[m];
                        hh[P.depth[M.dst - s0]]++;
                        hh[256 + mlev[m]]++;
                        hh[512 + mlev[m]] += M.len;
                    }
                }
                if (deps) {
                    std::vector<uint32_t> ids;
                    for (uint32_t b = b0; b < b1; b++) {
                        const uint64_t lo = P.block_first[b - b0];
                        const uint64_t hi = b + 1 < b1 ? P.block_first[b + 1 - b0] : P.emitted.size();
                        ids.clear();
                        for (uint64_t m = lo; m < hi; m++) {
                            const Parser::Emitted& M = P.emitted[m];
                            const uint64_t d = M.dst - M.src;
                            const uint64_t end = M.src + (d < M.len ? d : M.len);  // bytes the match reads
                            for (uint64_t a = M.src / kBlock; a <= (end - 1) / kBlock && a < b; a++)
                                ids.push_back((uint32_t)a);
                        }
                        std::sort(ids.begin(), ids.end());
                        ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
                        seg_deps[b] = ids;
                    }
                }
            } catch (...) {
                failed = 1;
            }
        };
        parallel_for(n_seg, std::min<int>(threads, (int)std::max<uint32_t>(n_seg, 1)), parse_segment);
        if (failed) return -3;
        if (stats) {
            *stats = EncDepthStats{};
            stats->blocks = nb;
            for (uint32_t b = 0; b < nb; b++) stats->block_max_depth[blk_depth[b]]++;
            for (const std::vector<uint64_t>& hh : seg_hist)
                for (size_t d = 0; d < 256 && d < hh.size(); d++) {
                    stats->match_depth[d] += hh[d];
                    stats->matches += hh[d];
                    stats->match_level[d] += hh[256 + d];
                    stats->level_bytes[d] += hh[512 + d];
                }
        }
        if (deps)
            for (uint32_t b = 0; b < nb; b++) {
                dep_off[b] = (uint32_t)dep_ids.size();
                dep_n[b] = (uint32_t)seg_deps[b].size();
                dep_ids.insert(dep_ids.end(), seg_deps[b].begin(), seg_deps[b].end());
            }
    } catch (...) {
        return -3;
    }
    // global frequency tables
    uint16_t freq[4][256];
    {
        std::vector<std::vector<uint64_t>> part(threads, std::vector<uint64_t>(4 * 256, 0));
        std::atomic<int> tid(0);
        const uint32_t per = (nb + threads - 1) / threads;
        parallel_for((uint32_t)threads, threads, [&](uint32_t t) {
            std::vector<uint64_t>& c = part[t];
            for (uint32_t b = t * per; b < std::min(nb, (t + 1) * per); b++)
                for (int s = 0; s < 4; s++)
                    for (uint8_t v : blocks[b].s[s]) c[s * 256 + v]++;
        });
        (void)tid;
        for (int s = 0; s < 4; s++) {
            uint64_t cnt[256] = {0};
            for (int t = 0; t < threads; t++)
                for (int k = 0; k < 256; k++) cnt[k] += part[t][s * 256 + k];
            normalise(cnt, freq[s]);
        }
    }
    // per-block payloads
    std::vector<std::vector<uint8_t>> pay(nb);
    parallel_for(nb, threads, [&](uint32_t b) {
        std::vector<uint8_t>& P = pay[b];
        P.assign(48, 0);
        // rANS lanes of each stream: powers of two up to max_lanes, at least 64
        // symbols a lane; the three short streams (cmd, len, off) take 16 symbols a
        // lane when their lanes then fit one warp together, which the decoder
        // decodes them on side by side, so that their dependent steps (a lane
        // decodes its symbols in sequence) stay few
        auto lanes_for = [&](uint32_t rn, uint32_t per_lane) {
            uint32_t k = 1;
            while (2 * k <= max_lanes && per_lane * (2 * k) <= rn) k *= 2;
            return k;
        };
        uint32_t lanes[4], short_sum = 0;
        for (int s = 0; s < 4; s++) lanes[s] = lanes_for((uint32_t)blocks[b].s[s].size(), 64);
        for (int s = 0; s < 3; s++) short_sum += lanes_for((uint32_t)blocks[b].s[s].size(), 16);
        if (short_sum <= 32)
            for (int s = 0; s < 3; s++) lanes[s] = lanes_for((uint32_t)blocks[b].s[s].size(), 16);
        for (int s = 0; s < 4; s++) {
            const std::vector<uint8_t>& raw = blocks[b].s[s];
            const uint32_t rn = (uint32_t)raw.size();
            std::vector<uint8_t> body;
            uint8_t mode = 0, K = 0;
            bool table = false;
            {
                uint32_t sum = 0;
                for (int k = 0; k < 256; k++) sum += freq[s][k];
                table = sum == kM;
            }
            if (rn >= 16 && table) {
                const uint32_t k = lanes[s];
                std::vector<uint8_t> enc = rans_encode(raw.data(), rn, k, freq[s]);
                if (enc.size() < rn) {
                    body.swap(enc);
                    mode = 1;
                    K = (uint8_t)k;
                }
            }
            if (!mode) body = raw;
            uint8_t* d = &P[12 * s];
            const uint32_t el = (uint32_t)body.size();
            memcpy(d, &rn, 4);
            memcpy(d + 4, &el, 4);
            d[8] = mode;
            d[9] = K;
            P.insert(P.end(), body.begin(), body.end());
            P.resize((P.size() + 15) & ~(size_t)15, 0);
        }
        if (levels) {  // the level body, stored, after the four stream bodies
            P.insert(P.end(), blocks[b].lvl.begin(), blocks[b].lvl.end());
            P.resize((P.size() + 15) & ~(size_t)15, 0);
        }
        blocks[b] = BlockStreams();
    });
    const uint64_t off_tab = 64, off_idx = 64 + 2048;
    const uint64_t off_deps = deps ? (off_idx + 40ull * nb + 15) & ~15ull : 0;
    const uint64_t off_pay = deps ? (off_deps + 4ull * dep_ids.size() + 15) & ~15ull : (off_idx + 40ull * nb + 15) & ~15ull;
    uint64_t total = off_pay;
    std::vector<uint64_t> poff(nb);
    for (uint32_t b = 0; b < nb; b++) {
        poff[b] = total;
        total += pay[b].size();
    }
    uint8_t* a = (uint8_t*)calloc(total ? total : 1, 1);
    if (!a) return -3;
    memcpy(a, "ACX1", 4);
    const uint16_t ver = 1, flags = (uint16_t)((no_rep ? 1 : 0) | (levels ? kFlagLevels : 0));
    const uint32_t bs = kBlock;
    memcpy(a + 4, &ver, 2);
    memcpy(a + 6, &flags, 2);
    memcpy(a + 8, &bs, 4);
    memcpy(a + 12, &min_match, 4);
    memcpy(a + 16, &n, 8);
    memcpy(a + 24, &nb, 4);
    memcpy(a + 32, &off_tab, 8);
    memcpy(a + 40, &off_idx, 8);
    memcpy(a + 48, &off_deps, 8);
    if (deps && !dep_ids.empty()) memcpy(a + off_deps, dep_ids.data(), 4 * dep_ids.size());
    memcpy(a + 56, &off_pay, 8);
    for (int s = 0; s < 4; s++) memcpy(a + off_tab + 512 * s, freq[s], 512);
    parallel_for(nb, threads, [&](uint32_t b) {
        uint8_t* e = a + off_idx + 40ull * b;
        const uint64_t B = (uint64_t)b * kBlock;
        const uint32_t R = (uint32_t)std::min<uint64_t>(kBlock, n - B);
        const uint32_t pl = (uint32_t)pay[b].size();
        uint32_t ntok;
        memcpy(&ntok, &pay[b][0], 4);  // cmd raw length = token count
        memcpy(e, &poff[b], 8);
        memcpy(e + 8, &pl, 4);
        memcpy(e + 12, &ntok, 4);
        memcpy(e + 16, &R, 4);
        memcpy(e + 20, &dep_off[b], 4);
        memcpy(e + 24, &dep_n[b], 4);
        const uint64_t h = fnv1a64(src + B, R);
        memcpy(e + 32, &h, 8);
        memcpy(a + poff[b], pay[b].data(), pay[b].size());
    });
    *out = a;
    *out_len = total;
    return 0;
}

}  // namespace acx
