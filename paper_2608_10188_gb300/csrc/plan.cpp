// Host-side archive validation and decode-plan construction (format v1).
//
// Everything structural is checked here once per archive (header, tables,
// index, payload descriptors, body bounds), so the kernels only have to
// validate what depends on decoded data (rANS end states, varints, token
// semantics).  The plan is one BlockDev per block plus the rANS decode
// entries of the four global frequency tables.
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace acx {

static inline uint16_t rd16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static inline uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static inline uint64_t rd64(const uint8_t* p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }
static inline uint64_t up16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

static bool lanes_ok(uint32_t K) { return K >= 1 && K <= kMaxLanes && (K & (K - 1)) == 0; }

int build_plan(const uint8_t* a, uint64_t len, Plan* P, std::string* why) {
    auto fail = [&](const char* m) {
        if (why) *why = m;
        return -2;
    };
    if (!a || len < 64) return fail("archive shorter than its header");
    if (memcmp(a, "ACX1", 4) != 0) return fail("bad magic");
    if (rd16(a + 4) != 1) return fail("unsupported version");
    if (rd32(a + 8) != kBlock) return fail("block size is not 16384");
    P->flags = rd16(a + 6);
    P->min_match = rd32(a + 12);
    P->total = rd64(a + 16);
    P->n_blocks = rd32(a + 24);
    const uint64_t off_tab = rd64(a + 32), off_idx = rd64(a + 40), off_deps = rd64(a + 48);
    if (P->min_match < 4 || P->min_match > kBlock) return fail("min_match out of range");
    if ((uint64_t)P->n_blocks != (P->total + kBlock - 1) / kBlock) return fail("block count does not match size");
    if (off_tab > len || len - off_tab < 2048) return fail("tables out of bounds");
    if (off_idx > len || (len - off_idx) / 40 < P->n_blocks) return fail("index out of bounds");
    P->archive_bytes = len;
    // frequency tables -> decode entries sym | (f-1)<<8 | (slot-c)<<20
    P->dtab.assign(4 * kM, 0);
    for (int s = 0; s < 4; s++) {
        uint32_t sum = 0;
        for (int k = 0; k < 256; k++) {
            P->freq[s][k] = rd16(a + off_tab + 512 * s + 2 * k);
            sum += P->freq[s][k];
        }
        if (sum != 0 && sum != kM) return fail("frequency table does not sum to 4096");
        P->table_ok[s] = sum == kM;
        uint32_t c = 0;
        for (int k = 0; k < 256 && P->table_ok[s]; k++) {
            const uint32_t f = P->freq[s][k];
            for (uint32_t r = 0; r < f; r++) P->dtab[s * kM + c + r] = (uint32_t)k | ((f - 1) << 8) | (r << 20);
            c += f;
        }
    }
    P->blk.assign(P->n_blocks, BlockDev{});
    P->has_deps = off_deps != 0;
    const bool has_levels = (P->flags & kFlagLevels) != 0;
    P->lvl_off.assign(has_levels ? P->n_blocks : 0, 0);
    P->deps.clear();
    P->max_tok = 1;
    P->max_lenb = 1;
    P->max_level = 0;
    P->tokens = 0;
    uint64_t scratch = 0;
    for (uint32_t b = 0; b < P->n_blocks; b++) {
        const uint8_t* e = a + off_idx + 40 * (uint64_t)b;
        const uint64_t poff = rd64(e);
        const uint32_t plen = rd32(e + 8), n_tok = rd32(e + 12), raw = rd32(e + 16);
        const uint32_t dep_off = rd32(e + 20), n_deps = rd32(e + 24);
        const uint64_t B = (uint64_t)b * kBlock;
        const uint64_t R = P->total - B < kBlock ? P->total - B : kBlock;
        if (raw != R) return fail("block raw length mismatch");
        if (off_deps == 0 && (dep_off || n_deps)) return fail("dependency list without a dependency section");
        BlockDev& bd = P->blk[b];
        if (off_deps) {
            if (off_deps > len || (len - off_deps) / 4 < (uint64_t)dep_off + n_deps) return fail("deps out of bounds");
            uint32_t prev = 0;
            bd.dep_off = (uint32_t)P->deps.size();
            bd.n_deps = n_deps;
            for (uint32_t k = 0; k < n_deps; k++) {
                const uint32_t id = rd32(a + off_deps + 4 * ((uint64_t)dep_off + k));
                if (id >= b || (k && id <= prev)) return fail("dependency list not ascending below the block");
                prev = id;
                P->deps.push_back(id);
            }
            if (P->deps.size() >= (1ull << 32)) return fail("dependency lists too long");
        }
        if ((poff & 15) || (plen & 15) || plen < 48) return fail("payload misaligned");
        if (poff > len || len - poff < plen) return fail("payload out of bounds");
        const uint8_t* pay = a + poff;
        bd.payload = poff;
        bd.raw_len = raw;
        bd.n_tok = n_tok;
        uint64_t off = 48, soff = 0;
        for (int s = 0; s < 4; s++) {
            const uint8_t* d = pay + 12 * s;
            const uint32_t sraw = rd32(d), enc = rd32(d + 4);
            const uint8_t mode = d[8], K = d[9];
            if (rd16(d + 10) != 0) return fail("descriptor reserved field");
            if (sraw > kMaxStreamRaw) return fail("stream too long");
            if (off + enc > plen) return fail("stream body out of bounds");
            if (mode == 0) {
                if (enc != sraw || K != 0) return fail("stored stream length mismatch");
            } else if (mode == 1) {
                if (sraw == 0 || !lanes_ok(K) || !P->table_ok[s]) return fail("bad rANS stream descriptor");
                const uint32_t hdr = (4u * K + 15) & ~15u;
                if (enc < hdr || ((enc - hdr) & 1)) return fail("bad rANS body length");
                bd.rans_mask |= 1u << s;
            } else {
                return fail("unknown stream mode");
            }
            bd.s_raw[s] = sraw;
            bd.s_body[s] = (uint32_t)off;
            bd.s_enc[s] = enc;
            bd.s_K[s] = K;
            bd.s_off[s] = (uint32_t)soff;
            soff = up16(soff + sraw);
            off = up16(off + enc);
        }
        if (has_levels) {  // the level body: n_tok stored bytes after the four stream bodies
            if (off + n_tok > plen) return fail("level body out of bounds");
            P->lvl_off[b] = (uint32_t)off;
            bd.lvl_body = (uint32_t)off;
            for (uint32_t k = 0; k < n_tok; k++) P->max_level = std::max<uint32_t>(P->max_level, pay[off + k]);
            off = up16(off + n_tok);
        }
        if (off != plen) return fail("payload length mismatch");
        if (bd.s_raw[kCmd] != n_tok) return fail("token count mismatch");
        if (bd.s_raw[kOff] % 5) return fail("offset stream not a multiple of 5");
        // the literals are output bytes of the block (the local pass stages them in a block-sized buffer)
        if (bd.s_raw[kLit] > raw) return fail("literal stream longer than the block");
        bd.n_new = bd.s_raw[kOff] / 5;
        bd.scratch = scratch;
        bd.span_base = (uint32_t)P->span_slots;
        P->span_slots += n_tok + kSpanSlack;
        scratch += soff;
        if (n_tok > P->max_tok) P->max_tok = n_tok;
        if (bd.s_raw[kLen] > P->max_lenb) P->max_lenb = bd.s_raw[kLen];
        P->tokens += n_tok;
        if (P->span_slots >= (1ull << 32)) return fail("too many tokens");
    }
    P->scratch_bytes = scratch + 64;
    return 0;
}

}  // namespace acx
