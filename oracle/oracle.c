/*
 * CPU oracle for format v1 of the blockwise absolute-offset LZ77 codec.
 * TEST INFRASTRUCTURE ONLY (see oracle.h): loaded by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; never by the product library.
 *
 * Layout of an archive (all integers little-endian):
 *   header   64 B   "ACX1", u16 version=1, u16 flags (bit0: history-free
 *                   encoding, informational; bit1: every payload carries
 *                   a level body), u32 block_size=16384,
 *                   u32 min_match, u64 total, u32 n_blocks, u32 0,
 *                   u64 off_tables, u64 off_index, u64 off_deps (0 = none),
 *                   u64 off_payload
 *   tables   4 x 256 x u16  frequencies of the cmd, len, off and lit
 *                   streams (each sums to 4096, or is all zero)
 *   index    40 B per block: u64 payload_off, u32 payload_len, u32 n_tokens,
 *                   u32 raw_len, u32 dep_off, u32 n_deps, u32 0, u64 fnv1a64
 *   deps     optional u32 source-block ids (ascending, < own id); when the
 *            section is present, every block other than its own that a
 *            match reads must be listed (else the archive is corrupt)
 *   payload  per block, 16-aligned: 4 descriptors of 12 B (u32 raw_len,
 *            u32 enc_len, u8 mode (0 stored, 1 rANS), u8 K, u16 0) in the
 *            order cmd, len, off, lit, then the 4 bodies, each starting on a
 *            16-byte boundary; with flags bit1 a fifth, stored body of
 *            n_tokens bytes follows at the next 16-byte boundary: each
 *            token's cross-block level (a scheduling hint for decoders that
 *            take cross-block copies level by level, the paper's waves;
 *            "Depth Does Not Govern Latency"; it never changes the decoded
 *            bytes and is not checked); payload_len = end of the last body
 *            rounded up to 16.
 *
 * Streams of a block with n tokens (paper, Setup: literals, lengths,
 * absolute offsets, commands):
 *   cmd  n bytes: 0 NEW (explicit offset), 1..4 REP0..REP3 (distance from
 *        the 4-entry history), 5 LIT_ONLY (last token only, no match)
 *   len  LEB128 varints, two per token (literal-run length LL, then match
 *        length ML), each at most 3 bytes
 *   off  5 byte planes of the NEW tokens' absolute source positions (u40):
 *        plane p holds byte p of every offset
 *   lit  the literal bytes in token order
 */
#include "oracle.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ---- little-endian helpers ------------------------------------------------ */
static uint16_t rd16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t rd64(const uint8_t* p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }
static void wr16(uint8_t* p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void wr32(uint8_t* p, uint32_t v) {
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void wr64(uint8_t* p, uint64_t v) {
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint64_t pad16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

/* ---- FNV-1a 64 ------------------------------------------------------------ */
uint64_t orc_fnv1a64(const uint8_t* p, uint64_t n) {
    uint64_t h = 0xcbf29ce484222325ULL;
    for (uint64_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

void orc_free(void* p) { free(p); }

/* ---- frequency normalisation ---------------------------------------------- */
int orc_normalize(const uint64_t counts[256], uint16_t freq[256]) {
    uint64_t total = 0;
    for (int s = 0; s < 256; s++) total += counts[s];
    memset(freq, 0, 256 * sizeof(uint16_t));
    if (total == 0) return ORC_OK;
    int64_t sum = 0;
    int best = -1;
    for (int s = 0; s < 256; s++) {
        if (!counts[s]) continue;
        uint64_t f = (counts[s] * ORC_M + total / 2) / total;
        if (f < 1) f = 1;
        freq[s] = (uint16_t)f;
        sum += (int64_t)f;
        if (best < 0 || counts[s] > counts[best]) best = s;
    }
    /* fix the sum: give surplus to / take deficit from the largest entries */
    while (sum != (int64_t)ORC_M) {
        if (sum < (int64_t)ORC_M) {
            freq[best] += (uint16_t)((int64_t)ORC_M - sum);
            sum = ORC_M;
        } else {
            int big = -1;
            for (int s = 0; s < 256; s++)
                if (freq[s] > 1 && (big < 0 || freq[s] > freq[big])) big = s;
            if (big < 0) return ORC_E_ARG; /* more than 4096 distinct symbols: impossible for bytes */
            freq[big]--;
            sum--;
        }
    }
    return ORC_OK;
}

static int table_sum(const uint16_t freq[256]) {
    int sum = 0;
    for (int s = 0; s < 256; s++) sum += freq[s];
    return sum;
}

/* ---- rANS ------------------------------------------------------------------ */
static int valid_lanes(uint32_t K) { return K >= 1 && K <= 128 && (K & (K - 1)) == 0; }

int64_t orc_rans_encode(const uint8_t* sym, uint32_t n, uint32_t K, const uint16_t freq[256], uint8_t* out,
                        uint64_t cap) {
    if (!valid_lanes(K) || table_sum(freq) != (int)ORC_M) return ORC_E_ARG;
    uint32_t cum[256];
    uint32_t c = 0;
    for (int s = 0; s < 256; s++) { cum[s] = c; c += freq[s]; }
    for (uint32_t i = 0; i < n; i++)
        if (!freq[sym[i]]) return ORC_E_ARG;
    uint32_t x[128];
    for (uint32_t j = 0; j < K; j++) x[j] = ORC_L;
    uint16_t* words = (uint16_t*)malloc(sizeof(uint16_t) * (n + 1));
    if (!words) return ORC_E_NOMEM;
    uint64_t nw = 0;
    /* symbols are encoded last-to-first; symbol i belongs to lane i mod K */
    for (uint32_t ii = n; ii-- > 0;) {
        uint32_t j = ii % K, s = sym[ii], f = freq[s];
        if ((uint64_t)x[j] >= ((uint64_t)f << 20)) {
            words[nw++] = (uint16_t)(x[j] & 0xffff);
            x[j] >>= 16;
        }
        x[j] = (x[j] / f) * ORC_M + (x[j] % f) + cum[s];
    }
    uint64_t hdr = pad16(4 * (uint64_t)K);
    uint64_t len = hdr + 2 * nw;
    if (len > cap) { free(words); return ORC_E_ARG; }
    memset(out, 0, hdr);
    for (uint32_t j = 0; j < K; j++) wr32(out + 4 * j, x[j]);
    /* the decoder consumes words in the reverse of emission order */
    for (uint64_t k = 0; k < nw; k++) wr16(out + hdr + 2 * k, words[nw - 1 - k]);
    free(words);
    return (int64_t)len;
}

int orc_rans_decode(const uint8_t* body, uint64_t enc_len, uint32_t n, uint32_t K, const uint16_t freq[256],
                    uint8_t* out) {
    if (!valid_lanes(K) || table_sum(freq) != (int)ORC_M) return ORC_E_CORRUPT;
    uint64_t hdr = pad16(4 * (uint64_t)K);
    if (enc_len < hdr || ((enc_len - hdr) & 1)) return ORC_E_CORRUPT;
    uint64_t W = (enc_len - hdr) / 2;
    uint8_t slot2sym[ORC_M];
    uint32_t cum[256];
    uint32_t c = 0;
    for (int s = 0; s < 256; s++) {
        cum[s] = c;
        for (uint32_t k = 0; k < freq[s]; k++) slot2sym[c + k] = (uint8_t)s;
        c += freq[s];
    }
    uint32_t x[128];
    for (uint32_t j = 0; j < K; j++) {
        x[j] = rd32(body + 4 * j);
        if (x[j] < ORC_L) return ORC_E_CORRUPT;
    }
    const uint8_t* w = body + hdr;
    uint64_t p = 0;
    for (uint32_t i = 0; i < n; i++) {
        uint32_t j = i % K;
        uint32_t slot = x[j] & (ORC_M - 1);
        uint32_t s = slot2sym[slot];
        out[i] = (uint8_t)s;
        x[j] = freq[s] * (x[j] >> ORC_PROB_BITS) + slot - cum[s];
        if (x[j] < ORC_L) {
            if (p >= W) return ORC_E_CORRUPT;
            x[j] = (x[j] << 16) | rd16(w + 2 * p);
            p++;
        }
    }
    if (p != W) return ORC_E_CORRUPT;
    for (uint32_t j = 0; j < K; j++)
        if (x[j] != ORC_L) return ORC_E_CORRUPT;
    return ORC_OK;
}

/* ---- growable byte buffer --------------------------------------------------- */
typedef struct { uint8_t* p; uint64_t n, cap; } buf_t;

static int buf_reserve(buf_t* b, uint64_t extra) {
    if (b->n + extra <= b->cap) return 0;
    uint64_t nc = b->cap ? b->cap : 256;
    while (nc < b->n + extra) nc *= 2;
    uint8_t* q = (uint8_t*)realloc(b->p, nc);
    if (!q) return -1;
    b->p = q;
    b->cap = nc;
    return 0;
}
static int buf_put(buf_t* b, uint8_t v) {
    if (buf_reserve(b, 1)) return -1;
    b->p[b->n++] = v;
    return 0;
}
static int buf_leb(buf_t* b, uint32_t v) {
    while (v >= 0x80) {
        if (buf_put(b, (uint8_t)((v & 0x7f) | 0x80))) return -1;
        v >>= 7;
    }
    return buf_put(b, (uint8_t)v);
}

/* ---- encoder ------------------------------------------------------------------ */
void orc_enc_defaults(orc_enc_params* p) {
    p->no_rep = 0;
    p->min_match = 4;
    p->new_min = 8;
    p->max_lanes = 32;
    p->chain = 16;
}

typedef struct {
    buf_t s[4];     /* cmd, len, off, lit raw streams */
    uint64_t* src;  /* NEW sources, before plane split */
    uint64_t n_new, cap_new;
    uint32_t n_tok;
} blk_t;

static uint32_t hash8(const uint8_t* p, int bits) {
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
    return (uint32_t)((v * 0x9E3779B97F4A7C15ULL) >> (64 - bits));
}

static uint32_t match_len(const uint8_t* s, uint64_t pos, uint64_t src, uint64_t limit) {
    uint64_t L = 0;
    while (L < limit && s[src + L] == s[pos + L]) L++;
    return (uint32_t)L;
}

static int blk_token(blk_t* bk, uint8_t cmd, uint32_t LL, uint32_t ML, const uint8_t* lits, int is_new,
                     uint64_t src) {
    if (buf_put(&bk->s[ORC_CMD], cmd)) return -1;
    if (buf_leb(&bk->s[ORC_LEN], LL) || buf_leb(&bk->s[ORC_LEN], ML)) return -1;
    if (buf_reserve(&bk->s[ORC_LIT], LL)) return -1;
    if (LL) memcpy(bk->s[ORC_LIT].p + bk->s[ORC_LIT].n, lits, LL);  /* (an empty buffer may have no storage yet) */
    bk->s[ORC_LIT].n += LL;
    if (is_new) {
        if (bk->n_new == bk->cap_new) {
            uint64_t nc = bk->cap_new ? 2 * bk->cap_new : 64;
            uint64_t* q = (uint64_t*)realloc(bk->src, nc * sizeof(uint64_t));
            if (!q) return -1;
            bk->src = q;
            bk->cap_new = nc;
        }
        bk->src[bk->n_new++] = src;
    }
    bk->n_tok++;
    return 0;
}

static void blk_free(blk_t* bk) {
    for (int s = 0; s < 4; s++) free(bk->s[s].p);
    free(bk->src);
}

int orc_encode(const uint8_t* src, uint64_t n, const orc_enc_params* prm, uint8_t** out, uint64_t* out_len) {
    orc_enc_params P;
    if (prm) P = *prm; else orc_enc_defaults(&P);
    if (!out || !out_len || (n && !src)) return ORC_E_ARG;
    if (P.min_match < 4 || P.min_match > 16384 || !valid_lanes(P.max_lanes)) return ORC_E_ARG;
    if (P.new_min < P.min_match) P.new_min = P.min_match;
    if (n >= ((uint64_t)1 << 32)) return ORC_E_ARG; /* the oracle encoder is for test-sized inputs */
    uint32_t nb = (uint32_t)((n + ORC_BLOCK - 1) / ORC_BLOCK);
    blk_t* blks = (blk_t*)calloc(nb ? nb : 1, sizeof(blk_t));
    int hbits = 16;
    while (hbits < 24 && ((uint64_t)1 << hbits) < n) hbits++;
    uint32_t* head = (uint32_t*)malloc(sizeof(uint32_t) << hbits);
    uint32_t* chain = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!blks || !head || !chain) { free(blks); free(head); free(chain); return ORC_E_NOMEM; }
    memset(head, 0xff, sizeof(uint32_t) << hbits);
    int rc = ORC_OK;
    uint64_t ins = 0; /* positions < ins are in the hash chains */
#define INSERT_UPTO(lim)                                          \
    for (; ins < (lim) && ins + 8 <= n; ins++) {                  \
        uint32_t h_ = hash8(src + ins, hbits);                    \
        chain[ins] = head[h_];                                    \
        head[h_] = (uint32_t)ins;                                 \
    }
    for (uint32_t b = 0; b < nb && rc == ORC_OK; b++) {
        blk_t* bk = &blks[b];
        uint64_t B = (uint64_t)b * ORC_BLOCK, E = B + ORC_BLOCK < n ? B + ORC_BLOCK : n;
        uint64_t hist[4] = {1, 2, 3, 4}; /* history resets at every block */
        uint64_t pos = B, lit0 = B;
        while (pos < E) {
            uint64_t limit = E - pos;
            uint32_t best = 0;
            uint64_t bd = 0;
            int brep = -1;
            for (int j = 0; j < 4; j++) {
                uint64_t d = hist[j];
                if (d > pos) continue;
                uint32_t L = match_len(src, pos, pos - d, limit);
                if (L >= P.min_match && L > best) { best = L; bd = d; brep = j; }
            }
            if (pos + 8 <= n) {
                INSERT_UPTO(pos);
                uint32_t cand = head[hash8(src + pos, hbits)];
                for (uint32_t k = 0; k < P.chain && cand != 0xffffffffu; k++) {
                    uint32_t L = match_len(src, pos, cand, limit);
                    if (L >= P.new_min && L > best) {
                        uint64_t d = pos - cand;
                        best = L;
                        bd = d;
                        brep = -1;
                        for (int j = 0; j < 4; j++)
                            if (hist[j] == d) { brep = j; break; }
                    }
                    cand = chain[cand];
                }
            }
            if (best == 0) { pos++; continue; }
            /* emit: repeat code if the distance is in the history (history mode),
             * else an explicit absolute offset */
            uint32_t LL = (uint32_t)(pos - lit0);
            int code_rep = (brep >= 0 && !P.no_rep);
            uint8_t cmd = code_rep ? (uint8_t)(1 + brep) : 0;
            if (blk_token(bk, cmd, LL, best, src + lit0, !code_rep, pos - bd)) { rc = ORC_E_NOMEM; break; }
            /* the encoder's history follows the history-mode semantics in both
             * modes, so the history-free archive keeps exactly the same matches */
            if (brep >= 0) {
                uint64_t d = hist[brep];
                for (int j = brep; j > 0; j--) hist[j] = hist[j - 1];
                hist[0] = d;
            } else {
                hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = bd;
            }
            pos += best;
            lit0 = pos;
        }
        if (rc == ORC_OK && lit0 < E) {
            if (blk_token(bk, 5, (uint32_t)(E - lit0), 0, src + lit0, 0, 0)) rc = ORC_E_NOMEM;
        }
        /* split NEW offsets into 5 byte planes */
        if (rc == ORC_OK && bk->n_new) {
            buf_t* o = &bk->s[ORC_OFF];
            if (buf_reserve(o, 5 * bk->n_new)) { rc = ORC_E_NOMEM; break; }
            for (int p = 0; p < 5; p++)
                for (uint64_t i = 0; i < bk->n_new; i++) o->p[o->n++] = (uint8_t)(bk->src[i] >> (8 * p));
        }
    }
#undef INSERT_UPTO
    free(head);
    free(chain);
    if (rc != ORC_OK) {
        for (uint32_t b = 0; b < nb; b++) blk_free(&blks[b]);
        free(blks);
        return rc;
    }
    /* global frequency tables per stream type */
    uint16_t freq[4][256];
    for (int s = 0; s < 4; s++) {
        uint64_t cnt[256] = {0};
        for (uint32_t b = 0; b < nb; b++)
            for (uint64_t i = 0; i < blks[b].s[s].n; i++) cnt[blks[b].s[s].p[i]]++;
        orc_normalize(cnt, freq[s]);
    }
    /* per-block payloads */
    buf_t pay = {0};
    uint64_t* poff = (uint64_t*)malloc(sizeof(uint64_t) * (nb ? nb : 1));
    uint32_t* plen = (uint32_t*)malloc(sizeof(uint32_t) * (nb ? nb : 1));
    uint8_t* tmp = (uint8_t*)malloc(2 * ORC_BLOCK * 4 + 1024);
    if (!poff || !plen || !tmp) rc = ORC_E_NOMEM;
    for (uint32_t b = 0; b < nb && rc == ORC_OK; b++) {
        blk_t* bk = &blks[b];
        uint64_t base = pay.n;
        if (buf_reserve(&pay, 48)) { rc = ORC_E_NOMEM; break; }
        memset(pay.p + base, 0, 48);
        pay.n += 48;
        for (int s = 0; s < 4; s++) {
            uint32_t raw = (uint32_t)bk->s[s].n;
            uint8_t mode = 0, K = 0;
            int64_t enc = -1;
            if (raw >= 16 && table_sum(freq[s]) == (int)ORC_M) {
                uint32_t k = 1;
                while (2 * k <= P.max_lanes && 64 * (2 * k) <= raw) k *= 2;
                uint64_t cap = pad16(4 * k) + 2 * (uint64_t)raw + 16;
                uint8_t* t = cap <= 2 * ORC_BLOCK * 4 + 1024 ? tmp : (uint8_t*)malloc(cap);
                enc = orc_rans_encode(bk->s[s].p, raw, k, freq[s], t, cap);
                if (enc >= 0 && (uint64_t)enc < raw) {
                    mode = 1;
                    K = (uint8_t)k;
                    if (buf_reserve(&pay, pad16((uint64_t)enc))) rc = ORC_E_NOMEM;
                    else {
                        memset(pay.p + pay.n, 0, pad16((uint64_t)enc));
                        memcpy(pay.p + pay.n, t, (size_t)enc);
                    }
                }
                if (t != tmp) free(t);
            }
            if (rc != ORC_OK) break;
            if (!mode) {
                enc = raw;
                if (buf_reserve(&pay, pad16(raw))) { rc = ORC_E_NOMEM; break; }
                memset(pay.p + pay.n, 0, pad16(raw));
                if (raw) memcpy(pay.p + pay.n, bk->s[s].p, raw);
            }
            uint8_t* d = pay.p + base + 12 * s;
            wr32(d, raw);
            wr32(d + 4, (uint32_t)enc);
            d[8] = mode;
            d[9] = K;
            pay.n += pad16((uint64_t)enc);
        }
        poff[b] = base;
        plen[b] = (uint32_t)(pay.n - base);
    }
    if (rc == ORC_OK) {
        uint64_t off_tables = 64, off_index = 64 + 2048, off_payload = pad16(off_index + 40 * (uint64_t)nb);
        uint64_t total = off_payload + pay.n;
        uint8_t* a = (uint8_t*)calloc(total ? total : 1, 1);
        if (!a) rc = ORC_E_NOMEM;
        else {
            memcpy(a, "ACX1", 4);
            wr16(a + 4, 1);
            wr16(a + 6, P.no_rep ? 1 : 0);
            wr32(a + 8, ORC_BLOCK);
            wr32(a + 12, P.min_match);
            wr64(a + 16, n);
            wr32(a + 24, nb);
            wr64(a + 32, off_tables);
            wr64(a + 40, off_index);
            wr64(a + 48, 0);
            wr64(a + 56, off_payload);
            for (int s = 0; s < 4; s++)
                for (int k = 0; k < 256; k++) wr16(a + off_tables + 512 * s + 2 * k, freq[s][k]);
            for (uint32_t b = 0; b < nb; b++) {
                uint8_t* e = a + off_index + 40 * (uint64_t)b;
                uint64_t B = (uint64_t)b * ORC_BLOCK;
                uint32_t R = (uint32_t)(n - B < ORC_BLOCK ? n - B : ORC_BLOCK);
                wr64(e, off_payload + poff[b]);
                wr32(e + 8, plen[b]);
                wr32(e + 12, blks[b].n_tok);
                wr32(e + 16, R);
                wr32(e + 20, 0);
                wr32(e + 24, 0);
                wr32(e + 28, 0);
                wr64(e + 32, orc_fnv1a64(src + B, R));
            }
            if (pay.n) memcpy(a + off_payload, pay.p, pay.n);
            *out = a;
            *out_len = total;
        }
    }
    free(pay.p);
    free(poff);
    free(plen);
    free(tmp);
    for (uint32_t b = 0; b < nb; b++) blk_free(&blks[b]);
    free(blks);
    return rc;
}

/* ---- archive reading ------------------------------------------------------------ */
typedef struct {
    const uint8_t* a;
    uint64_t len, total, off_tables, off_index, off_deps, off_payload;
    uint32_t nb, flags, min_match;
    uint16_t freq[4][256];
} arc_t;

static int arc_open(const uint8_t* a, uint64_t len, arc_t* A) {
    if (!a || len < 64) return ORC_E_CORRUPT;
    if (memcmp(a, "ACX1", 4) != 0 || rd16(a + 4) != 1) return ORC_E_CORRUPT;
    if (rd32(a + 8) != ORC_BLOCK) return ORC_E_CORRUPT;
    A->a = a;
    A->len = len;
    A->flags = rd16(a + 6);
    A->min_match = rd32(a + 12);
    A->total = rd64(a + 16);
    A->nb = rd32(a + 24);
    A->off_tables = rd64(a + 32);
    A->off_index = rd64(a + 40);
    A->off_deps = rd64(a + 48);
    A->off_payload = rd64(a + 56);
    if (A->min_match < 4 || A->min_match > ORC_BLOCK) return ORC_E_CORRUPT;
    if (A->nb != (A->total + ORC_BLOCK - 1) / ORC_BLOCK) return ORC_E_CORRUPT;
    if (A->off_tables > len || len - A->off_tables < 2048) return ORC_E_CORRUPT;
    if (A->off_index > len || (len - A->off_index) / 40 < A->nb) return ORC_E_CORRUPT;
    if (A->off_payload > len) return ORC_E_CORRUPT;
    for (int s = 0; s < 4; s++) {
        for (int k = 0; k < 256; k++) A->freq[s][k] = rd16(a + A->off_tables + 512 * s + 2 * k);
        int sum = table_sum(A->freq[s]);
        if (sum != 0 && sum != (int)ORC_M) return ORC_E_CORRUPT;
    }
    return ORC_OK;
}

int orc_info(const uint8_t* arc, uint64_t arc_len, uint64_t* total, uint32_t* n_blocks, uint32_t* flags,
             uint32_t* min_match) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    if (total) *total = A.total;
    if (n_blocks) *n_blocks = A.nb;
    if (flags) *flags = A.flags;
    if (min_match) *min_match = A.min_match;
    return ORC_OK;
}

typedef struct {
    uint32_t raw_len, n_tok, payload_len;
    uint32_t dep_off, n_deps; /* dependency list (archives that carry lists) */
    uint64_t payload_off, fnv;
    uint8_t* s[4];      /* decoded streams (malloc'ed) */
    uint32_t n[4];      /* their lengths */
    uint64_t enc[4];
    uint64_t lvl_off;   /* payload offset of the level body (flags bit1), else 0 */
} dblk_t;

static void dblk_free(dblk_t* d) {
    for (int s = 0; s < 4; s++) free(d->s[s]);
}

/* Read the index entry of block b and entropy-decode its four streams. */
static int block_streams(const arc_t* A, uint32_t b, dblk_t* d) {
    memset(d, 0, sizeof *d);
    const uint8_t* e = A->a + A->off_index + 40 * (uint64_t)b;
    d->payload_off = rd64(e);
    d->payload_len = rd32(e + 8);
    d->n_tok = rd32(e + 12);
    d->raw_len = rd32(e + 16);
    uint32_t dep_off = rd32(e + 20), n_deps = rd32(e + 24);
    d->dep_off = dep_off;
    d->n_deps = n_deps;
    d->fnv = rd64(e + 32);
    uint64_t B = (uint64_t)b * ORC_BLOCK;
    uint64_t R = A->total - B < ORC_BLOCK ? A->total - B : ORC_BLOCK;
    if (d->raw_len != R) return ORC_E_CORRUPT;
    if (A->off_deps == 0 && (dep_off || n_deps)) return ORC_E_CORRUPT;
    if (A->off_deps) {
        if (A->off_deps > A->len || (A->len - A->off_deps) / 4 < (uint64_t)dep_off + n_deps) return ORC_E_CORRUPT;
        for (uint32_t k = 0; k < n_deps; k++) {
            uint32_t id = rd32(A->a + A->off_deps + 4 * ((uint64_t)dep_off + k));
            if (id >= b) return ORC_E_CORRUPT;
            if (k && id <= rd32(A->a + A->off_deps + 4 * ((uint64_t)dep_off + k - 1))) return ORC_E_CORRUPT;
        }
    }
    if ((d->payload_off & 15) || (d->payload_len & 15) || d->payload_len < 48) return ORC_E_CORRUPT;
    if (d->payload_off > A->len || A->len - d->payload_off < d->payload_len) return ORC_E_CORRUPT;
    const uint8_t* P = A->a + d->payload_off;
    uint64_t off = 48;
    for (int s = 0; s < 4; s++) {
        const uint8_t* ds = P + 12 * s;
        uint32_t raw = rd32(ds), enc = rd32(ds + 4);
        uint8_t mode = ds[8], K = ds[9];
        if (rd16(ds + 10) != 0) return ORC_E_CORRUPT;
        if (off + enc > d->payload_len) return ORC_E_CORRUPT;
        if (raw > 4 * ORC_BLOCK + 16) return ORC_E_CORRUPT;
        d->n[s] = raw;
        d->enc[s] = enc;
        d->s[s] = (uint8_t*)malloc(raw ? raw : 1);
        if (!d->s[s]) return ORC_E_NOMEM;
        if (mode == 0) {
            if (enc != raw || K != 0) return ORC_E_CORRUPT;
            memcpy(d->s[s], P + off, raw);
        } else if (mode == 1) {
            if (raw == 0 || !valid_lanes(K) || table_sum(A->freq[s]) != (int)ORC_M) return ORC_E_CORRUPT;
            int rc = orc_rans_decode(P + off, enc, raw, K, A->freq[s], d->s[s]);
            if (rc) return rc;
        } else {
            return ORC_E_CORRUPT;
        }
        off = pad16(off + enc);
    }
    if (A->flags & 2) {  /* the level body: n_tok stored bytes */
        if (off + d->n_tok > d->payload_len) return ORC_E_CORRUPT;
        d->lvl_off = off;
        off = pad16(off + d->n_tok);
    }
    if (off != d->payload_len) return ORC_E_CORRUPT;
    if (d->n[ORC_CMD] != d->n_tok) return ORC_E_CORRUPT;
    if (d->n[ORC_OFF] % 5) return ORC_E_CORRUPT;
    return ORC_OK;
}

/* The sequential parse and byte-serial decode of one block.  When out is
 * NULL only the parse runs.  tok_* arrays (optional) receive the per-token
 * parse. */
typedef struct {
    uint8_t* cmd;
    uint32_t *ll, *ml, *lit;
    uint64_t *dst, *src;
    uint64_t cap;
} tok_out_t;

/* Format v1 dependency lists: the match at pos reading from src reads the
 * bytes [src, src + min(ML, pos - src)) (a self-overlapping match reads one
 * period); every block of that window other than block b itself must appear
 * in block b's list. */
static int deps_cover(const arc_t* A, const dblk_t* d, uint32_t b, uint64_t src, uint64_t pos, uint32_t ML) {
    uint64_t dist = pos - src;
    uint64_t end = src + (dist < ML ? dist : ML);
    for (uint64_t blk = src / ORC_BLOCK; blk <= (end - 1) / ORC_BLOCK; blk++) {
        if (blk == b) continue;
        int found = 0;
        for (uint32_t k = 0; k < d->n_deps; k++)
            if (rd32(A->a + A->off_deps + 4 * ((uint64_t)d->dep_off + k)) == blk) found = 1;
        if (!found) return 0;
    }
    return 1;
}

static int block_decode(const arc_t* A, uint32_t b, const dblk_t* d, uint8_t* out, tok_out_t* T) {
    uint64_t B = (uint64_t)b * ORC_BLOCK, R = d->raw_len, E = B + R;
    const uint8_t* cmd = d->s[ORC_CMD];
    const uint8_t* lb = d->s[ORC_LEN];
    const uint8_t* off = d->s[ORC_OFF];
    const uint8_t* lit = d->s[ORC_LIT];
    uint32_t n_len = d->n[ORC_LEN], n_lit = d->n[ORC_LIT];
    uint64_t n_new = d->n[ORC_OFF] / 5;
    uint64_t hist[4] = {1, 2, 3, 4}; /* initial history, reset per block */
    uint64_t pos = B, lp = 0, ni = 0;
    uint32_t vp = 0; /* read position in the len stream */
    for (uint32_t i = 0; i < d->n_tok; i++) {
        uint32_t v[2];
        for (int q = 0; q < 2; q++) {
            uint32_t val = 0;
            int k = 0;
            for (;;) {
                if (vp >= n_len || k == 3) return ORC_E_CORRUPT;
                uint8_t c = lb[vp++];
                val |= (uint32_t)(c & 0x7f) << (7 * k);
                k++;
                if (c < 0x80) break;
            }
            v[q] = val;
        }
        uint32_t LL = v[0], ML = v[1];
        uint8_t k = cmd[i];
        if (LL > E - pos || LL > n_lit - lp) return ORC_E_CORRUPT;
        if (out) for (uint32_t j = 0; j < LL; j++) out[pos + j] = lit[lp + j];
        uint64_t lit_i = lp;
        pos += LL;
        lp += LL;
        uint64_t src = 0;
        if (k == 5) {
            if (ML != 0 || i != d->n_tok - 1 || LL == 0) return ORC_E_CORRUPT;
        } else if (k == 0) {
            if (ni >= n_new) return ORC_E_CORRUPT;
            src = 0;
            for (int p = 0; p < 5; p++) src |= (uint64_t)off[p * n_new + ni] << (8 * p);
            ni++;
            if (src >= pos) return ORC_E_CORRUPT; /* every absolute offset precedes its destination */
            uint64_t dd = pos - src;
            hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = dd;
        } else if (k <= 4) {
            int j = k - 1;
            uint64_t dd = hist[j];
            if (dd < 1 || dd > pos) return ORC_E_CORRUPT;
            src = pos - dd;
            for (int q = j; q > 0; q--) hist[q] = hist[q - 1]; /* move entry j to the front */
            hist[0] = dd;
        } else {
            return ORC_E_CORRUPT;
        }
        if (k != 5) {
            if (ML < A->min_match || ML > E - pos) return ORC_E_CORRUPT;
            if (A->off_deps && src < B && !deps_cover(A, d, b, src, pos, ML)) return ORC_E_CORRUPT;
            if (out) for (uint32_t j = 0; j < ML; j++) out[pos + j] = out[src + j]; /* byte-serial */
        }
        if (T && i < T->cap) {
            if (T->cmd) T->cmd[i] = k;
            if (T->ll) T->ll[i] = LL;
            if (T->ml) T->ml[i] = ML;
            if (T->dst) T->dst[i] = pos;
            if (T->src) T->src[i] = src;
            if (T->lit) T->lit[i] = (uint32_t)lit_i;
        }
        pos += ML;
    }
    if (pos != E || lp != n_lit || ni != n_new || vp != n_len) return ORC_E_CORRUPT;
    return ORC_OK;
}

int orc_decode(const uint8_t* arc, uint64_t arc_len, uint8_t* out, uint64_t out_cap, int verify_fnv) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    if (!out && A.total) return ORC_E_ARG;
    if (out_cap < A.total) return ORC_E_ARG;
    for (uint32_t b = 0; b < A.nb; b++) {
        dblk_t d;
        rc = block_streams(&A, b, &d);
        if (rc == ORC_OK) rc = block_decode(&A, b, &d, out, NULL);
        dblk_free(&d);
        if (rc) return rc;
        if (verify_fnv && orc_fnv1a64(out + (uint64_t)b * ORC_BLOCK, d.raw_len) != d.fnv) return ORC_E_CORRUPT;
    }
    return ORC_OK;
}

int64_t orc_parse_block(const uint8_t* arc, uint64_t arc_len, uint32_t b, uint64_t cap, uint8_t* cmd,
                        uint32_t* ll, uint32_t* ml, uint64_t* dst, uint64_t* src, uint32_t* lit) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    if (b >= A.nb) return ORC_E_ARG;
    dblk_t d;
    rc = block_streams(&A, b, &d);
    tok_out_t T = {cmd, ll, ml, lit, dst, src, cap};
    if (rc == ORC_OK) rc = block_decode(&A, b, &d, NULL, &T);
    int64_t n = d.n_tok;
    dblk_free(&d);
    return rc ? rc : n;
}

int64_t orc_block_stream(const uint8_t* arc, uint64_t arc_len, uint32_t b, int which, uint8_t* out, uint64_t cap) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    if (b >= A.nb || which < 0 || which > 3) return ORC_E_ARG;
    dblk_t d;
    rc = block_streams(&A, b, &d);
    int64_t n = d.n[which];
    if (rc == ORC_OK) {
        if ((uint64_t)n > cap) rc = ORC_E_ARG;
        else if (n) memcpy(out, d.s[which], (size_t)n);
    }
    dblk_free(&d);
    return rc ? rc : n;
}

int64_t orc_block_levels(const uint8_t* arc, uint64_t arc_len, uint32_t b, uint8_t* out, uint64_t cap) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    if (b >= A.nb || !(A.flags & 2)) return ORC_E_ARG;
    dblk_t d;
    rc = block_streams(&A, b, &d);
    int64_t n = d.n_tok;
    if (rc == ORC_OK) {
        if ((uint64_t)n > cap) rc = ORC_E_ARG;
        else if (n) memcpy(out, A.a + d.payload_off + d.lvl_off, (size_t)n);
    }
    dblk_free(&d);
    return rc ? rc : n;
}

static int cmp_u64(const void* x, const void* y) {
    uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return a < b ? -1 : a > b;
}

int orc_archive_stats(const uint8_t* arc, uint64_t arc_len, orc_stats* st) {
    arc_t A;
    int rc = arc_open(arc, arc_len, &A);
    if (rc) return rc;
    memset(st, 0, sizeof *st);
    st->n_blocks = A.nb;
    uint64_t cap_runs = 1024, n_runs = 0;
    uint64_t* runs = (uint64_t*)malloc(cap_runs * sizeof(uint64_t));
    uint64_t tcap = 4 * ORC_BLOCK + 16;
    uint8_t* cmd = (uint8_t*)malloc(tcap);
    uint32_t* ll = (uint32_t*)malloc(tcap * 4);
    uint32_t* ml = (uint32_t*)malloc(tcap * 4);
    uint64_t* dst = (uint64_t*)malloc(tcap * 8);
    uint64_t* src = (uint64_t*)malloc(tcap * 8);
    if (!runs || !cmd || !ll || !ml || !dst || !src) rc = ORC_E_NOMEM;
    for (uint32_t b = 0; b < A.nb && rc == ORC_OK; b++) {
        dblk_t d;
        rc = block_streams(&A, b, &d);
        tok_out_t T = {cmd, ll, ml, NULL, dst, src, tcap};
        if (rc == ORC_OK) rc = block_decode(&A, b, &d, NULL, &T);
        if (rc == ORC_OK) {
            for (int s = 0; s < 4; s++) { st->stream_raw[s] += d.n[s]; st->stream_enc[s] += d.enc[s]; }
            for (uint32_t i = 0; i < d.n[ORC_LEN]; i++) {
                if (d.s[ORC_LEN][i] < 0x80) st->n_values++;
                if (d.s[ORC_LEN][i] >= 0x80 && (i == 0 || d.s[ORC_LEN][i - 1] < 0x80)) st->n_multibyte_values++;
            }
            st->n_tokens += d.n_tok;
            if (d.n_tok > st->max_tokens_block) st->max_tokens_block = d.n_tok;
            uint64_t B = (uint64_t)b * ORC_BLOCK, run = 0;
            for (uint32_t i = 0; i < d.n_tok; i++) {
                st->n_literal_bytes += ll[i];
                if (cmd[i] == 5) { st->n_litonly++; run++; continue; }
                st->n_match_bytes += ml[i];
                if (dst[i] - src[i] < ml[i]) st->n_overlap_tokens++;
                if (src[i] < B) st->n_external_tokens++;
                if (cmd[i] == 0) { st->n_new++; run++; }
                else {
                    st->n_rep[cmd[i] - 1]++;
                    st->hist_dependent++;
                    if (n_runs == cap_runs) { cap_runs *= 2; runs = (uint64_t*)realloc(runs, cap_runs * 8); }
                    runs[n_runs++] = run;
                    run = 0;
                }
            }
            if (n_runs == cap_runs) { cap_runs *= 2; runs = (uint64_t*)realloc(runs, cap_runs * 8); }
            runs[n_runs++] = run; /* a block boundary ends a run: the history resets */
        }
        dblk_free(&d);
    }
    if (rc == ORC_OK && n_runs) {
        for (uint64_t i = 0; i < n_runs; i++) st->run_len_sum += runs[i];
        qsort(runs, n_runs, sizeof(uint64_t), cmp_u64);
        st->runs = n_runs;
        st->median_run = runs[n_runs / 2];
    }
    free(runs); free(cmd); free(ll); free(ml); free(dst); free(src);
    return rc;
}
