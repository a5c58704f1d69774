// Host-side code under AddressSanitizer and UndefinedBehaviorSanitizer (test
// infrastructure, built and run by tests/test_sanitize_cpu.py).
//
// The library's host code parses untrusted archives: the plan builder behind
// aceapex_archive_open / aceapex_archive_check, the byte-level closure walk
// of range decodes and serving, the parse statistics; the encoder writes
// them.  The CPU oracle parses them too.  This driver runs all of them on
// archives from both encoders (several option sets, several corpora and
// sizes) and on truncations and bit flips of every archive, and exits 0 only
// when every valid archive round-trips.  A sanitizer report aborts it.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/aceapex.h"
#include "../../oracle/oracle.h"
#include "plan.h"

extern "C" int synth_dna(uint8_t* out, uint64_t n, uint64_t seed, double n_frac, double copy_frac, double tandem_frac,
                         void* st);
extern "C" int synth_text(uint8_t* out, uint64_t n, uint64_t seed, uint32_t n_vocab, double zipf_s, double p_repeat,
                          void* st);
extern "C" int acx_debug_parse_stats(const uint32_t* recs, const uint32_t* n_tok, uint32_t n_blocks,
                                     aceapex_parse_stats* out);
extern "C" int acx_debug_closure(const uint8_t* h_arc, uint64_t arc_len, const uint64_t* first, uint64_t n_match,
                                 const uint16_t* o, const uint16_t* ml, const uint64_t* src, uint64_t start,
                                 uint64_t len, uint32_t* blocks, uint32_t* iv_count, uint32_t* ivs,
                                 uint32_t cap_blocks, uint32_t cap_ivs, uint32_t* n_blocks);

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() {  // xorshift64*
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545F4914F6CDD1Dull;
}

static int failures = 0;
#define CHECK(c, ...)                          \
    do {                                       \
        if (!(c)) {                            \
            fprintf(stderr, "FAIL: " __VA_ARGS__); \
            fprintf(stderr, "\n");             \
            failures++;                        \
        }                                      \
    } while (0)

// The parse of every block by the oracle, as a match index and as the token
// records the device's parse-only pass writes.
struct Parse {
    std::vector<uint64_t> first;
    std::vector<uint16_t> o, ml;
    std::vector<uint64_t> src;
    std::vector<uint32_t> recs, n_tok;
};

static bool oracle_parse(const std::vector<uint8_t>& a, uint32_t nb, Parse* P) {
    const uint64_t cap = 4 * ORC_BLOCK + 16;
    std::vector<uint8_t> cmd(cap);
    std::vector<uint32_t> ll(cap), ml(cap), lit(cap);
    std::vector<uint64_t> dst(cap), src(cap);
    P->first.assign(1, 0);
    for (uint32_t b = 0; b < nb; b++) {
        const int64_t n = orc_parse_block(a.data(), a.size(), b, cap, cmd.data(), ll.data(), ml.data(), dst.data(),
                                          src.data(), lit.data());
        if (n < 0) return false;
        P->n_tok.push_back((uint32_t)n);
        const uint64_t B = (uint64_t)b * ORC_BLOCK;
        for (int64_t t = 0; t < n; t++) {
            // token record: source (x, y), destination offset | length << 16, command
            P->recs.push_back((uint32_t)src[t]);
            P->recs.push_back((uint32_t)(src[t] >> 32));
            P->recs.push_back((uint32_t)(dst[t] - B) | (ml[t] << 16));
            P->recs.push_back(cmd[t]);
            if (ml[t]) {
                P->o.push_back((uint16_t)(dst[t] - B));
                P->ml.push_back((uint16_t)ml[t]);
                P->src.push_back(src[t]);
            }
        }
        P->first.push_back(P->o.size());
    }
    return true;
}

static void check_valid(const std::vector<uint8_t>& a, const std::vector<uint8_t>& data, const char* tag) {
    acx::Plan plan;
    std::string why;
    CHECK(acx::build_plan(a.data(), a.size(), &plan, &why) == 0, "%s: plan: %s", tag, why.c_str());
    aceapex_archive_info info;
    CHECK(aceapex_archive_check(a.data(), a.size(), &info) == ACEAPEX_OK && info.total_size == data.size(),
          "%s: archive_check", tag);
    std::vector<uint8_t> out(data.size() + 1);
    CHECK(orc_decode(a.data(), a.size(), out.data(), data.size(), 1) == ORC_OK &&
              (data.empty() || memcmp(out.data(), data.data(), data.size()) == 0),
          "%s: oracle round trip", tag);
    const uint32_t nb = plan.n_blocks;
    Parse P;
    CHECK(oracle_parse(a, nb, &P), "%s: oracle parse", tag);
    aceapex_parse_stats st;
    if (nb)
        CHECK(acx_debug_parse_stats(P.recs.data(), P.n_tok.data(), nb, &st) == 0 && st.blocks == nb,
              "%s: parse stats", tag);
    // byte-level closures of random regions
    std::vector<uint32_t> blocks(nb + 1), ivc(nb + 1), ivs(64 * (nb + 1));
    for (int k = 0; k < 24 && data.size(); k++) {
        const uint64_t len = 1 + rnd() % std::min<uint64_t>(data.size(), 70000);
        const uint64_t start = rnd() % (data.size() - len + 1);
        uint32_t n = 0;
        const int rc = acx_debug_closure(a.data(), a.size(), P.first.data(), P.o.size(), P.o.data(), P.ml.data(),
                                         P.src.data(), start, len, blocks.data(), ivc.data(), ivs.data(),
                                         (uint32_t)blocks.size(), (uint32_t)ivs.size(), &n);
        CHECK(rc == 0 || rc == -1, "%s: closure rc %d", tag, rc);
        if (rc == 0) CHECK(n >= 1 && blocks[n - 1] == (start + len - 1) / ORC_BLOCK, "%s: closure ends", tag);
    }
}

// Truncations and bit flips: the plan builder, the archive check and the
// oracle must return a status (valid or corrupt) without touching memory
// outside the archive.
static void check_corruptions(const std::vector<uint8_t>& a, uint64_t total, int reps) {
    std::vector<uint8_t> out(total + 1);
    for (int k = 0; k < reps; k++) {
        std::vector<uint8_t> b;
        if (k & 1) {
            b.assign(a.begin(), a.begin() + rnd() % a.size());  // truncated
        } else {
            b = a;
            const int flips = 1 + (int)(rnd() % 4);
            for (int f = 0; f < flips; f++) b[rnd() % b.size()] ^= (uint8_t)(1u << (rnd() % 8));
        }
        acx::Plan plan;
        std::string why;
        const int rc = acx::build_plan(b.data(), b.size(), &plan, &why);
        CHECK(rc == 0 || rc == -2, "plan status %d", rc);
        aceapex_archive_info info;
        const int rc2 = aceapex_archive_check(b.data(), b.size(), &info);
        CHECK((rc2 == ACEAPEX_OK) == (rc == 0), "archive_check disagrees with the plan");
        uint64_t t = 0;
        uint32_t nb = 0, flags = 0, mm = 0;
        if (orc_info(b.data(), b.size(), &t, &nb, &flags, &mm) == ORC_OK && t <= total)
            (void)orc_decode(b.data(), b.size(), out.data(), t, 1);
    }
}

int main(int argc, char** argv) {
    const int reps = argc > 1 ? atoi(argv[1]) : 60;
    struct Corpus {
        const char* name;
        std::vector<uint8_t> data;
    };
    std::vector<Corpus> corpora;
    const uint64_t sizes[] = {0, 1, 17, 16384, 16385, 150000, 600000};
    for (uint64_t n : sizes) {
        Corpus c{"dna", std::vector<uint8_t>(n)};
        synth_dna(c.data.data(), n, 7 + n, 0.005, 0.24, 0.06, nullptr);
        corpora.push_back(c);
    }
    {
        Corpus c{"text", std::vector<uint8_t>(400000)};
        synth_text(c.data.data(), c.data.size(), 9, 50000, 1.1, 0.05, nullptr);
        corpora.push_back(c);
        Corpus r{"random", std::vector<uint8_t>(70000)};
        for (auto& x : r.data) x = (uint8_t)rnd();
        corpora.push_back(r);
    }
    int archives = 0;
    for (const Corpus& c : corpora) {
        const uint64_t n = c.data.size();
        // library encoder under several option sets
        for (int v = 0; v < 6; v++) {
            aceapex_enc_params p;
            memset(&p, 0, sizeof p);
            p.no_rep = v & 1;
            p.max_lanes = v == 2 ? 128 : v == 3 ? 1 : 32;
            p.levels = v >= 2;
            p.deps = v == 4;
            p.segment = v == 5 ? 65536 : 0;
            p.max_depth = v == 3 ? 1 : 0;
            p.threads = 2;
            uint8_t* out = nullptr;
            uint64_t len = 0;
            aceapex_enc_stats es;
            const int rc = aceapex_encode_ex(n ? c.data.data() : nullptr, n, &p, &out, &len, &es);
            CHECK(rc == ACEAPEX_OK, "%s %llu: encode option set %d", c.name, (unsigned long long)n, v);
            if (rc != ACEAPEX_OK) continue;
            std::vector<uint8_t> a(out, out + len);
            aceapex_free(out);
            char tag[64];
            snprintf(tag, sizeof tag, "%s %llu lib/%d", c.name, (unsigned long long)n, v);
            check_valid(a, c.data, tag);
            check_corruptions(a, n, reps);
            archives++;
        }
        // the oracle's own encoder
        for (int v = 0; v < 2; v++) {
            orc_enc_params p;
            orc_enc_defaults(&p);
            p.no_rep = v;
            uint8_t* out = nullptr;
            uint64_t len = 0;
            const int rc = orc_encode(n ? c.data.data() : nullptr, n, &p, &out, &len);
            CHECK(rc == ORC_OK, "%s %llu: oracle encode %d", c.name, (unsigned long long)n, v);
            if (rc != ORC_OK) continue;
            std::vector<uint8_t> a(out, out + len);
            orc_free(out);
            char tag[64];
            snprintf(tag, sizeof tag, "%s %llu oracle/%d", c.name, (unsigned long long)n, v);
            check_valid(a, c.data, tag);
            check_corruptions(a, n, reps);
            archives++;
        }
    }
    printf("sanitized host checks: %d archives, %d failures\n", archives, failures);
    return failures ? 1 : 0;
}
