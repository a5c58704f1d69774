"""Hand-worked examples that pin the oracle to the format definition.

Nothing here was produced by running the oracle or the GPU library: every
expected value is derived by hand below, from the definitions it cites.

FNV-1a 64 vectors: published with the FNV specification (Fowler, Noll, Vo;
IETF draft-eastlake-fnv), offset basis 0xcbf29ce484222325, prime
0x100000001b3.

rANS examples: textbook interleaved rANS as fixed for format v1 (32-bit state
x, L = 2^16, 12-bit probabilities M = 4096, 16-bit renormalisation words,
symbol i on lane i mod K, words consumed in (step, lane) order).  The paper
names only "ANS" as the entropy stage (Table 1, "ANS + one match kernel";
Table 2, "ANS+parse"); these parameters are format v1's reading.

Encoder step for symbol s with frequency f and cumulative c:
    if x >= f * 2^20: emit x & 0xffff; x >>= 16
    x = (x // f) * 4096 + x % f + c
Decoder step:
    slot = x & 4095; s = symbol whose [c, c+f) holds slot
    x = f * (x >> 12) + slot - c; if x < 2^16: x = (x << 16) | next word
"""

FNV1A64_VECTORS = [
    (b"", 0xCBF29CE484222325),
    (b"a", 0xAF63DC4C8601EC8C),
    (b"foobar", 0x85944171F73967E8),
]

# splitmix64 reference outputs for seed 1234567 (published alongside the
# generator's definition; used to pin the seeded input generators).
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423]

RANS_WORKED = [
    {
        # f(A)=3072 c=0, f(B)=1024 c=3072; K=1; symbols "AB" (encoded B first).
        # i=1 'B': x=65536 < 1024*2^20, x = 64*4096 + 0 + 3072 = 265216
        # i=0 'A': x < 3072*2^20,       x = 86*4096 + 1024 + 0 = 353280
        # final state 353280 = 0x00056400, no words; body = state + 12 pad bytes
        "name": "two-symbol, no renormalisation",
        "freq": {0x41: 3072, 0x42: 1024},
        "K": 1,
        "symbols": b"AB",
        "body_hex": "00640500" + "00" * 12,
    },
    {
        # f(A)=4095 c=0, f(B)=1 c=4095; K=1; symbols "BB".
        # i=1: x = 65536*4096 + 4095 = 268439551 (= 2^28 + 4095), no emit
        # i=0: x >= 1*2^20 -> emit x & 0xffff = 4095; x = 4096;
        #      x = 4096*4096 + 0 + 4095 = 16781311 = 0x01000FFF
        # words in decode order: [4095]; enc_len = 16 + 2 = 18
        "name": "renormalisation word",
        "freq": {0x41: 4095, 0x42: 1},
        "K": 1,
        "symbols": b"BB",
        "body_hex": "ff0f0001" + "00" * 12 + "ff0f",
    },
    {
        # Same table as the first example, K=2: lane 0 gets 'A', lane 1 'B'.
        # lane 1: x1 = 64*4096 + 0 + 3072 = 265216 = 0x00040C00
        # lane 0: x0 = 21*4096 + 1024 + 0 = 87040 = 0x00015400
        "name": "two lanes",
        "freq": {0x41: 3072, 0x42: 1024},
        "K": 2,
        "symbols": b"AB",
        "body_hex": "00540100" + "000c0400" + "00" * 8,
    },
    {
        # f(A)=4094 c=0, f(B)=1 c=4094, f(C)=1 c=4095; K=2; symbols "BCBC"
        # (lanes 0,1,0,1).  Encoding runs i=3..0:
        # i=3 lane1 'C': x1 = 65536*4096 + 4095 = 268439551
        # i=2 lane0 'B': x0 = 65536*4096 + 4094 = 268439550
        # i=1 lane1 'C': emit 4095, x1 = 4096 -> 4096*4096 + 4095 = 16781311
        # i=0 lane0 'B': emit 4094, x0 = 4096 -> 4096*4096 + 4094 = 16781310
        # emitted [4095, 4094] -> decode order [4094, 4095]: step 0 lane 0
        # takes the first word, lane 1 the second.
        "name": "word order is (step, lane)",
        "freq": {0x41: 4094, 0x42: 1, 0x43: 1},
        "K": 2,
        "symbols": b"BCBC",
        "body_hex": "fe0f0001" + "ff0f0001" + "00" * 8 + "fe0f" + "ff0f",
    },
]

# Hand-built archives (all streams stored).  Each token: cmd (0 NEW,
# 1..4 REP0..REP3, 5 LIT_ONLY), literal bytes, match length ML, and for NEW
# the absolute source position.  Paper, Setup: back-references are absolute
# positions in the decompressed output; "What Does: Periods, Not Chains":
# an overlapping match is the periodic fill out[dst+k] = out[src + k mod d].
ARCHIVE_WORKED = [
    {
        "name": "periodic overlap and repeat distance, one block",
        # t0 NEW: literals ACGT at 0..3; match dst=4, src=0, d=4, ML=10:
        #     out[4..13] = out[0 + k mod 4] = ACGTACGTAC
        # history after t0: [4, 1, 2, 3]
        # t1 REP0 (d=4): literals NN at 14..15; dst=16, src=12, ML=5:
        #     source bytes out[12..15] = A C N N, periodic -> ACNNA
        # t2 LIT_ONLY: TTT
        "blocks": [[
            {"cmd": 0, "lits": b"ACGT", "ml": 10, "src": 0},
            {"cmd": 1, "lits": b"NN", "ml": 5},
            {"cmd": 5, "lits": b"TTT", "ml": 0},
        ]],
        "expected": b"ACGTACGTACGTAC" + b"NN" + b"ACNNA" + b"TTT",
    },
    {
        "name": "cross-block absolute offsets, history move-to-front, 3-byte varint",
        # block 0: one LIT_ONLY token of 16384 literals, byte i = i mod 256
        #   (LL = 16384 needs the 3-byte varint 80 80 01)
        # block 1 (100 bytes), B = 16384:
        #  t0 NEW LL=0 ML=10 src=300: out[16384..16393] = (300..309) mod 256
        #       = 44..53; history [16084, 1, 2, 3]
        #  t1 NEW LL=1 (0xAA) ML=4 src=16380: dst=16395, bytes 252..255;
        #       d = 15, history [15, 16084, 1, 2]
        #  t2 REP1 (d=16084) LL=0 ML=6: dst=16399, src=315 -> 59..64;
        #       history [16084, 15, 1, 2]
        #  t3 REP2 (d=1) LL=2 (0x10 0x20) ML=8: dst=16407, src=16406 ->
        #       eight copies of 0x20; history [1, 16084, 15, 2]
        #  t4 REP1 (d=16084) LL=0 ML=4: dst=16415, src=331 -> 75..78;
        #       history [16084, 1, 15, 2]
        #  t5 LIT_ONLY: 65 bytes 'a' (16419 + 65 = 16484 = B + 100)
        # off stream of block 1: two NEW offsets 300 = 0x12C and 16380 = 0x3FFC
        #   as 5 planes: 2C FC | 01 3F | 00 00 | 00 00 | 00 00
        "blocks": [
            [{"cmd": 5, "lits": bytes(range(256)) * 64, "ml": 0}],
            [
                {"cmd": 0, "lits": b"", "ml": 10, "src": 300},
                {"cmd": 0, "lits": b"\xaa", "ml": 4, "src": 16380},
                {"cmd": 2, "lits": b"", "ml": 6},
                {"cmd": 3, "lits": b"\x10\x20", "ml": 8},
                {"cmd": 2, "lits": b"", "ml": 4},
                {"cmd": 5, "lits": b"a" * 65, "ml": 0},
            ],
        ],
        "expected": bytes(range(256)) * 64
        + bytes(range(44, 54)) + b"\xaa" + bytes([252, 253, 254, 255]) + bytes(range(59, 65))
        + b"\x10\x20" + b"\x20" * 8 + bytes(range(75, 79)) + b"a" * 65,
        "off_stream_block1_hex": "2cfc013f000000000000",
        "len_stream_block0_hex": "80800100",
    },
]
