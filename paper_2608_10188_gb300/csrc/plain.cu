// Plain comparison decoder for the parse and match layer: one thread per
// block parses sequentially (varints one byte at a time, the 4-entry distance
// history applied token by token) and copies every match byte by byte in
// token order, as a straightforward port of the byte-serial reference decode
// would.  It produces the same intermediate as k_local (the block with its
// cross-block bytes left pending, the pending spans and bitmap), so the same
// cross-block pass finishes it and the two variants differ only in the
// paper's two levers: scan parse and periodic fill.
#include "common.cuh"
#include "launch.h"

namespace acx {

constexpr int kPlainThreads = 32;

__global__ void __launch_bounds__(kPlainThreads) k_plain(JobDev job) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* sout = sm;
    uint32_t* pend = reinterpret_cast<uint32_t*>(sm + kBlock);
    volatile uint32_t* misc = reinterpret_cast<volatile uint32_t*>(sm + kBlock + kBlock / 8);
    const int lane = threadIdx.x;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&job.counters[1], 1u);
        item = __shfl_sync(ACX_FULL, item, 0);
        if (item >= job.n_items) return;
        const int a = find_arc(job, item);
        const ArcJob J = load_arc(job, a);
        const ItemRef ir = item_ref(J, item - J.item_base);
        const uint32_t b = ir.blk;
        const BlockDev& bd = J.blk[b];
        const uint64_t B = (uint64_t)b * kBlock;
        for (uint32_t i = lane; i < kBlock / 32; i += 32) pend[i] = 0;
        __syncwarp();
        if (lane == 0) {
            const uint8_t* scr = J.scratch + ir.scratch;
            const uint8_t* cmd = scr + bd.s_off[kCmd];
            const uint8_t* lb = scr + bd.s_off[kLen];
            const uint8_t* off = scr + bd.s_off[kOff];
            const uint8_t* lit = scr + bd.s_off[kLit];
            const uint32_t n = bd.n_tok, LB = bd.s_raw[kLen], n_lit = bd.s_raw[kLit], n_new = bd.n_new;
            uint64_t hist[4] = {1, 2, 3, 4};
            const uint64_t E = B + bd.raw_len;
            uint64_t pos = B;
            uint32_t lp = 0, ni = 0, vp = 0, np = 0, pb = 0;
            bool bad = false;
            for (uint32_t i = 0; i < n && !bad; i++) {
                uint32_t v[2] = {0, 0};
                for (int qv = 0; qv < 2 && !bad; qv++) {
                    uint32_t val = 0;
                    int k = 0;
                    for (;;) {
                        if (vp >= LB || k == 3) { bad = true; break; }
                        const uint8_t c = lb[vp++];
                        val |= (uint32_t)(c & 0x7f) << (7 * k);
                        k++;
                        if (c < 0x80) break;
                    }
                    v[qv] = val;
                }
                if (bad) break;
                const uint32_t LL = v[0], ML = v[1];
                const uint8_t k = cmd[i];
                if (LL > E - pos || LL > n_lit - lp) { bad = true; break; }
                for (uint32_t j = 0; j < LL; j++) sout[pos - B + j] = lit[lp + j];
                pos += LL;
                lp += LL;
                uint64_t src = 0;
                if (k == kLitOnly) {
                    if (ML != 0 || i != n - 1 || LL == 0) bad = true;
                    continue;
                } else if (k == kNew) {
                    if (ni >= n_new) { bad = true; break; }
                    for (int p = 0; p < 5; p++) src |= (uint64_t)off[(uint64_t)p * n_new + ni] << (8 * p);
                    ni++;
                    if (src >= pos) { bad = true; break; }
                    hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = pos - src;
                } else if (k <= 4) {
                    const int j = k - 1;
                    const uint64_t d = hist[j];
                    if (d < 1 || d > pos) { bad = true; break; }
                    src = pos - d;
                    for (int q = j; q > 0; q--) hist[q] = hist[q - 1];
                    hist[0] = d;
                } else {
                    bad = true;
                    break;
                }
                if (ML < J.min_match || ML > E - pos) { bad = true; break; }
                if (J.deps && src < B) {  // blocks read outside this block must be listed
                    const uint64_t d = pos - src, e = src + (d < ML ? d : ML);
                    for (uint64_t a = src >> 14; a <= (e - 1) >> 14 && a < b && !bad; a++)
                        bad = !listed(J.deps + bd.dep_off, bd.n_deps, (uint32_t)a);
                    if (bad) break;
                }
                const uint32_t o = (uint32_t)(pos - B);
                // in-block source whose bytes are all final: copy byte by byte now
                bool local = src >= B;
                if (local) {
                    const uint64_t d = pos - src;
                    const uint32_t s0 = (uint32_t)(src - B), se = s0 + (uint32_t)(d < ML ? d : ML);
                    for (uint32_t w = s0 >> 5; w <= ((se - 1) >> 5) && local; w++)
                        if (pend[w] & range_mask(w, s0, se)) local = false;
                }
                if (local) {
                    for (uint32_t j = 0; j < ML; j++) sout[o + j] = sout[src - B + j];
                } else {
                    for (uint32_t w = o >> 5; w <= ((o + ML - 1) >> 5); w++) pend[w] |= range_mask(w, o, o + ML);
                    np += emit_pieces(J.spans + ir.span_base + np, o, src, ML, pos - src);
                    pb += ML;
                }
                pos += ML;
            }
            if (!bad && (pos != E || lp != n_lit || ni != n_new || vp != LB)) bad = true;
            if (bad) {
                set_err_arc(job, a, kErrCorrupt, kStagePlain << 24, b);
                np = 0;
                pb = 0;
            }
            misc[0] = np;
            misc[1] = pb;
        }
        __syncwarp();
        const uint32_t np = misc[0], pbytes = misc[1];
        uint8_t* gout = J.out + (uint64_t)ir.slot * kBlock;
        const uint32_t R = bd.raw_len, nv = R / 16;
        for (uint32_t i = lane; i < nv; i += 32) reinterpret_cast<uint4*>(gout)[i] = reinterpret_cast<uint4*>(sout)[i];
        for (uint32_t x = 16 * nv + lane; x < R; x += 32) gout[x] = sout[x];
        {
            // written for every block; all clear when nothing is pending (also for a
            // corrupt block, so other blocks never wait on its bytes)
            uint32_t* gp = J.pmap + (uint64_t)ir.slot * (kBlock / 32);
            for (uint32_t i = lane; i < kBlock / 32; i += 32) gp[i] = np ? pend[i] : 0u;
        }
        if (lane == 0) {
            J.npend[ir.slot] = np;
            if (np) {
                atomicAdd(&job.counters[kStatPending], np);
                atomicAdd(reinterpret_cast<unsigned long long*>(job.counters + kStatPendBytes), (unsigned long long)pbytes);
            }
        }
        __syncwarp();
    }
}

size_t plain_smem_bytes() { return kBlock + kBlock / 8 + 64; }

cudaError_t launch_plain(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = plain_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_plain<<<grid, kPlainThreads, sm, st>>>(job);
    return cudaGetLastError();
}

int plain_occupancy() {
    const size_t sm = plain_smem_bytes();
    cudaFuncSetAttribute(k_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain, kPlainThreads, sm) != cudaSuccess) return 0;
    return n;
}

}  // namespace acx
