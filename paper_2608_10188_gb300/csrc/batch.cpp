// Batched decode (aceapex_batch_*): many archives, one set of launches.
//
// Every archive of a batch gets its own partition of the batch's scratch
// (decoded streams, pending counts and bitmaps, pieces) and its own rANS
// ticket and status word; one job table in device memory lists them, and the
// kernels take (archive, block) work items from shared tickets across all of
// them, so archives of very different sizes and token counts share the GPU
// without a launch per archive (Setup, Table 1: the persistent-queue decoder
// whose time follows the token count).  With ACEAPEX_BATCH_GRAPH the four
// launches are captured once into a CUDA graph and every run replays it.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "host.h"

using namespace acx;

struct aceapex_batch {
    aceapex_ctx* ctx = nullptr;
    int n = 0;
    uint32_t flags = 0;
    uint64_t bytes = 0, blocks = 0;
    JobDev job{};
    LaunchPlan lp;
    DevBuf scratch;             // streams | npend | pmap | spans | lists | job table | counters | status words
    int* d_errs = nullptr;      // [0..3] job status, [4 + a] archive a
    std::vector<int> h_errs;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

inline uint64_t up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

void batch_free(aceapex_batch* B) {
    if (!B) return;
    if (B->ctx) cudaSetDevice(B->ctx->device);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (auto& e : B->ev)
        if (e) cudaEventDestroy(e);
    B->scratch.release();
    delete B;
}

}  // namespace

extern "C" {

int aceapex_batch_create(aceapex_ctx* c, const aceapex_batch_item* items, int n, uint32_t flags,
                         aceapex_batch** out) {
    if (!c || !out || n < 0 || (n > 0 && !items)) return fail(c, ACEAPEX_E_ARG, "batch_create: null argument");
    *out = nullptr;
    if ((uint32_t)n > kMaxArcsPerJob) return fail(c, ACEAPEX_E_ARG, "batch_create: too many archives");
    cudaSetDevice(c->device);
    aceapex_batch* B = new (std::nothrow) aceapex_batch();
    if (!B) return fail(c, ACEAPEX_E_NOMEM, "batch_create: host allocation");
    B->ctx = c;
    B->n = n;
    B->flags = flags;

    // scratch layout: one partition per archive in each region
    std::vector<ArcJob> tab(std::max(n, 1));
    std::vector<uint64_t> o_str(n), o_np(n), o_pm(n), o_sp(n);
    uint64_t s_str = 0, s_np = 0, s_pm = 0, s_sp = 0, slots = 0, items_total = 0;
    uint32_t max_tok = 0, max_lenb = 0;
    for (int a = 0; a < n; a++) {
        const aceapex_archive* A = items[a].arc;
        if (!A || (!items[a].d_out && A->plan.total)) {
            batch_free(B);
            return fail(c, ACEAPEX_E_ARG, "batch_create: item " + std::to_string(a) + " has a null archive or output");
        }
        if (A->ctx && A->ctx->device != c->device) {
            batch_free(B);
            return fail(c, ACEAPEX_E_ARG, "batch_create: item " + std::to_string(a) + " was opened on another device");
        }
        if (items[a].out_cap < A->plan.total) {
            batch_free(B);
            return fail(c, ACEAPEX_E_ARG, "batch_create: item " + std::to_string(a) + " output buffer too small");
        }
        const Plan& P = A->plan;
        o_str[a] = s_str;
        s_str += up(P.scratch_bytes, 256);
        o_np[a] = s_np;
        s_np += up((uint64_t)P.n_blocks * 4, 256);
        o_pm[a] = s_pm;
        s_pm += (uint64_t)P.n_blocks * (kBlock / 8);
        o_sp[a] = s_sp;
        s_sp += P.span_slots * sizeof(SpanRec);
        slots += P.span_slots;
        items_total += P.n_blocks;
        max_tok = std::max(max_tok, P.max_tok);
        max_lenb = std::max(max_lenb, P.max_lenb);
        B->bytes += P.total;
    }
    if (items_total >= 0xffffffffull) {
        batch_free(B);
        return fail(c, ACEAPEX_E_ARG, "batch_create: too many blocks in one batch");
    }
    B->blocks = items_total;
    int rc = launch_plan(c, c->params, max_tok, max_lenb, &B->lp);
    if (rc) {
        batch_free(B);
        return rc;
    }
    slots = std::max<uint64_t>(slots, 1);
    const uint64_t r_str = 0;
    const uint64_t r_np = up(r_str + s_str, 256);
    const uint64_t r_pm = up(r_np + s_np, 256);
    const uint64_t r_sp = up(r_pm + s_pm, 256);
    const uint64_t r_ls = up(r_sp + s_sp, 256);
    const uint64_t r_tab = up(r_ls + 2 * slots * sizeof(JobDev::ListEnt), 256);
    const uint64_t r_cnt = up(r_tab + tab.size() * sizeof(ArcJob), 256);
    const uint64_t r_err = up(r_cnt + kCounterWords * sizeof(uint32_t), 256);
    const uint64_t total = r_err + (4 + (uint64_t)n) * sizeof(int);
    cudaError_t e = B->scratch.ensure(total);
    if (e != cudaSuccess) {
        batch_free(B);
        return e == cudaErrorMemoryAllocation ? fail(c, ACEAPEX_E_NOMEM, "batch_create: device scratch")
                                              : cuda_fail(c, e, "batch_create: device scratch");
    }
    uint8_t* base = (uint8_t*)B->scratch.p;
    uint32_t item_base = 0;
    for (int a = 0; a < n; a++) {
        const aceapex_archive* A = items[a].arc;
        const Plan& P = A->plan;
        ArcJob& J = tab[a];
        memset(&J, 0, sizeof J);
        J.arc = (const uint8_t*)A->d_arc;
        J.blk = A->d_blk;
        J.dtab = A->d_dtab;
        J.scratch = base + r_str + o_str[a];
        J.out = (uint8_t*)items[a].d_out;
        J.npend = (uint32_t*)(base + r_np + o_np[a]);
        J.pmap = (uint32_t*)(base + r_pm + o_pm[a]);
        J.spans = (SpanRec*)(base + r_sp + o_sp[a]);
        J.total = P.total;
        J.n_blocks = P.n_blocks;
        J.lo = 0;
        J.hi = P.n_blocks;
        J.min_match = P.min_match;
        J.item_base = item_base;
        J.deps = A->d_deps;
        J.order = A->d_order;
        item_base += P.n_blocks;
    }
    JobDev& job = B->job;
    job.arcs = (const ArcJob*)(base + r_tab);
    job.n_arcs = (uint32_t)n;
    job.n_items = item_base;
    job.counters = (uint32_t*)(base + r_cnt);
    B->d_errs = (int*)(base + r_err);
    job.err = B->d_errs;
    job.arc_err = B->d_errs + 4;
    job.timeout_ns = (uint64_t)c->params.timeout_us * 1000ull;
    job.max_tok = max_tok;
    job.max_lenb = max_lenb;
    job.lists[0] = (JobDev::ListEnt*)(base + r_ls);
    job.lists[1] = job.lists[0] + slots;
    B->h_errs.assign(4 + n, 0);
    if (n > 0) e = cudaMemcpy(base + r_tab, tab.data(), n * sizeof(ArcJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(base + r_cnt, 0, r_err - r_cnt + (4 + (uint64_t)n) * sizeof(int));
    for (auto& ev : B->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        batch_free(B);
        return cuda_fail(c, e, "batch_create");
    }
    if ((flags & ACEAPEX_BATCH_GRAPH) && job.n_items > 0) {
        // capture the four launches once; runs replay the graph
        e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            batch_free(B);
            return cuda_fail(c, e, "batch_create: stream capture");
        }
        rc = enqueue_job(c, job, B->lp, 3 + (uint32_t)n, B->d_errs, 4 + (uint32_t)n, B->cap, nullptr);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(B->cap, &g);
        B->graph = g;
        if (rc || e != cudaSuccess) {
            batch_free(B);
            return rc ? rc : cuda_fail(c, e, "batch_create: end of capture");
        }
        if ((e = cudaGraphInstantiate(&B->exec, B->graph, 0)) != cudaSuccess) {
            batch_free(B);
            return cuda_fail(c, e, "batch_create: graph instantiation");
        }
    }
    *out = B;
    return ACEAPEX_OK;
}

int aceapex_batch_destroy(aceapex_batch* B) {
    if (!B) return ACEAPEX_E_ARG;
    batch_free(B);
    return ACEAPEX_OK;
}

int aceapex_batch_run_async(aceapex_batch* B, void* stream) {
    if (!B) return ACEAPEX_E_ARG;
    aceapex_ctx* c = B->ctx;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaEventRecord(B->ev[0], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    if (B->job.n_items > 0) {
        if (B->exec) {
            if ((e = cudaGraphLaunch(B->exec, st)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
        } else {
            const int rc = enqueue_job(c, B->job, B->lp, 3 + (uint32_t)B->n, B->d_errs, 4 + (uint32_t)B->n, st, B->ev);
            if (rc) return rc;
        }
    }
    if ((e = cudaEventRecord(B->ev[3], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    return ACEAPEX_OK;
}

int aceapex_batch_wait(aceapex_batch* B, void* stream, aceapex_batch_item* items, aceapex_stats* stats) {
    if (!B) return ACEAPEX_E_ARG;
    aceapex_ctx* c = B->ctx;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if ((e = cudaMemcpy(B->h_errs.data(), B->d_errs, B->h_errs.size() * sizeof(int), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
        return cuda_fail(c, e, "status words");
    const int job_rc = B->h_errs[0];
    bool attributed = false;
    for (int a = 0; a < B->n; a++) attributed |= B->h_errs[4 + a] != 0;
    if (items)
        for (int a = 0; a < B->n; a++)
            // an error that no archive claims (a grid-wide wait) applies to all
            items[a].status = B->h_errs[4 + a] ? B->h_errs[4 + a] : (attributed ? ACEAPEX_OK : job_rc);
    if (stats) {
        memset(stats, 0, sizeof *stats);
        float t = 0;
        cudaEventElapsedTime(&t, B->ev[0], B->ev[3]);
        stats->ms_total = t;
        if (!B->exec && B->job.n_items > 0) {
            float a = 0, b = 0, x = 0;
            cudaEventElapsedTime(&a, B->ev[0], B->ev[1]);
            cudaEventElapsedTime(&b, B->ev[1], B->ev[2]);
            cudaEventElapsedTime(&x, B->ev[2], B->ev[3]);
            stats->ms_ans = a;
            stats->ms_parse = b;
            stats->ms_copy = x;
        }
        stats->blocks = B->blocks;
        stats->bytes = B->bytes;
        uint32_t st2[6] = {0, 0, 0, 0, 0, 0};
        cudaMemcpy(st2, B->job.counters + kStatPendBytes, sizeof st2, cudaMemcpyDeviceToHost);
        stats->pending_bytes = (uint64_t)st2[0] | ((uint64_t)st2[1] << 32);
        stats->pending_spans = st2[kStatPending - kStatPendBytes];
        stats->wait_polls = st2[kStatPolls - kStatPendBytes];
    }
    if (job_rc) return fail(c, job_rc, "batch: " + device_error_text(B->h_errs.data()));
    return ACEAPEX_OK;
}

int aceapex_batch_run(aceapex_batch* B, void* stream, aceapex_batch_item* items, aceapex_stats* stats) {
    const int rc = aceapex_batch_run_async(B, stream);
    if (rc) return rc;
    return aceapex_batch_wait(B, stream, items, stats);
}

int aceapex_batch_decode(aceapex_ctx* c, aceapex_batch_item* items, int n, void* stream, aceapex_stats* stats) {
    aceapex_batch* B = nullptr;
    int rc = aceapex_batch_create(c, items, n, 0, &B);
    if (rc) return rc;
    rc = aceapex_batch_run(B, stream, items, stats);
    aceapex_batch_destroy(B);
    return rc;
}

}  // extern "C"

// ---- autotuner ----------------------------------------------------------------------------
// Times one batch under every point of the decoder's launch space — CTAs per
// SM of the local pass and of the entropy stage, blocks per queue ticket —
// with the L2 flushed before each run, and keeps the fastest.
extern "C" int aceapex_autotune(aceapex_ctx* c, const aceapex_batch_item* items, int n, int reps,
                                aceapex_tune_point* points, int max_points, int* n_points, aceapex_dec_params* best) {
    if (!c || n <= 0 || !items || max_points < 0 || (max_points && !points))
        return fail(c, ACEAPEX_E_ARG, "autotune: bad argument");
    if (reps <= 0) reps = 3;
    cudaSetDevice(c->device);
    const aceapex_dec_params base = c->params;
    aceapex_batch* B = nullptr;
    int rc = aceapex_batch_create(c, items, n, 0, &B);
    if (rc) return rc;
    void* flush = nullptr;
    const size_t flush_bytes = 256u << 20;  // larger than L2
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&flush, flush_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        aceapex_batch_destroy(B);
        if (flush) cudaFree(flush);
        return cuda_fail(c, e, "autotune");
    }
    const size_t lsm = local_smem_bytes(B->job.max_tok, B->job.max_lenb);
    const int occ_local = base.variant == ACEAPEX_VARIANT_PLAIN ? 1 : std::max(1, local_occupancy(lsm));
    std::vector<uint32_t> locals, ranss;
    for (int v : {1, 2, 3, 4, 6, 8, 12, 16})
        if (v <= occ_local) locals.push_back((uint32_t)v);
    for (int v = 1; v <= c->occ_rans; v++) ranss.push_back((uint32_t)v);
    const uint32_t chunks[] = {1, 4, 16};
    double best_ms = 1e30;
    aceapex_dec_params best_p = base;
    int np = 0;
    std::vector<float> t;
    for (uint32_t lc : locals)
        for (uint32_t rcn : ranss)
            for (uint32_t ch : chunks) {
                aceapex_dec_params p = base;
                p.ctas_per_sm = lc;
                p.rans_ctas_per_sm = rcn;
                p.queue_chunk = ch;
                LaunchPlan lp;
                if ((rc = launch_plan(c, p, B->job.max_tok, B->job.max_lenb, &lp))) break;
                B->lp = lp;
                t.clear();
                for (int r = 0; r <= reps && rc == ACEAPEX_OK; r++) {
                    cudaMemsetAsync(flush, r & 0xff, flush_bytes, st);
                    if ((rc = aceapex_batch_run_async(B, st))) break;
                    aceapex_stats s;
                    if ((rc = aceapex_batch_wait(B, st, nullptr, &s))) break;
                    if (r) t.push_back((float)s.ms_total);  // the first run warms up
                }
                if (rc) break;
                std::sort(t.begin(), t.end());
                const double ms = t[t.size() / 2];
                if (np < max_points) {
                    points[np].ctas_per_sm = lc;
                    points[np].rans_ctas_per_sm = rcn;
                    points[np].queue_chunk = ch;
                    points[np].ms = ms;
                }
                np++;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_p = p;
                }
            }
    cudaStreamDestroy(st);
    cudaFree(flush);
    aceapex_batch_destroy(B);
    if (n_points) *n_points = std::min(np, max_points);
    if (rc) return rc;
    c->params = best_p;
    if (best) *best = best_p;
    return ACEAPEX_OK;
}
