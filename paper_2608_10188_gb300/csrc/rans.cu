// Entropy stage of the decode (paper, Table 1/2: "ANS"): the persistent
// k_rans kernel (one warp per block, see rans_dev.cuh) and the launchers.
#include <algorithm>
#include <atomic>

#include "launch.h"
#include "rans_dev.cuh"

namespace acx {

// Start of a decode call: every ticket and statistic restarts at zero.
__global__ void k_prologue(uint32_t* counters, uint32_t n_counters, int* errs, uint32_t n_errs) {
    for (uint32_t i = threadIdx.x; i < n_counters; i += blockDim.x) counters[i] = 0;
    for (uint32_t i = threadIdx.x; i < n_errs; i += blockDim.x) errs[i] = 0;
    if (threadIdx.x < kLvStripes) counters[kLvTickets + threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        counters[kStatPending] = 0;
        counters[kStatPolls] = 0;
        counters[kListCnt] = 0;
        counters[kListCnt + 1] = 0;
        counters[kBarCount] = 0;
        counters[kStatPendBytes] = 0;
        counters[kStatPendBytes + 1] = 0;
    }
}

// Each CTA works on one archive at a time (its tables in shared memory);
// its warps take blocks of that archive from the archive's ticket, and when
// the archive is exhausted the CTA moves to the archive with the most blocks
// left.
__global__ void __launch_bounds__(kRansWarps * 32) k_rans(JobDev job) {
    extern __shared__ __align__(128) uint8_t smraw[];
    RansSmem& S = *reinterpret_cast<RansSmem*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kSlots) mbar_init(&S.bar[warp][lane], 1);
    if (lane == kSlots) mbar_init(&S.sbar[warp], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (threadIdx.x == 0) {
        const uint64_t target = (uint64_t)blockIdx.x * job.n_items / gridDim.x;
        S.next_arc = job.n_arcs > 1 ? find_arc(job, (uint32_t)target) : 0;
        S.arc = -1;
    }
    __syncthreads();
    const uint64_t deadline = gtimer() + kCopyWaitNs;  // the entropy stage waits only for its copies
    uint32_t seq = 0, sphase = 0;
    uint32_t* tickets = job.counters + 3;
    const uint32_t ring_s = ring_addr(S, warp);
    for (;;) {
        const int a = S.next_arc;
        if (a < 0) break;
        const ArcJob J = load_arc(job, a);
        if (S.arc != a) {
            const uint4* src = reinterpret_cast<const uint4*>(J.dtab);
            uint4* dst = reinterpret_cast<uint4*>(&S.tab[0][0]);
            for (int i = threadIdx.x; i < (int)(4 * kM / 4); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) S.arc = a;
        }
        const uint32_t n_a = J.hi - J.lo;
        const uint32_t chunk = job.chunk ? job.chunk : 1u;
        uint32_t cnext = 0, cleft = 0;  // this warp's current run of `chunk` tickets
        for (;;) {
            if (cleft == 0) {
                uint32_t t0 = 0;
                if (lane == 0) t0 = atomicAdd(&tickets[a], chunk);
                cnext = __shfl_sync(ACX_FULL, t0, 0);
                cleft = chunk;
            }
            const uint32_t tk = cnext++;
            cleft--;
            if (tk >= n_a) break;
            rans_block(job, a, J, item_ref(J, J.order ? J.order[tk] : tk), smem_u32(&S.tab[0][0]), ring_s,
                       smem_u32(&S.stage[warp][0]), &S.bar[warp][0], &S.sbar[warp], seq, sphase, lane, deadline);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int best = -1;
            uint32_t best_left = 0;
            for (uint32_t k = 0; k < job.n_arcs; k++) {
                const ArcJob Jk = load_arc(job, (int)k);
                const uint32_t taken = *((volatile uint32_t*)&tickets[k]);
                const uint32_t n_k = Jk.hi - Jk.lo;
                const uint32_t left = taken < n_k ? n_k - taken : 0;
                if (left > best_left) { best_left = left; best = (int)k; }
            }
            S.next_arc = best;
        }
        __syncthreads();
    }
}

size_t rans_smem_bytes() { return sizeof(RansSmem); }

static std::atomic<int> g_sm_count{0};

void note_sm_count(int n_sms) { g_sm_count.store(n_sms); }

int job_grid(int full, uint64_t need) {
    const int n_sms = std::max(g_sm_count.load(), 1);
    const uint64_t g = std::max<uint64_t>(need, (uint64_t)n_sms);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)full, g));
}

cudaError_t launch_prologue(uint32_t* counters, uint32_t n_counters, cudaStream_t st, int* errs, uint32_t n_errs) {
    k_prologue<<<1, 128, 0, st>>>(counters, n_counters, errs, n_errs);
    return cudaGetLastError();
}

cudaError_t launch_rans(const JobDev& job, int grid, cudaStream_t st) {
    const size_t sm = rans_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // a small job needs no more CTAs than its warps can take ticket runs
    const uint64_t per_cta = (uint64_t)kRansWarps * (job.chunk ? job.chunk : 1);
    grid = job_grid(grid, (job.n_items + per_cta - 1) / per_cta);
    k_rans<<<grid, kRansWarps * 32, sm, st>>>(job);
    return cudaGetLastError();
}

int rans_occupancy() {
    const size_t sm = rans_smem_bytes();
    cudaFuncSetAttribute(k_rans, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rans, kRansWarps * 32, sm) != cudaSuccess) return 0;
    return n;
}

}  // namespace acx
