// Fused entropy stage + local pass of a whole-archive decode (paper, Table 1:
// the dense full-pipe decoder runs an ANS kernel, then a match kernel; here
// both run at once on every SM).
//
// The entropy stage is bound by its instruction issue (a dependent chain of
// table load, multiply-add and renormalisation per lane), the local pass by
// latency (CTA scans, barriers, shared-memory round trips).  Run one after the
// other, each leaves the SMs half idle; in one persistent CTA per SM they fill
// each other's gaps:
//   * warps [0, R) are entropy warps: they share the archive's four decode
//     tables in shared memory, take blocks from a ticket in the hand-out order
//     (most symbols first), decode a block's four streams into its scratch
//     region with the same lane decoders as k_rans, and publish the block with
//     a release store of its ready flag;
//   * the other warps form G groups of 128 threads, each a local pass with
//     its own shared-memory workspace and named barrier (the same code as
//     k_local); a group takes tickets in the same order and, before it stages
//     a block's streams with bulk copies, waits (bounded) for its ready flag.
// The launch is cooperative, so every CTA is resident: the entropy warps never
// wait on the groups, so every flag is eventually set and every group wait
// ends.  The cross-block pass (k_external) follows as its own launch.
#include <algorithm>

#include "launch.h"
#include "local_dev.cuh"
#include "rans_dev.cuh"

namespace acx {

constexpr int kFusedRansWarps = 12;
constexpr int kFusedMaxGroups = 3;
constexpr int kFusedMaxThreads = 32 * (kFusedRansWarps + kLocWarps * kFusedMaxGroups);

struct FusedLayout {
    uint32_t tab, ring, bar, stage, loc, loc_stride, total;
};

// Shared memory of a fused CTA with G local groups whose workspaces hold
// blocks of up to T tokens and LB length bytes.
__host__ __device__ inline FusedLayout fused_layout(uint32_t T, uint32_t LB, int G, bool lvl) {
    FusedLayout F;
    F.tab = 0;                                           // 4 x 4096 decode entries
    F.ring = 4 * kM * 4;                                 // (R + 1) x 2 KiB: R rings, 2 KiB-aligned inside
    F.bar = F.ring + (kFusedRansWarps + 1) * 2 * kRingWords;  // R x (kSlots + 1) mbarriers
    F.stage = F.bar + kFusedRansWarps * (kSlots + 1) * 8;  // R x kStageBytes symbol stages (16-aligned)
    const uint32_t end = F.stage + kFusedRansWarps * kStageBytes;
    F.loc = (end + 127) & ~127u;
    F.loc_stride = loc_layout(T, LB, false, lvl).total;  // 128-byte multiple
    F.total = F.loc + (uint32_t)G * F.loc_stride;
    return F;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(kFusedMaxThreads, 1) k_fused(JobDev job, int G) {
    extern __shared__ __align__(128) uint8_t sm[];
    const FusedLayout F = fused_layout(job.max_tok, job.max_lenb, G, (job.flags & kJobLevels) != 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ArcJob& J = job.one;
    {
        const uint4* src = reinterpret_cast<const uint4*>(J.dtab);
        uint4* dst = reinterpret_cast<uint4*>(sm + F.tab);
        for (uint32_t i = threadIdx.x; i < 4 * kM / 4; i += blockDim.x) dst[i] = src[i];
    }
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + F.bar) + warp * (kSlots + 1);
    if (warp < kFusedRansWarps && lane <= kSlots) mbar_init(&bars[lane], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const uint64_t deadline = gtimer() + kCopyWaitNs;  // the entropy warps wait only for their copies
    if (warp < kFusedRansWarps) {
        const uint32_t ring_s =
            ((smem_u32(sm + F.ring) + kRingMask) & ~(uint32_t)kRingMask) + (uint32_t)warp * (2 * kRingWords);
        const uint32_t tab0_s = smem_u32(sm + F.tab);
        const uint32_t n_a = J.hi - J.lo;
        uint32_t seq = 0, sphase = 0;
        for (;;) {
            uint32_t t0 = 0;
            if (lane == 0) t0 = atomicAdd(&job.counters[3], 1u);
            const uint32_t tk = __shfl_sync(ACX_FULL, t0, 0);
            if (tk >= n_a) break;
            const uint32_t item = J.order ? J.order[tk] : tk;
            rans_block(job, 0, J, item_ref(J, item), tab0_s, ring_s, smem_u32(sm + F.stage) + warp * kStageBytes,
                       &bars[0], &bars[kSlots], seq, sphase, lane, deadline);
            // publish: every lane's stream stores, then the flag (a corrupt
            // block is published too; its local pass finds it corrupt)
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");
                st_release_u32(job.ready + item, 1u);
            }
        }
        return;
    }
    const int g = (warp - kFusedRansWarps) / kLocWarps;
    if (g >= G) return;
    local_worker(job, sm + F.loc + g * F.loc_stride, 1 + g, threadIdx.x - 32 * (kFusedRansWarps + kLocWarps * g));
}

int fused_groups(uint32_t max_tok, uint32_t max_lenb, bool lvl) {
    for (int G = kFusedMaxGroups; G >= 1; G--)
        if (fused_layout(max_tok, max_lenb, G, lvl).total <= 227u * 1024) return G;
    return 0;
}

cudaError_t launch_fused(const JobDev& job, int G, int grid, cudaStream_t st) {
    const FusedLayout F = fused_layout(job.max_tok, job.max_lenb, G, (job.flags & kJobLevels) != 0);
    cudaError_t e = cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F.total);
    if (e != cudaSuccess) return e;
    struct Arg {
        const JobDev* job;
        int G, grid;
        size_t smem;
        cudaStream_t st;
    } a{&job, G, grid, F.total, st};
    return coop_ordered(st, [](void* p) -> cudaError_t {
        const Arg* a = static_cast<const Arg*>(p);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(a->grid);
        cfg.blockDim = dim3(32 * (kFusedRansWarps + kLocWarps * a->G));
        cfg.dynamicSmemBytes = a->smem;
        cfg.stream = a->st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_fused, *a->job, a->G);
    }, &a);
}

int fused_occupancy(int G, uint32_t max_tok, uint32_t max_lenb, bool lvl) {
    const FusedLayout F = fused_layout(max_tok, max_lenb, G, lvl);
    if (cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F.total) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused, 32 * (kFusedRansWarps + kLocWarps * G), F.total) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace acx
