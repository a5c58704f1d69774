// Gather of decoded regions out of block slots (range decodes, serving):
// request r copies the original bytes [start, start + len) into its own
// device buffer, reading block a's bytes at out + slot[a] * kBlock.
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace acx {

// Each thread moves one 16-byte piece of a request's output: sixteen byte
// loads (the source of a piece may straddle two slots) and one 16-byte store
// when the destination is aligned.
__global__ void __launch_bounds__(256) k_gather(GatherReq one, const GatherReq* list, uint32_t n_req,
                                                const uint8_t* __restrict__ out, const uint32_t* __restrict__ slot) {
    const uint32_t r = blockIdx.y;
    if (r >= n_req) return;
    const GatherReq q = list ? list[r] : one;
    const uint64_t pieces = (q.len + 15) / 16;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pieces; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t o = p * 16;
        const uint32_t m = q.len - o < 16 ? (uint32_t)(q.len - o) : 16u;
        uint8_t v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            if ((uint32_t)k < m) {
                const uint64_t pos = q.start + o + k;
                v[k] = out[(uint64_t)slot[pos >> 14] * kBlock + (pos & (kBlock - 1))];
            } else {
                v[k] = 0;
            }
        }
        uint8_t* d = q.dst + o;
        if (m == 16 && ((uintptr_t)d & 15) == 0) {
            uint4 w;
            memcpy(&w, v, 16);
            *reinterpret_cast<uint4*>(d) = w;
        } else {
            for (uint32_t k = 0; k < m; k++) d[k] = v[k];
        }
    }
}

cudaError_t launch_gather(const GatherReq* one, const GatherReq* list, uint32_t n_req, uint64_t max_len,
                          const uint8_t* out, const uint32_t* slot, cudaStream_t st) {
    if (n_req == 0) return cudaSuccess;
    const uint64_t pieces = (max_len + 15) / 16;
    const uint32_t gx = (uint32_t)std::min<uint64_t>(std::max<uint64_t>((pieces + 255) / 256, 1), 1024);
    k_gather<<<dim3(gx, n_req), 256, 0, st>>>(one ? *one : GatherReq{}, list, n_req, out, slot);
    return cudaGetLastError();
}

}  // namespace acx
