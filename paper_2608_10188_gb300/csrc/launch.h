// Host-side launchers of the decode kernels (defined in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "internal.h"

namespace acx {

// Clears counters[0, n_counters) and the statistics/list/barrier words, and
// errs[0, n_errs) (status words that the kernels set).
cudaError_t launch_prologue(uint32_t* counters, uint32_t n_counters, cudaStream_t st, int* errs = nullptr,
                            uint32_t n_errs = 0);
cudaError_t launch_rans(const JobDev& job, int grid, cudaStream_t st);
cudaError_t launch_local(const JobDev& job, int grid, cudaStream_t st);
// Cooperative launch (every CTA resident); recorded as a cooperative kernel
// node when the stream is being captured into a graph.
cudaError_t launch_external(const JobDev& job, int grid, cudaStream_t st);
// Run launch(arg) (a cooperative launch on st) after the previous cooperative
// launch of this process on the current device has completed, and make it the
// one the next waits for (see assemble.cu).
cudaError_t coop_ordered(cudaStream_t st, cudaError_t (*launch)(void*), void* arg);
// The level list of a level-ordered job (kJobLevels): a per-level scan over
// the items, then one warp per item writes its pieces' entries.
cudaError_t launch_level_list(const JobDev& job, cudaStream_t st);
// Pending pieces above which the automatic policy takes a level-ordered job's
// pieces in level order: 16 per thread of the cross-block pass's grid.
uint32_t lvl_auto_min_pieces_for(int ext_ctas);
cudaError_t launch_plain(const JobDev& job, int grid, cudaStream_t st);
// Fused entropy stage + local pass of a whole single-archive job (job.ready
// set, its flags cleared): G local groups per CTA, one CTA per SM
// (cooperative).  fused_groups: the most groups whose workspaces fit a CTA
// for blocks of max_tok tokens and max_lenb length bytes (0: none fits).
cudaError_t launch_fused(const JobDev& job, int G, int grid, cudaStream_t st);
int fused_groups(uint32_t max_tok, uint32_t max_lenb, bool lvl);
int fused_occupancy(int G, uint32_t max_tok, uint32_t max_lenb, bool lvl);
size_t local_smem_bytes(uint32_t T, uint32_t LB, bool need = false, bool lvl = false);
int rans_occupancy();
// Grid of a persistent kernel for a job that can use `need` CTAs at most:
// no more than `full`, and no fewer than one per SM, so that a mid-size job
// spreads its warps over the whole GPU instead of packing a few SMs.  The SM
// count is recorded when a context is created (no API call at launch time,
// which may be inside a graph capture).
int job_grid(int full, uint64_t need);
void note_sm_count(int n_sms);
int local_occupancy(size_t smem);
int external_occupancy();
int plain_occupancy();
// Copy regions out of block slots (block a at out + slot[a]*kBlock): the one
// request `one` (list == nullptr) or list[0, n_req); max_len sizes the grid.
cudaError_t launch_gather(const GatherReq* one, const GatherReq* list, uint32_t n_req, uint64_t max_len,
                          const uint8_t* out, const uint32_t* slot, cudaStream_t st);

}  // namespace acx
