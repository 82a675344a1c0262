// Host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "xd_device.cuh"

namespace xd {

constexpr int kNumCtr = 8;

cudaError_t launch_pack(int alpha, const uint8_t* codes, uint64_t n_codes, uint32_t* store,
                        uint32_t* err, int n_sm, cudaStream_t st);
cudaError_t launch_units(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                         const uint32_t* lengths, uint32_t n_seqs, int32_t max_abs,
                         uint32_t max_len, Unit* units, uint32_t* bucket_of, uint32_t* hist,
                         uint32_t* err, cudaStream_t st);
cudaError_t launch_order(uint32_t* hist, uint32_t* ctr, int n_ctr, const uint32_t* bucket_of,
                         uint32_t n_units, uint32_t* order, cudaStream_t st);
cudaError_t launch_route_all_generic(const Queues& Q, cudaStream_t st);
cudaError_t launch_generic(const Problem& P, const Queues& Q, int32_t* scratch,
                           uint64_t stride, int n_blocks, cudaStream_t st);
cudaError_t launch_totals(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                          const uint32_t* lengths, uint32_t n_seqs, const Problem& P,
                          cudaStream_t st);

cudaError_t launch_accumulate(const unsigned long long* batch, unsigned long long* total, int n,
                              cudaStream_t st);

// Register tiers (xd_tiers.cu).  tier 0: one thread per unit; tier 1: one warp per unit.
struct TierConfig {
    int narrow_blocks, narrow_threads;
    int wide_blocks, wide_threads;
    int chunk;                  // units pulled per queue access in tier 0
    int narrow_minb;            // tier-0 register budget: resident 128-thread blocks per SM
};
cudaError_t launch_narrow(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st);
cudaError_t launch_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st);

}  // namespace xd
