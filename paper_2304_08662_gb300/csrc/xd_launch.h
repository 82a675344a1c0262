// Host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "xd_device.cuh"

namespace xd {

// queue counters: [0] order pull, [1 + 2k] / [2 + 2k] length / pull of q[k], then producer
// warps finished (roles 0 and 1), the record counter, the pull counter of the long-side
// head, and producer warps finished in role 2 (four-role grids)
constexpr int kNumCtr = 6 + 2 * kLevels;
constexpr int kLongPull = 4 + 2 * kLevels;
constexpr int kDone2 = 5 + 2 * kLevels;

cudaError_t launch_pack(int alpha, const uint8_t* codes, uint64_t n_codes, uint32_t* store,
                        uint32_t* err, int n_sm, cudaStream_t st);
cudaError_t launch_units(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                         const uint32_t* lengths, uint32_t n_seqs, uint64_t n_res, int32_t max_abs,
                         uint32_t max_len, uint32_t pair_base, uint64_t res_base, Unit* units,
                         uint32_t* bucket_of, uint32_t* hist, uint32_t* err, cudaStream_t st);
cudaError_t launch_order(uint32_t* hist, uint32_t* ctr, int n_ctr, const uint32_t* bucket_of,
                         uint32_t n_units, uint32_t* order, cudaStream_t st);
cudaError_t launch_route_all_generic(const Queues& Q, cudaStream_t st);
cudaError_t launch_generic(const Problem& P, const Queues& Q, int32_t* scratch,
                           uint64_t stride, int n_blocks, cudaStream_t st);
// Band tier with nw warps per side (1, 2, 4, 8, 16 or 32: 32 - 1024 threads per alignment).
cudaError_t launch_band(const Problem& P, const Queues& Q, int n_sm, int nw, cudaStream_t st);
cudaError_t launch_totals(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                          const uint32_t* lengths, uint32_t n_seqs, uint64_t n_res, uint32_t pair_base,
                          uint64_t res_base, const Problem& P, cudaStream_t st);

cudaError_t launch_accumulate(const unsigned long long* batch, unsigned long long* total, int n,
                              cudaStream_t st);

// Register tiers (xd_tiers.cu): a chain of up to kLevels - 2 register levels, each a
// group kernel with G lanes per side extension and CG slots per lane (window G * CG),
// followed by the generic tier.  Variant ids name the compiled (G, CG) pairs.
enum GroupVariant {
    kG1C16 = 0, kG1C32 = 1, kG4C16 = 2, kG8C16 = 3, kG16C16 = 4, kG32C16 = 5, kG32C32 = 6,
    kG4C32 = 7, kG8C32 = 8, kG16C32 = 9, kG4C8 = 10, kG8C8 = 11, kG16C8 = 12, kG32C8 = 13,
    kG1C24 = 14, kG1C20 = 15, kG2C32 = 16, kG2C16 = 17,
    kNumGroupVariants = 18
};

struct TierConfig {
    int n_levels;                       // register levels before the generic tier
    int variant[kLevels - 2];           // GroupVariant of each level
    int blocks_per_sm[kNumGroupVariants];
    int chunk;                          // units pulled per queue access (single-lane groups)
    bool fused;                         // fuse levels 0-2 into one persistent grid
    int every1, every2;                 // fused grid: warps starting in role 1 / role 2
    int every3;                         // four-role grid: warps starting in role 3 (0: three roles)
    int fused_minb;                     // fused grid register budget: 3 = three resident blocks per SM
                                        // (no long role), else the 128-register build (four)
    int long_permille;                  // fused grid: head of the cost order (per mille of the
                                        // units) run first by wider groups (0 = none)
    int long_shape;                     // their groups: 0 = 32 lanes x 4 slots, 1 = 8 x 4, 2 = 4 x 8
    int wait_limit_ms;                  // fused grid: live-queue wait limit (0 = default, 10 s)
    bool phantom_producer;              // failure-detection test: one producer never finishes
    int band_warps;                     // band tier: warps per side (1 - 32; 0 = default 8)
    bool fused4;                        // a compiled four-level grid is used when the chain has one
};

// Runs register level `level` of the chain: pulls the cost-ordered list (level 0) or
// q[level - 1], escalates to q[level] (the generic queue after the last level).
cudaError_t launch_level(const Problem& P, const Queues& Q, const TierConfig& cfg, int level,
                         int n_sm, cudaStream_t st);
int variant_window(int variant);

// Levels 0-2 fused into one cooperatively launched persistent grid (consumers of the
// escalation queues start while the narrower levels still run).  Only some variant
// triples are compiled (per alphabet: 4 = DNA, 20 = protein).
bool fused_supported(const TierConfig& cfg, int alpha);
cudaError_t launch_fused_levels(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                cudaStream_t st);
// Levels 0-3 in one grid (four roles); fused_roles(cfg, alpha) is 4 when the variant
// quadruple is compiled and cfg asks for it, 3 for the triple, else 0.
int fused_roles(const TierConfig& cfg, int alpha);
// The fused grids with 32-slot wide levels (xd_tiers_wide.cu).
cudaError_t launch_fused_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm, cudaStream_t st);
cudaError_t launch_fused_wide4(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm, cudaStream_t st);

// DNA levels (xd_tiers_dna.cu) and protein instantiations (xd_tiers_prot.cu), reached
// through the launchers above.
cudaError_t launch_level_dna(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                             int blocks, int chunk, cudaStream_t st);
cudaError_t launch_level_dna16(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                               int blocks, int chunk, cudaStream_t st);
cudaError_t launch_level_prot16(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                                int blocks, int chunk, cudaStream_t st);
// Batches whose scores fit the packed 16-bit levels (fused grids are compiled for these
// only; other batches run one launch per level).
bool packed_batch(const Problem& P);
cudaError_t launch_level_prot(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                              int blocks, int chunk, cudaStream_t st);
bool fused_supported_prot(int a, int b, int d);
cudaError_t launch_fused_levels_prot(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                     cudaStream_t st);

// Throughput probes (xd_roof.cu).
cudaError_t probe_rate(int op, int n_sm, double* rate, float* ms);

}  // namespace xd
