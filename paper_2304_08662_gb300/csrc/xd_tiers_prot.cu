// Register tiers, protein instantiations: the 32-bit level kernels (A = 20, for batches
// outside the packed range) and the fused grids (16-bit packed scores, A = kProt16), the
// group kernels of xd_group.cuh with 16-bit similarity-table offsets as residue slices.
#include "xd_group.cuh"

namespace xd {

cudaError_t launch_level_prot(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                              int blocks, int chunk, cudaStream_t st) {
    switch (variant) {
        case kG1C16: return launch_group<1, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C16: return launch_group<4, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C16: return launch_group<8, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C16: return launch_group<16, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C16: return launch_group<32, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C32: return launch_group<32, 32, 2, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C8: return launch_group<8, 8, 4, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C8: return launch_group<32, 8, 4, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C32: return launch_group<1, 32, 2, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C24: return launch_group<1, 24, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C8: return launch_group<4, 8, 4, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C32: return launch_group<2, 32, 2, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C16: return launch_group<2, 16, 3, 20>(P, Q, in_q, out_q, blocks, chunk, st);
        default: return cudaErrorInvalidValue;
    }
}

bool fused_supported_prot(int a, int b, int d) {
    return (a == kG4C16 && b == kG16C16 && d == kG32C32) || (a == kG1C16 && b == kG4C16 && d == kG16C16) ||
           (a == kG4C16 && b == kG8C16 && d == kG16C16);
}

cudaError_t launch_fused_levels_prot(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                     cudaStream_t st) {
    const int a = cfg.variant[0], b = cfg.variant[1], d = cfg.variant[2];
    if (!packed_ok(P)) return cudaErrorInvalidValue;   // protein grids are compiled packed only
    if (a == kG4C16 && b == kG16C16 && d == kG32C32) return launch_fused<4, 16, 16, 16, 32, 32, 2, kProt16>(P, Q, cfg, n_sm, st);
    if (a == kG1C16 && b == kG4C16 && d == kG16C16) return launch_fused<1, 16, 4, 16, 16, 16, 3, kProt16>(P, Q, cfg, n_sm, st);
    // 16-slot levels only: 128 registers, four blocks per SM, like the separate level launches
    if (a == kG4C16 && b == kG8C16 && d == kG16C16) return launch_fused<4, 16, 8, 16, 16, 16, 4, kProt16>(P, Q, cfg, n_sm, st);
    return cudaErrorInvalidValue;
}

}  // namespace xd
