// Register tiers, DNA level kernels with 16-bit packed scores (A = kDna16): the group
// kernels of xd_group.cuh, one launch per register level.  Used when packed_ok holds for
// the batch (X, gap and scores within the packed range); other DNA batches take the
// 32-bit levels of xd_tiers_dna.cu.
#include "xd_group.cuh"

namespace xd {

cudaError_t launch_level_dna16(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                               int blocks, int chunk, cudaStream_t st) {
    switch (variant) {
        case kG1C16: return launch_group<1, 16, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C32: return launch_group<1, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C16: return launch_group<4, 16, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C16: return launch_group<8, 16, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C16: return launch_group<16, 16, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C16: return launch_group<32, 16, 3, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C32: return launch_group<32, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C32: return launch_group<4, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C32: return launch_group<8, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C32: return launch_group<16, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C8: return launch_group<4, 8, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C8: return launch_group<8, 8, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C8: return launch_group<16, 8, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C8: return launch_group<32, 8, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C24: return launch_group<1, 24, 3, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C20: return launch_group<1, 20, 3, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C32: return launch_group<2, 32, 2, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C16: return launch_group<2, 16, 4, kDna16>(P, Q, in_q, out_q, blocks, chunk, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace xd
