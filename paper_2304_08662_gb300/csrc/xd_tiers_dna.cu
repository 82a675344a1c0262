// Register tiers, DNA level kernels with 32-bit scores (A = 4): the group kernels of
// xd_group.cuh, one launch per register level, for DNA batches outside the packed range
// (packed_ok false: X too large for 16-bit scores, X = infinity, or gap outside [-127, 0]).
#include "xd_group.cuh"

namespace xd {

cudaError_t launch_level_dna(const Problem& P, const Queues& Q, int variant, int in_q, int out_q,
                             int blocks, int chunk, cudaStream_t st) {
    switch (variant) {
        case kG1C16: return launch_group<1, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C32: return launch_group<1, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C16: return launch_group<4, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C16: return launch_group<8, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C16: return launch_group<16, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C16: return launch_group<32, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C32: return launch_group<32, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C32: return launch_group<4, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C32: return launch_group<8, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C32: return launch_group<16, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG4C8: return launch_group<4, 8, 4, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG8C8: return launch_group<8, 8, 4, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG16C8: return launch_group<16, 8, 4, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG32C8: return launch_group<32, 8, 4, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C24: return launch_group<1, 24, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG1C20: return launch_group<1, 20, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C32: return launch_group<2, 32, 2, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        case kG2C16: return launch_group<2, 16, 3, 4>(P, Q, in_q, out_q, blocks, chunk, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace xd
