// Register tiers: fused DNA grids (16-bit packed scores) whose wide levels have 32 slots per
// lane -- 1 x 16 / 1 x 20 / 1 x 24 / 1 x 32 -> 4 x 32 -> 8 x 32 (windows 128 and 256 for the wide
// sides, with the fewest lanes per side), and 1 x 16 -> 2 x 32 -> 8 x 32.  These are the chains of launches whose time is set by the
// total work; built for four blocks per SM (128 registers; the default of launches of 2^20 or
// more side extensions), three (166-168 registers) and, for the 1 x 32 one, two.
#include "xd_group.cuh"

namespace xd {

cudaError_t launch_fused_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm, cudaStream_t st) {
    if (!packed_ok(P) || P.alpha != 4) return cudaErrorInvalidValue;
    const int a = cfg.variant[0], b = cfg.variant[1];
    if (a == kG1C16 && b == kG2C32) return launch_fused<1, 16, 2, 32, 8, 32, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG1C16) return launch_fused<1, 16, 4, 32, 8, 32, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG1C20)
        return cfg.fused_minb == 4 ? launch_fused<1, 20, 4, 32, 8, 32, 4, kDna16>(P, Q, cfg, n_sm, st)
                                   : launch_fused<1, 20, 4, 32, 8, 32, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG1C24)
        return cfg.fused_minb == 4 ? launch_fused<1, 24, 4, 32, 8, 32, 4, kDna16>(P, Q, cfg, n_sm, st)
                                   : launch_fused<1, 24, 4, 32, 8, 32, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (cfg.fused_minb == 4) return launch_fused<1, 32, 4, 32, 8, 32, 4, kDna16>(P, Q, cfg, n_sm, st);
    return cfg.fused_minb == 3 ? launch_fused<1, 32, 4, 32, 8, 32, 3, kDna16>(P, Q, cfg, n_sm, st)
                               : launch_fused<1, 32, 4, 32, 8, 32, 2, kDna16>(P, Q, cfg, n_sm, st);
}

// Four levels in one grid: the 32-slot wide levels, then 16 x 32, 32 x 32 or 32 x 16 as the
// fourth role, whose sides (bands wider than 254 cells, the longest serial chains of a
// launch) then start as soon as they escalate instead of after the grid.
cudaError_t launch_fused_wide4(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm, cudaStream_t st) {
    if (!packed_ok(P) || P.alpha != 4) return cudaErrorInvalidValue;
    switch (cfg.variant[3]) {
        case kG16C32: return launch_fused4<1, 32, 4, 32, 8, 32, 16, 32, 3, kDna16, 0, 4>(P, Q, cfg, n_sm, st);
        case kG32C32: return launch_fused4<1, 32, 4, 32, 8, 32, 32, 32, 3, kDna16, 0, 4>(P, Q, cfg, n_sm, st);
        case kG32C16: return launch_fused4<1, 32, 4, 32, 8, 32, 32, 16, 3, kDna16, 0, 4>(P, Q, cfg, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace xd
