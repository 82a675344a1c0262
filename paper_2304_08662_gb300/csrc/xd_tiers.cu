// Register tiers: the fused DNA grids (16-bit packed scores, A = kDna16) and the dispatch
// of register levels to the DNA or protein kernels (packed or 32-bit).  The kernels
// themselves are the templates of xd_group.cuh.
#include "xd_group.cuh"

namespace xd {

int variant_window(int v) {
    switch (v) {
        case kG1C16: return 16;
        case kG1C32: return 32;
        case kG4C16: return 64;
        case kG8C16: return 128;
        case kG16C16: return 256;
        case kG32C16: return 512;
        case kG32C32: return 1024;
        case kG4C32: return 128;
        case kG8C32: return 256;
        case kG16C32: return 512;
        case kG4C8: return 32;
        case kG8C8: return 64;
        case kG16C8: return 128;
        case kG32C8: return 256;
        case kG1C24: return 24;
        case kG1C20: return 20;
        case kG2C32: return 64;
        case kG2C16: return 32;
        default: return 0;
    }
}

cudaError_t launch_level(const Problem& P, const Queues& Q, const TierConfig& cfg, int level,
                         int n_sm, cudaStream_t st) {
    const int v = cfg.variant[level];
    const int in_q = level == 0 ? -1 : level - 1;
    const int out_q = level == cfg.n_levels - 1 ? kBandQ : level;
    const int blocks = n_sm * cfg.blocks_per_sm[v];
    if (P.alpha == 20)
        return packed_ok(P) ? launch_level_prot16(P, Q, v, in_q, out_q, blocks, cfg.chunk, st)
                            : launch_level_prot(P, Q, v, in_q, out_q, blocks, cfg.chunk, st);
    if (packed_ok(P)) return launch_level_dna16(P, Q, v, in_q, out_q, blocks, cfg.chunk, st);
    return launch_level_dna(P, Q, v, in_q, out_q, blocks, cfg.chunk, st);
}

bool packed_batch(const Problem& P) { return packed_ok(P);
}

bool fused_supported(const TierConfig& c, int alpha) {
    if (c.n_levels < 3) return false;
    const int a = c.variant[0], b = c.variant[1], d = c.variant[2];
    if (alpha == 20) return fused_supported_prot(a, b, d);
    return ((a == kG1C32 || a == kG1C24 || a == kG1C20 || a == kG1C16) && b == kG4C32 && d == kG8C32) ||
           (a == kG1C16 && b == kG2C32 && d == kG8C32) ||
           (a == kG1C32 && b == kG8C16 && d == kG16C16) ||
           (a == kG1C32 && b == kG16C16 && d == kG32C16) || (a == kG1C32 && b == kG8C16 && d == kG32C16) ||
           (a == kG1C16 && b == kG4C16 && d == kG16C16) || (a == kG1C16 && b == kG8C16 && d == kG32C16) ||
           (a == kG4C16 && b == kG16C16 && d == kG32C32) || (a == kG1C32 && b == kG32C8 && d == kG32C16) ||
           (a == kG1C16 && b == kG32C8 && d == kG32C16) || (a == kG1C16 && b == kG1C32 && d == kG16C16) ||
           (a == kG1C24 && b == kG16C16 && d == kG32C16) || (a == kG1C20 && b == kG16C16 && d == kG32C16) ||
           (a == kG1C32 && b == kG8C32 && d == kG32C16) || (a == kG1C32 && b == kG8C32 && d == kG16C32);
}

// Four-role grids compiled (packed scores only).
static bool fused4_supported(const TierConfig& c, int alpha) {
    if (c.n_levels < 4 || !c.fused4) return false;
    const int a = c.variant[0], b = c.variant[1], d = c.variant[2], e = c.variant[3];
    if (alpha == 20) return a == kG4C16 && b == kG8C16 && d == kG16C16 && e == kG32C32;
    if (a == kG1C32 && b == kG4C32 && d == kG8C32 && (e == kG16C32 || e == kG32C32 || e == kG32C16)) return true;
    return (a == kG1C32 && b == kG8C16 && d == kG16C16 && e == kG32C16) ||
           (a == kG1C24 && b == kG8C16 && d == kG16C16 && e == kG32C16) ||
           (a == kG1C20 && b == kG8C16 && d == kG16C16 && e == kG32C16) ||
           (a == kG1C32 && b == kG4C16 && d == kG8C16 && e == kG16C16);
}

int fused_roles(const TierConfig& c, int alpha) {
    if (!c.fused) return 0;
    if (fused4_supported(c, alpha)) return 4;
    return fused_supported(c, alpha) ? 3 : 0;
}

static cudaError_t launch_fused4_levels(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                        cudaStream_t st) {
    const int a = cfg.variant[0], b = cfg.variant[1], d = cfg.variant[2], e = cfg.variant[3];
    if (!packed_ok(P)) return cudaErrorInvalidValue;
    if (P.alpha == 20) {
        if (a == kG4C16 && b == kG8C16 && d == kG16C16 && e == kG32C32)
            return launch_fused4<4, 16, 8, 16, 16, 16, 32, 32, 2, kProt16, 0, 4>(P, Q, cfg, n_sm, st);
        return cudaErrorInvalidValue;
    }
    if (a == kG1C32 && b == kG4C32 && d == kG8C32) return launch_fused_wide4(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG8C16 && d == kG16C16 && e == kG32C16)
        return launch_fused4<1, 32, 8, 16, 16, 16, 32, 16, 4, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C24 && b == kG8C16 && d == kG16C16 && e == kG32C16)
        return launch_fused4<1, 24, 8, 16, 16, 16, 32, 16, 2, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C20 && b == kG8C16 && d == kG16C16 && e == kG32C16)
        return launch_fused4<1, 20, 8, 16, 16, 16, 32, 16, 2, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG4C16 && d == kG8C16 && e == kG16C16)
        return launch_fused4<1, 32, 4, 16, 8, 16, 16, 16, 2, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_levels(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                cudaStream_t st) {
    const int a = cfg.variant[0], b = cfg.variant[1], d = cfg.variant[2];
    if (fused_roles(cfg, P.alpha) == 4) return launch_fused4_levels(P, Q, cfg, n_sm, st);
    if (P.alpha == 20) return launch_fused_levels_prot(P, Q, cfg, n_sm, st);
    if (!packed_ok(P)) return cudaErrorInvalidValue;   // DNA grids are compiled packed only
    // 32-slot wide levels after a 20-, 24- or 32-slot first level (xd_tiers_wide.cu)
    if ((b == kG4C32 && d == kG8C32 && (a == kG1C32 || a == kG1C24 || a == kG1C20 || a == kG1C16)) ||
        (a == kG1C16 && b == kG2C32 && d == kG8C32))
        return launch_fused_wide(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG8C16 && d == kG16C16) return launch_fused<1, 32, 8, 16, 16, 16, 2, kDna16>(P, Q, cfg, n_sm, st);
    // 128 registers (four blocks per SM, no spills) unless fused_minb asks for three blocks
    if (a == kG1C32 && b == kG16C16 && d == kG32C16)
        return cfg.fused_minb == 3   ? launch_fused<1, 32, 16, 16, 32, 16, 3, kDna16>(P, Q, cfg, n_sm, st)
               : cfg.long_shape == 2 ? launch_fused<1, 32, 16, 16, 32, 16, 4, kDna16, 4, 8>(P, Q, cfg, n_sm, st)
               : cfg.long_shape == 0 ? launch_fused<1, 32, 16, 16, 32, 16, 4, kDna16, 32, 4>(P, Q, cfg, n_sm, st)
                                     : launch_fused<1, 32, 16, 16, 32, 16, 4, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG8C16 && d == kG32C16) return launch_fused<1, 32, 8, 16, 32, 16, 2, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG32C8 && d == kG32C16) return launch_fused<1, 32, 32, 8, 32, 16, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C16 && b == kG32C8 && d == kG32C16) return launch_fused<1, 16, 32, 8, 32, 16, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C16 && b == kG1C32 && d == kG16C16) return launch_fused<1, 16, 1, 32, 16, 16, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C24 && b == kG16C16 && d == kG32C16) return launch_fused<1, 24, 16, 16, 32, 16, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C20 && b == kG16C16 && d == kG32C16) return launch_fused<1, 20, 16, 16, 32, 16, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG8C32 && d == kG32C16) return launch_fused<1, 32, 8, 32, 32, 16, 2, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C32 && b == kG8C32 && d == kG16C32)
        return cfg.fused_minb == 3 ? launch_fused<1, 32, 8, 32, 16, 32, 3, kDna16>(P, Q, cfg, n_sm, st)
                                   : launch_fused<1, 32, 8, 32, 16, 32, 2, kDna16, 8, 4>(P, Q, cfg, n_sm, st);
    if (a == kG1C16 && b == kG4C16 && d == kG16C16) return launch_fused<1, 16, 4, 16, 16, 16, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG1C16 && b == kG8C16 && d == kG32C16) return launch_fused<1, 16, 8, 16, 32, 16, 3, kDna16>(P, Q, cfg, n_sm, st);
    if (a == kG4C16 && b == kG16C16 && d == kG32C32) return launch_fused<4, 16, 16, 16, 32, 32, 2, kDna16, 32, 4>(P, Q, cfg, n_sm, st);
    return cudaErrorInvalidValue;
}

}  // namespace xd
