// Register tiers of the X-Drop library.
//
// Slot layout shared by both tiers.  The live band of the paper's sweep (Sec. 3,
// Algorithm 1) is a few tens to a few hundred cells for realistic X, so the two previous
// anti-diagonals of a side extension live in registers: a window of W slots per
// anti-diagonal, where slot s of anti-diagonal d holds cell i = floor(d/2) + rb + s.  In
// these coordinates the diagonal predecessor S(i-1, j-1) sits in the same slot two
// anti-diagonals back, the two gap predecessors sit in slots (s-1, s) on odd d and
// (s, s+1) on even d, and a band that follows the main diagonal does not move; it only
// drifts with the indels of the alignment.  The window is re-centred when the band nears
// its edge (one guard slot on each side keeps the gap predecessors of the band's end
// cells), and a side whose band outgrows the window is handed to the next tier, which
// restarts it.  The two anti-diagonals are the paper's memory-restricted pair (Gotoh's
// two-diagonal scheme, Sec. 3): the new anti-diagonal overwrites d-2 slot by slot.
//
// Tier 0 ("narrow"): one thread per side extension, W = 32 slots.
// Tier 1 ("wide"):   one warp per side extension, W = 32 lanes x CW slots (256 or 1024);
//                    lanes exchange the boundary slot with a shuffle and reduce the
//                    anti-diagonal with REDUX.
//
// Per cell: the similarity from two packed 2-bit residue slices (xor + field test), the
// recurrence of Sec. 2.2 as max(S(i-1,j-1) + Sim, max(S(i-1,j), S(i,j-1)) + gap) with the
// DPX add-max, the X-Drop test against T of the completed anti-diagonals, a live bit for
// the band update, and a key v * 64 + (63 - t) whose maximum yields both the best score
// of the anti-diagonal and its lowest-i cell.
#include <cstdint>
#include <cuda_runtime.h>
#include "xd_device.cuh"
#include "xd_launch.h"

namespace xd {

// Register tiers keep scores in a narrower range so that a (score, slot) key fits 32 bits.
constexpr int32_t kNegR = -(1 << 24);
constexpr int32_t kDeadR = -(1 << 23);
constexpr int64_t kRegLimit = int64_t(1) << 23;

enum { kCont = 0, kDone = 1, kOverflow = 2 };

__device__ __forceinline__ uint32_t ld_word(const uint32_t* store, uint64_t n_words, int64_t w) {
    w = w < 0 ? 0 : w;
    w = w >= int64_t(n_words) ? int64_t(n_words) - 1 : w;
    return __ldg(store + w);
}

// Three raw store words from which a 32-residue slice is cut; loaded ahead of use.
struct Raw {
    uint32_t a, b, c, sh;
};

// Words covering residues [p, p + 32) of the packed DNA store (positions outside the store
// read clamped words; only cells outside the band ever use them).
__device__ __forceinline__ Raw load_raw(const uint32_t* store, uint64_t nw, int64_t p) {
    const int64_t w = p >> 4;
    Raw r;
    r.a = ld_word(store, nw, w);
    r.b = ld_word(store, nw, w + 1);
    r.c = ld_word(store, nw, w + 2);
    r.sh = uint32_t(p & 15) * 2u;
    return r;
}

// Field f (bits 2f, 2f+1) = residue p + f, or residue p + 31 - f when rev.
__device__ __forceinline__ uint64_t make_slice(const Raw& r, bool rev) {
    const uint64_t lo = (uint64_t(r.b) << 32) | r.a;
    uint64_t x = r.sh ? (lo >> r.sh) | (uint64_t(r.c) << (64 - r.sh)) : lo;
    if (rev) {
        x = __brevll(x);
        x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    }
    return x;
}

// Slice positions.  Field t of the H slice is H_side[hpos + t]; field t of the V slice is
// V_side[vpos - t].  H_side[k] = store[h0 + k] (right side) or store[h0 - k] (left side).
__device__ __forceinline__ int64_t h_base(int64_t h0, uint32_t side, int64_t hpos) {
    return side ? h0 - hpos - 31 : h0 + hpos;
}
__device__ __forceinline__ int64_t v_base(int64_t v0, uint32_t side, int64_t vpos) {
    return side ? v0 - vpos : v0 + vpos - 31;
}

// Per-side state shared by both tiers (replicated across the lanes of a warp in tier 1).
struct SideState {
    int64_t h0, v0;
    uint64_t cells;
    uint64_t hs, vs;          // residue slices of the current window (this lane's slots)
    Raw hn, vn;               // prefetched words of the next slice advance
    int32_t m, n, d, rb;
    int32_t L, U, T, best, bi, bj, barg;
    uint32_t flags, side;
    bool refresh;
};

// Band [lo, hi] of anti-diagonal d: [first live, last live + 1] of d-1 clipped to the
// matrix (Algorithm 1), then to delta_b cells centred on d-1's best cell when restricted.
__device__ __forceinline__ void band_of(const SideState& s, const Problem& P, int32_t d,
                                        int32_t& lo, int32_t& hi, uint32_t& flags) {
    lo = max(max(s.L, d - s.n), 0);
    hi = min(min(s.U + 1, s.m), d);
    if (P.delta && hi - lo + 1 > int32_t(P.delta)) {
        flags |= 1u;
        const int32_t start = min(s.barg - int32_t(P.delta >> 1), hi - int32_t(P.delta) + 1);
        lo = max(lo, start);
        hi = lo + int32_t(P.delta) - 1;
    }
}

// Keep the slices in step with the window: the H slice advances on even d, the V slice on
// odd d; the words of the next advance are always loaded one advance ahead.
template <bool ODD>
__device__ __forceinline__ void update_slices(SideState& s, const Problem& P, int64_t hpos, int64_t vpos) {
    if (s.refresh) {
        s.hs = make_slice(load_raw(P.store, P.n_words, h_base(s.h0, s.side, hpos)), s.side);
        s.vs = make_slice(load_raw(P.store, P.n_words, v_base(s.v0, s.side, vpos)), !s.side);
        s.hn = load_raw(P.store, P.n_words, h_base(s.h0, s.side, hpos + 1));
        s.vn = load_raw(P.store, P.n_words, v_base(s.v0, s.side, vpos + 1));
        s.refresh = false;
    } else if (!ODD) {
        s.hs = make_slice(s.hn, s.side);
        s.hn = load_raw(P.store, P.n_words, h_base(s.h0, s.side, hpos + 1));
    } else {
        s.vs = make_slice(s.vn, !s.side);
        s.vn = load_raw(P.store, P.n_words, v_base(s.v0, s.side, vpos + 1));
    }
}

// Cells of one lane's CW slots.  P1 holds d-1, P2 holds d-2 and receives d.  upb / lfb are
// the neighbours beyond the lane's first / last slot (another lane's, or -inf).
template <int CW, bool ODD>
__device__ __forceinline__ void cells_of(int32_t (&P1)[CW], int32_t (&P2)[CW], int32_t upb,
                                         int32_t lfb, uint64_t x, uint32_t bm, int32_t thr,
                                         int32_t gap, int32_t mat, int32_t mis, int32_t& kmax,
                                         uint32_t& lm) {
    kmax = INT32_MIN;
    lm = 0;
#pragma unroll
    for (int t = 0; t < CW; t++) {
        const int32_t up = ODD ? (t > 0 ? P1[t - 1] : upb) : P1[t];
        const int32_t lf = ODD ? P1[t] : (t < CW - 1 ? P1[t + 1] : lfb);
        const int32_t sig = ((x >> (2 * t)) & 3ull) ? mis : mat;
        const int32_t raw = __viaddmax_s32(max(up, lf), gap, P2[t] + sig);
        const bool live = raw >= thr && ((bm >> t) & 1u);
        const int32_t v = live ? raw : kNegR;
        P2[t] = v;
        lm |= live ? (1u << t) : 0u;
        kmax = max(kmax, v * 64 + (63 - t));
    }
}

__device__ __forceinline__ uint32_t slot_mask(int32_t from, int32_t to, int cw) {
    // bits [from, to] of a cw-bit lane mask, empty when the range misses the lane
    const int32_t a = max(from, 0), b = min(to + 1, cw);
    if (a >= b) return 0u;
    const uint64_t m = ((1ull << b) - 1ull) & ~((1ull << a) - 1ull);
    return uint32_t(m);
}

__device__ __forceinline__ void init_side(SideState& s, const Unit& u, int32_t rb) {
    s.h0 = int64_t(u.h0);
    s.v0 = int64_t(u.v0);
    s.m = int32_t(u.m);
    s.n = int32_t(u.n);
    s.side = u.side;
    s.rb = rb;
    s.d = 1;
    s.L = s.U = 0;
    s.T = s.best = s.bi = s.bj = s.barg = 0;
    s.flags = 0;
    s.cells = 1;
    s.hs = s.vs = 0;
    s.refresh = true;
}

// ---------------------------------------------------------------------------------------
// Tier 0: one thread per side extension, 32 slots.

template <bool ODD>
__device__ __forceinline__ int narrow_step(SideState& s, int32_t (&P1)[32], int32_t (&P2)[32],
                                           const Problem& P, int32_t mat, int32_t mis,
                                           int32_t* shbuf, int stride) {
    constexpr int C = 32;
    const int32_t d = s.d;
    int32_t ib = (d >> 1) + s.rb;
    int32_t lo, hi;
    band_of(s, P, d, lo, hi, s.flags);
    int32_t slo = lo - ib, shi = hi - ib;
    if (slo < 1 || shi > C - 2) {
        const int32_t w = hi - lo + 1;
        if (w > C - 2) return kOverflow;
        const int32_t k = slo - (1 + (C - 2 - w) / 2);
#pragma unroll
        for (int t = 0; t < C; t++) {
            shbuf[t * stride] = P1[t];
            shbuf[(C + t) * stride] = P2[t];
        }
#pragma unroll
        for (int t = 0; t < C; t++) {
            const int src = t + k;
            const bool in = src >= 0 && src < C;
            P1[t] = in ? shbuf[src * stride] : kNegR;
            P2[t] = in ? shbuf[(C + src) * stride] : kNegR;
        }
        s.rb += k;
        ib += k;
        slo -= k;
        shi -= k;
        s.refresh = true;
    }
    update_slices<ODD>(s, P, int64_t(ib) - 1, int64_t(d) - ib - 1);
    const uint32_t bm = (0xffffffffu >> (31 - shi)) & (0xffffffffu << slo);
    const int32_t thr = max(s.T - P.X, kDeadR);
    int32_t kmax;
    uint32_t lm;
    cells_of<C, ODD>(P1, P2, kNegR, kNegR, s.hs ^ s.vs, bm, thr, P.gap, mat, mis, kmax, lm);
    s.cells += uint64_t(hi - lo + 1);
    if (lm == 0) return kDone;
    s.L = ib + __ffs(lm) - 1;
    s.U = ib + 31 - __clz(lm);
    const int32_t vmax = kmax >> 6;
    const int32_t arg = ib + (63 - (kmax & 63));
    if (vmax > s.T) {
        s.T = vmax;
        s.best = vmax;
        s.bi = arg;
        s.bj = d - arg;
    }
    s.barg = arg;
    s.d = d + 1;
    return d == s.m + s.n ? kDone : kCont;
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_narrow(Problem P, Queues Q, int chunk) {
    constexpr int C = 32;
    extern __shared__ int32_t shift_smem[];
    int32_t* shbuf = shift_smem + threadIdx.x;
    const int stride = blockDim.x;
    const int32_t mat = P.sim[0], mis = P.sim[1];
    int32_t A[C], B[C];
    SideState s{};
    uint32_t uidx = 0, pair = 0, next = 0, end = 0;
    bool active = false;
    for (;;) {
        if (!active) {
            // pull the next unit; units this tier cannot run go to the wider tiers
            bool got = false;
            for (;;) {
                if (next >= end) {
                    const uint32_t base = atomicAdd(&Q.ctr[0], uint32_t(chunk));
                    if (base >= Q.n_units) break;
                    next = base;
                    end = min(base + uint32_t(chunk), Q.n_units);
                }
                uidx = Q.order[next++];
                const Unit u = P.units[uidx];
                if ((int64_t(u.m) + u.n) * P.max_abs >= kRegLimit || P.alpha != 4) {
                    push_unit(Q, 2, uidx);
                    continue;
                }
                init_side(s, u, -C / 2);
                pair = u.pair;
                got = true;
                break;
            }
            if (!got) break;
            if (s.m + s.n == 0) {
                write_side(P.results, pair, s.side, 0, 0, 0, 0, 1);
                atomicAdd(&P.stats[0], 1ull);
                atomicAdd(&P.stats[4], 1ull);
                continue;
            }
            // S(0,0) = 0 in the middle of the window, every other cell -inf (Sec. 2.2)
#pragma unroll
            for (int t = 0; t < C; t++) {
                A[t] = kNegR;
                B[t] = kNegR;
            }
            A[C / 2] = 0;
            active = true;
        }
        int r = narrow_step<true>(s, A, B, P, mat, mis, shbuf, stride);
        if (r == kCont) r = narrow_step<false>(s, B, A, P, mat, mis, shbuf, stride);
        if (r == kCont) continue;
        active = false;
        if (r == kDone) {
            write_side(P.results, pair, s.side, s.best, uint32_t(s.bi), uint32_t(s.bj), s.flags, s.cells);
            atomicAdd(&P.stats[0], 1ull);
            atomicAdd(&P.stats[4], (unsigned long long)s.cells);
        } else {
            push_unit(Q, 0, uidx);
            atomicAdd(&P.stats[3], 1ull);
            atomicAdd(&P.stats[7], (unsigned long long)s.cells);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Tier 1: one warp per side extension, 32 lanes x CW slots.  Lane l holds slots
// [l*CW, (l+1)*CW).  Every lane computes the band bookkeeping redundantly; the
// anti-diagonal's live range and best cell come from warp reductions.

template <int CW, bool ODD>
__device__ __forceinline__ int wide_step(SideState& s, int32_t (&P1)[CW], int32_t (&P2)[CW],
                                         const Problem& P, int32_t mat, int32_t mis, int lane) {
    constexpr int W = 32 * CW;
    const int32_t d = s.d;
    int32_t ib = (d >> 1) + s.rb;
    int32_t lo, hi;
    band_of(s, P, d, lo, hi, s.flags);
    int32_t slo = lo - ib, shi = hi - ib;
    if (slo < 1 || shi > W - 2) {
        // re-centre by whole lanes; any band of up to W - 2 - CW cells can be placed
        const int32_t w = hi - lo + 1;
        if (w > W - 2 - CW) return kOverflow;
        const int32_t target = (W - w) / 2;
        const int32_t diff = slo - target;
        const int32_t kl = diff >= 0 ? (diff + CW / 2) / CW : -((-diff + CW / 2) / CW);
        const int src = lane + kl;
        const bool in = src >= 0 && src < 32;
#pragma unroll
        for (int t = 0; t < CW; t++) {
            const int32_t a = __shfl_sync(0xffffffffu, P1[t], src & 31);
            const int32_t b = __shfl_sync(0xffffffffu, P2[t], src & 31);
            P1[t] = in ? a : kNegR;
            P2[t] = in ? b : kNegR;
        }
        s.rb += kl * CW;
        ib += kl * CW;
        slo -= kl * CW;
        shi -= kl * CW;
        s.refresh = true;
    }
    const int32_t sb = lane * CW;
    update_slices<ODD>(s, P, int64_t(ib) - 1 + sb, int64_t(d) - ib - 1 - sb);
    const uint32_t bm = slot_mask(slo - sb, shi - sb, CW);
    const int32_t thr = max(s.T - P.X, kDeadR);
    int32_t upb = kNegR, lfb = kNegR;
    if (ODD) {
        upb = __shfl_up_sync(0xffffffffu, P1[CW - 1], 1);
        if (lane == 0) upb = kNegR;
    } else {
        lfb = __shfl_down_sync(0xffffffffu, P1[0], 1);
        if (lane == 31) lfb = kNegR;
    }
    int32_t kmax;
    uint32_t lm;
    cells_of<CW, ODD>(P1, P2, upb, lfb, s.hs ^ s.vs, bm, thr, P.gap, mat, mis, kmax, lm);
    s.cells += uint64_t(hi - lo + 1);
    const bool any = lm != 0;
    if (__ballot_sync(0xffffffffu, any) == 0u) return kDone;
    const int32_t first = __reduce_min_sync(0xffffffffu, any ? sb + __ffs(lm) - 1 : INT32_MAX);
    const int32_t last = __reduce_max_sync(0xffffffffu, any ? sb + 31 - __clz(lm) : -1);
    s.L = ib + first;
    s.U = ib + last;
    const int32_t lv = kmax >> 6;
    const int32_t wmax = __reduce_max_sync(0xffffffffu, lv);
    const int32_t arg = ib + __reduce_min_sync(0xffffffffu, lv == wmax ? sb + (63 - (kmax & 63)) : INT32_MAX);
    if (wmax > s.T) {
        s.T = wmax;
        s.best = wmax;
        s.bi = arg;
        s.bj = d - arg;
    }
    s.barg = arg;
    s.d = d + 1;
    return d == s.m + s.n ? kDone : kCont;
}

template <int CW>
__global__ void __launch_bounds__(128) k_wide(Problem P, Queues Q, int level) {
    constexpr int W = 32 * CW;
    const int lane = threadIdx.x & 31;
    const int32_t mat = P.sim[0], mis = P.sim[1];
    const uint32_t n_q = *reinterpret_cast<volatile uint32_t*>(&Q.ctr[1 + 2 * level]);
    int32_t A[CW], B[CW];
    SideState s{};
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&Q.ctr[2 + 2 * level], 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n_q) break;
        const uint32_t uidx = Q.q[level][k];
        const Unit u = P.units[uidx];
        init_side(s, u, -W / 2);
        // S(0,0) = 0 in the middle of the window (lane 16, slot 0), every other cell -inf
#pragma unroll
        for (int t = 0; t < CW; t++) {
            A[t] = kNegR;
            B[t] = kNegR;
        }
        if (lane == 16) A[0] = 0;
        int r = kDone;
        if (s.m + s.n > 0) {
            for (;;) {
                r = wide_step<CW, true>(s, A, B, P, mat, mis, lane);
                if (r != kCont) break;
                r = wide_step<CW, false>(s, B, A, P, mat, mis, lane);
                if (r != kCont) break;
            }
        }
        if (lane == 0) {
            if (r == kDone) {
                write_side(P.results, u.pair, s.side, s.best, uint32_t(s.bi), uint32_t(s.bj), s.flags, s.cells);
                atomicAdd(&P.stats[1], 1ull);
                atomicAdd(&P.stats[5], (unsigned long long)s.cells);
            } else {
                push_unit(Q, level + 1, uidx);
                atomicAdd(&P.stats[3], 1ull);
                atomicAdd(&P.stats[7], (unsigned long long)s.cells);
            }
        }
        __syncwarp();
    }
}

template <int MINB>
static cudaError_t launch_narrow_v(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    constexpr int C = 32;
    const size_t smem = size_t(2) * C * cfg.narrow_threads * sizeof(int32_t);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_narrow<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_narrow<MINB><<<cfg.narrow_blocks, cfg.narrow_threads, smem, st>>>(P, Q, cfg.chunk);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    // register budget variants: 2 (255 registers), 3 (168), 4 (128) resident blocks per SM
    switch (cfg.narrow_minb) {
        case 2: return launch_narrow_v<2>(P, Q, cfg, st);
        case 4: return launch_narrow_v<4>(P, Q, cfg, st);
        default: return launch_narrow_v<3>(P, Q, cfg, st);
    }
}

cudaError_t launch_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    k_wide<8><<<cfg.wide_blocks, cfg.wide_threads, 0, st>>>(P, Q, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_wide<32><<<cfg.wide_blocks, cfg.wide_threads, 0, st>>>(P, Q, 1);
    return cudaGetLastError();
}

}  // namespace xd
