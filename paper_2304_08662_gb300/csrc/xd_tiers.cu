// Register tiers of the X-Drop library.
//
// Tier 0 ("narrow"): one thread per side extension.  The live band of the paper's sweep
// (Sec. 3, Algorithm 1) is a few tens of cells for realistic X, so a thread keeps the two
// previous anti-diagonals of its unit entirely in registers: a window of C slots per
// anti-diagonal, where slot s of anti-diagonal d holds cell i = floor(d/2) + rb + s.  In
// these coordinates the diagonal predecessor S(i-1, j-1) sits in the same slot two
// anti-diagonals back, the two gap predecessors sit in slots (s-1, s) on odd d and
// (s, s+1) on even d, and a band that follows the main diagonal does not move at all; it
// only drifts with the indels of the alignment.  The window is re-centred (through
// shared memory) when the band nears its edge, and a unit whose band outgrows the window
// is handed to the next tier, which restarts it.  The two anti-diagonals are the
// paper's memory-restricted pair A1/A2 (Gotoh's two-diagonal scheme, Sec. 3): the new
// anti-diagonal overwrites d-2 in place, slot by slot.
//
// Per cell: the similarity from two packed 2-bit residue slices (xor + field test), the
// recurrence of Sec. 2.2 as max(S(i-1,j-1) + Sim, max(S(i-1,j), S(i,j-1)) + gap) with the
// DPX add-max, the X-Drop test against T of the completed anti-diagonals, a live bit for
// the band update, and a key v * 64 + (63 - s) whose maximum yields both T' and the
// lowest-i best cell of the anti-diagonal.
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

// 32 DNA residues: field f (bits 2f, 2f+1) = residue at absolute position pos + f.
// Positions outside the store read clamped words (only cells outside the band use them).
__device__ __forceinline__ uint64_t slice_fwd(const uint32_t* store, uint64_t nw, int64_t pos) {
    const int64_t w = pos >> 4;
    const uint32_t sh = uint32_t(pos & 15) * 2u;
    const uint64_t lo = (uint64_t(ld_word(store, nw, w + 1)) << 32) | ld_word(store, nw, w);
    const uint64_t hi = ld_word(store, nw, w + 2);
    return sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
}

// field f = residue at pos - f
__device__ __forceinline__ uint64_t slice_bwd(const uint32_t* store, uint64_t nw, int64_t pos) {
    const uint64_t x = __brevll(slice_fwd(store, nw, pos - 31));
    return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

struct NarrowState {
    int64_t h0, v0;
    uint64_t cells;
    uint64_t hs, vs;          // residue slices of the current window
    int32_t m, n, d, rb;
    int32_t L, U, T, best, bi, bj, barg;
    uint32_t flags, side;
};

// One anti-diagonal d = s.d of the unit.  P1 holds d-1, P2 holds d-2 and receives d.
template <int C, bool ODD>
__device__ __forceinline__ int narrow_step(NarrowState& s, int32_t (&P1)[C], int32_t (&P2)[C],
                                           const Problem& P, int32_t mat, int32_t mis,
                                           int32_t* shbuf, int stride) {
    static_assert(C == 32, "slot masks assume 32 slots");
    const int32_t d = s.d;
    int32_t ib = (d >> 1) + s.rb;
    // band of this anti-diagonal: [first live, last live + 1] of d-1, clipped to the matrix
    int32_t lo = max(max(s.L, d - s.n), 0);
    int32_t hi = min(min(s.U + 1, s.m), d);
    if (P.delta && hi - lo + 1 > int32_t(P.delta)) {
        // memory-restricted window of delta_b cells, centred on the best cell of d-1
        s.flags |= 1u;
        const int32_t start = min(s.barg - int32_t(P.delta >> 1), hi - int32_t(P.delta) + 1);
        lo = max(lo, start);
        hi = lo + int32_t(P.delta) - 1;
    }
    int32_t slo = lo - ib, shi = hi - ib;
    bool refresh = false;
    if (slo < 1 || shi > C - 2) {
        // one guard slot each side holds the gap predecessors of the band's end cells
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
        refresh = true;
    }
    // residue slices: slot t pairs H_side[ib - 1 + t] with V_side[d - ib - 1 - t]; the H
    // slice moves on even d, the V slice on odd d
    if (!ODD || refresh) {
        const int64_t hpos = ib - 1;
        s.hs = s.side ? slice_bwd(P.store, P.n_words, s.h0 - hpos) : slice_fwd(P.store, P.n_words, s.h0 + hpos);
    }
    if (ODD || refresh) {
        const int64_t vpos = int64_t(d) - ib - 1;
        s.vs = s.side ? slice_fwd(P.store, P.n_words, s.v0 - vpos) : slice_bwd(P.store, P.n_words, s.v0 + vpos);
    }
    const uint32_t bm = (0xffffffffu >> (31 - shi)) & (0xffffffffu << slo);
    const int32_t thr = max(s.T - P.X, kDeadR);
    const uint64_t x = s.hs ^ s.vs;
    int32_t kmax = INT32_MIN;
    uint32_t lm = 0;
#pragma unroll
    for (int t = 0; t < C; t++) {
        const int32_t up = ODD ? (t > 0 ? P1[t - 1] : kNegR) : P1[t];
        const int32_t lf = ODD ? P1[t] : (t < C - 1 ? P1[t + 1] : kNegR);
        const int32_t sig = ((x >> (2 * t)) & 3ull) ? mis : mat;
        const int32_t raw = __viaddmax_s32(max(up, lf), P.gap, P2[t] + sig);
        const bool live = raw >= thr && ((bm >> t) & 1u);
        const int32_t v = live ? raw : kNegR;
        P2[t] = v;
        lm |= live ? (1u << t) : 0u;
        kmax = max(kmax, v * 64 + (63 - t));
    }
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

template <int C>
__global__ void __launch_bounds__(128, 4) k_narrow(Problem P, Queues Q, int chunk) {
    extern __shared__ int32_t shift_smem[];
    int32_t* shbuf = shift_smem + threadIdx.x;
    const int stride = blockDim.x;
    const int32_t mat = P.sim[0], mis = P.sim[1];
    int32_t A[C], B[C];
    NarrowState s{};
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
                if ((int64_t(u.m) + u.n) * P.max_abs >= kRegLimit) {
                    Q.q2[atomicAdd(&Q.ctr[3], 1u)] = uidx;
                    continue;
                }
                if (P.alpha != 4) {
                    Q.q1[atomicAdd(&Q.ctr[1], 1u)] = uidx;
                    continue;
                }
                s.h0 = int64_t(u.h0);
                s.v0 = int64_t(u.v0);
                s.m = int32_t(u.m);
                s.n = int32_t(u.n);
                s.side = u.side;
                pair = u.pair;
                got = true;
                break;
            }
            if (!got) break;
            // S(0,0) = 0 in the middle of the window, every other cell -inf (Sec. 2.2)
#pragma unroll
            for (int t = 0; t < C; t++) {
                A[t] = kNegR;
                B[t] = kNegR;
            }
            A[C / 2] = 0;
            s.rb = -C / 2;
            s.d = 1;
            s.L = s.U = 0;
            s.T = s.best = s.bi = s.bj = s.barg = 0;
            s.flags = 0;
            s.cells = 1;
            s.hs = s.vs = 0;
            active = s.m + s.n > 0;
            if (!active) {
                write_side(P.results, pair, s.side, 0, 0, 0, 0, 1);
                atomicAdd(&P.stats[0], 1ull);
                atomicAdd(&P.stats[4], 1ull);
                continue;
            }
            // the first (odd) step loads the V slice; the H slice of d = 1 starts at ib - 1
            const int64_t hpos = s.rb - 1;
            s.hs = s.side ? slice_bwd(P.store, P.n_words, s.h0 - hpos) : slice_fwd(P.store, P.n_words, s.h0 + hpos);
        }
        int r = narrow_step<C, true>(s, A, B, P, mat, mis, shbuf, stride);
        if (r == kCont) r = narrow_step<C, false>(s, B, A, P, mat, mis, shbuf, stride);
        if (r == kCont) continue;
        active = false;
        if (r == kDone) {
            write_side(P.results, pair, s.side, s.best, uint32_t(s.bi), uint32_t(s.bj), s.flags, s.cells);
            atomicAdd(&P.stats[0], 1ull);
            atomicAdd(&P.stats[4], (unsigned long long)s.cells);
        } else {
            Q.q1[atomicAdd(&Q.ctr[1], 1u)] = uidx;
            atomicAdd(&P.stats[3], 1ull);
            atomicAdd(&P.stats[7], (unsigned long long)s.cells);
        }
    }
}

// Tier 1 placeholder: forwards every escalated unit to the generic tier.
__global__ void k_forward_q1(Queues Q) {
    const uint32_t n1 = Q.ctr[1];
    const uint32_t base = Q.ctr[3];
    for (uint32_t t = threadIdx.x; t < n1; t += blockDim.x) Q.q2[base + t] = Q.q1[t];
    __syncthreads();
    if (threadIdx.x == 0) Q.ctr[3] = base + n1;
}

cudaError_t launch_narrow(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    constexpr int C = 32;
    const size_t smem = size_t(2) * C * cfg.narrow_threads * sizeof(int32_t);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_narrow<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_narrow<C><<<cfg.narrow_blocks, cfg.narrow_threads, smem, st>>>(P, Q, cfg.chunk);
    return cudaGetLastError();
}

cudaError_t launch_wide(const Problem& P, const Queues& Q, const TierConfig& cfg, cudaStream_t st) {
    (void)P;
    (void)cfg;
    k_forward_q1<<<1, 256, 0, st>>>(Q);
    return cudaGetLastError();
}

}  // namespace xd
