// The plain anti-diagonal sweep of one side extension with one warp, rows in global
// memory: shared by the generic tier (xd_kernels.cu, packed store) and the
// allocation-free entry point (xd_noalloc.cu, unpacked codes), which differ only in how a
// cell's similarity is fetched.
//
// Per anti-diagonal d (Sec. 3, Algorithm 1): the band [lo, hi] is [first live, last live
// + 1] of d-1 clipped to the matrix and, when restricted, to delta_b cells centred on
// d-1's best cell; each cell takes the recurrence of Sec. 2.2 and the X-Drop test against
// T of the completed anti-diagonals; then warp reductions of the first / last live cell and
// of the best cell (lowest i on ties).  The three rows hold d-2, d-1 and d, indexed by i
// (capacity m + 1 each).
#pragma once
#include <cstdint>
#include "xd_device.cuh"

namespace xd {

struct SweepOut {
    int32_t best;
    int64_t bi, bj;
    uint32_t flags;
    uint64_t cells;
};

// sim_at(i, j), i, j >= 1: Sim(H_side[i-1], V_side[j-1]).
// zdrop > 0: the Z-Drop rule after each anti-diagonal (flag bit 1 when it ends the side).
template <class SimAt>
__device__ __forceinline__ SweepOut generic_sweep(int64_t m, int64_t n, int32_t gap, int32_t X, uint32_t delta,
                                                  int32_t zdrop, SimAt sim_at, int32_t* A, int32_t* B, int32_t* Cc,
                                                  int lane) {
    int32_t* P1 = A;
    int32_t* P2 = B;
    int32_t* C = Cc;
    int64_t p1lo = 0, p1hi = 0, p2lo = 1, p2hi = 0;
    if (lane == 0) P1[0] = 0;
    __syncwarp();
    SweepOut o{0, 0, 0, 0u, 1};
    int32_t T = 0;
    int64_t L = 0, U = 0, prev_arg = 0;
    for (int64_t d = 1; d <= m + n; d++) {
        int64_t lo = L, hi = U + 1;
        if (d - n > lo) lo = d - n;
        if (lo < 0) lo = 0;
        if (hi > m) hi = m;
        if (hi > d) hi = d;
        if (delta && hi - lo + 1 > int64_t(delta)) {
            o.flags = 1;
            int64_t start = prev_arg - int64_t(delta / 2);
            const int64_t latest = hi - int64_t(delta) + 1;
            if (latest < start) start = latest;
            if (start > lo) lo = start;
            hi = lo + int64_t(delta) - 1;
        }
        const int32_t thr = max(T - X, kDeadLine);
        int32_t first = INT32_MAX, last = -1, bmax = kNeg, barg = INT32_MAX;
        for (int64_t i = lo + lane; i <= hi; i += 32) {
            const int64_t j = d - i;
            int32_t c = kNeg;
            if (i >= 1 && j >= 1 && i - 1 >= p2lo && i - 1 <= p2hi) c = P2[i - 1] + sim_at(i, j);
            if (i >= 1 && i - 1 >= p1lo && i - 1 <= p1hi) c = max(c, P1[i - 1] + gap);
            if (j >= 1 && i >= p1lo && i <= p1hi) c = max(c, P1[i] + gap);
            if (c < thr) c = kNeg;
            C[i] = c;
            if (c != kNeg) {
                if (first == INT32_MAX) first = int32_t(i);
                last = int32_t(i);
                if (c > bmax) {
                    bmax = c;
                    barg = int32_t(i);
                }
            }
        }
        o.cells += uint64_t(hi - lo + 1);
        first = __reduce_min_sync(0xffffffffu, first);
        last = __reduce_max_sync(0xffffffffu, last);
        const int32_t wmax = __reduce_max_sync(0xffffffffu, bmax);
        barg = __reduce_min_sync(0xffffffffu, bmax == wmax ? barg : INT32_MAX);
        __syncwarp();
        if (first == INT32_MAX) break;
        if (wmax > T) {
            T = wmax;
            o.best = wmax;
            o.bi = barg;
            o.bj = d - barg;
        }
        prev_arg = barg;
        if (zdrop > 0) {
            const int64_t shift = llabs((int64_t(barg) - o.bi) - ((d - barg) - o.bj));
            if (int64_t(o.best) - wmax > int64_t(zdrop) + int64_t(-gap) * shift) {
                o.flags |= 2u;
                break;
            }
        }
        L = first;
        U = last;
        int32_t* old = P2;
        P2 = P1;
        p2lo = p1lo;
        p2hi = p1hi;
        P1 = C;
        p1lo = lo;
        p1hi = hi;
        C = old;
    }
    return o;
}

}  // namespace xd
