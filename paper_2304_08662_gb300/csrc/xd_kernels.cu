// Device pipeline of one batch: pack -> work units -> cost ordering -> tier kernels ->
// pair totals.  The alignment tiers live in xd_tiers.cu; this file holds the
// bandwidth-bound preparation kernels and the generic (any band width) tier.
#include <cstdint>
#include <cuda_runtime.h>
#include "xd_device.cuh"
#include "xd_launch.h"
#include "xd_sweep.cuh"

namespace xd {

// ---------------------------------------------------------------------------------------
// a1: sequence store.  The caller's residue codes (one byte each) are packed in place of
// their flat position: DNA 2 bits (16 per 32-bit word), protein 5 bits (6 per word).
// One thread per output word; codes outside the alphabet raise kErrCode.
__global__ void k_pack_dna(const uint8_t* __restrict__ codes, uint64_t n_codes,
                           uint32_t* __restrict__ store, uint64_t n_words, uint32_t* err) {
    uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    bool aligned = (reinterpret_cast<uintptr_t>(codes) & 15u) == 0;
    for (; w < n_words; w += stride) {
        uint64_t base = w * 16;
        uint32_t word = 0, bad = 0;
        if (aligned && base + 16 <= n_codes) {
            uint4 q = __ldg(reinterpret_cast<const uint4*>(codes + base));
            uint32_t parts[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int p = 0; p < 4; p++) {
                uint32_t x = parts[p];
                bad |= x & 0xFCFCFCFCu;
#pragma unroll
                for (int b = 0; b < 4; b++) word |= ((x >> (8 * b)) & 3u) << (2 * (4 * p + b));
            }
        } else {
            for (int t = 0; t < 16 && base + t < n_codes; t++) {
                uint32_t c = codes[base + t];
                bad |= c & ~3u;
                word |= (c & 3u) << (2 * t);
            }
        }
        store[w] = word;
        if (bad) atomicOr(err, kErrCode);
    }
}

__global__ void k_pack_prot(const uint8_t* __restrict__ codes, uint64_t n_codes,
                            uint32_t* __restrict__ store, uint64_t n_words, uint32_t* err) {
    uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (; w < n_words; w += stride) {
        uint64_t base = w * 6;
        uint32_t word = 0;
        bool bad = false;
        for (int t = 0; t < 6 && base + t < n_codes; t++) {
            uint32_t c = codes[base + t];
            bad |= c >= 20u;
            word |= (c & 31u) << (5 * t);
        }
        store[w] = word;
        if (bad) atomicOr(err, kErrCode);
    }
}

// ---------------------------------------------------------------------------------------
// a2: work units.  Each pair gives a right and a left unit (Sec. 4.1.2).  Units run longest
// first.  The cost proxy is the anti-diagonal count rather than the quadratic maximum work
// m * n of Sec. 4.2: an X-Drop side's work is its band times its anti-diagonals, and its
// latency (the serial chain that bounds a batch's makespan) is its anti-diagonal count,
// about 2 min(m, n) when the alignment runs to the end of the shorter sequence.  Buckets are
// quarter octaves of min(m, n) + 1.  Invalid tuples raise kErrSeed and become empty units;
// sides whose scores could leave the exact range raise kErrRange and also become empty.
// n_res: residues of the batch; a sequence whose offset + length passes it is invalid.
// Several batches can share one launch: batch-local pair p becomes pair pair_base + p (units
// 2 (pair_base + p) and + 1), and its residues start at res_base in the shared store.
__device__ __forceinline__ uint32_t cost_bucket(uint32_t m, uint32_t n) {
    const uint32_t s = min(m, n) + 1u;
    const uint32_t lg = 31u - uint32_t(__clz(s));               // floor(log2 s)
    const uint32_t frac = lg >= 2 ? (s >> (lg - 2)) & 3u : 0u;  // next two bits
    return min(4u * lg + frac, 63u);                             // 0 .. 63
}

__global__ void k_units(const xd_pair* __restrict__ pairs, uint32_t n_pairs,
                        const uint64_t* __restrict__ offsets, const uint32_t* __restrict__ lengths,
                        uint32_t n_seqs, uint64_t n_res, int32_t max_abs, uint32_t max_len,
                        uint32_t pair_base, uint64_t res_base,
                        Unit* __restrict__ units, uint32_t* __restrict__ bucket_of,
                        uint32_t* __restrict__ hist, uint32_t* err) {
    __shared__ uint32_t sh[64];
    for (int t = threadIdx.x; t < 64; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pairs) {
        xd_pair e = pairs[p];
        uint32_t bad = 0;
        uint64_t ho = 0, vo = 0;
        uint32_t lh = 0, lv = 0;
        if (e.h_id >= n_seqs || e.v_id >= n_seqs) {
            bad = kErrSeed;
        } else {
            ho = offsets[e.h_id]; vo = offsets[e.v_id];
            lh = lengths[e.h_id]; lv = lengths[e.v_id];
            // a seed outside its sequence, or a sequence past the end of the residues
            if (uint64_t(e.h_seed) + e.seed_len > lh || uint64_t(e.v_seed) + e.seed_len > lv ||
                ho + lh > n_res || vo + lv > n_res)
                bad = kErrSeed;
        }
        Unit r{}, l{};
        r.pair = l.pair = pair_base + p;
        ho += res_base;
        vo += res_base;
        r.side = 0; l.side = 1;
        if (!bad) {
            r.h0 = ho + e.h_seed + e.seed_len; r.m = lh - e.h_seed - e.seed_len;
            r.v0 = vo + e.v_seed + e.seed_len; r.n = lv - e.v_seed - e.seed_len;
            l.h0 = e.h_seed ? ho + e.h_seed - 1 : ho; l.m = e.h_seed;
            l.v0 = e.v_seed ? vo + e.v_seed - 1 : vo; l.n = e.v_seed;
            uint32_t range = 0;
            if ((int64_t(r.m) + r.n) * max_abs >= kScoreLimit || r.m > max_len) { r.m = r.n = 0; range = kErrRange; }
            if ((int64_t(l.m) + l.n) * max_abs >= kScoreLimit || l.m > max_len) { l.m = l.n = 0; range = kErrRange; }
            bad |= range;
        }
        if (bad) atomicOr(err, bad);
        const uint32_t u = 2 * (pair_base + p);
        units[u] = r;
        units[u + 1] = l;
        uint32_t br = cost_bucket(r.m, r.n), bl = cost_bucket(l.m, l.n);
        bucket_of[u] = br;
        bucket_of[u + 1] = bl;
        atomicAdd(&sh[br], 1u);
        atomicAdd(&sh[bl], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 64; t += blockDim.x)
        if (sh[t]) atomicAdd(&hist[t], sh[t]);
}

// One block: exclusive offsets of the cost buckets in descending cost order; resets the
// queue counters of the batch.
__global__ void k_bucket_scan(uint32_t* hist, uint32_t* ctr, int n_ctr) {
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 63; b >= 0; b--) {
            uint32_t c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    for (int t = threadIdx.x; t < n_ctr; t += blockDim.x) ctr[t] = 0;
}

__global__ void k_bucket_scatter(const uint32_t* __restrict__ bucket_of, uint32_t n_units,
                                 uint32_t* hist_pos, uint32_t* __restrict__ order) {
    uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_units) order[atomicAdd(&hist_pos[bucket_of[u]], 1u)] = u;
}

// ---------------------------------------------------------------------------------------
// Generic tier: one warp per unit, the three anti-diagonals in a global-memory ring
// indexed by i (capacity max_m + 1 per array), any band width.  It is the fallback for
// units whose band does not fit the register tiers.  The step follows the method
// directly: band [lo, hi] from the previous anti-diagonal (Algorithm 1), optional
// delta_b window centred on the previous anti-diagonal's best cell, the recurrence of
// Sec. 2.2, the X-Drop test against T of completed anti-diagonals, then warp
// reductions of first/last live cell and of the best cell (lowest i on ties).
__device__ __forceinline__ int32_t sim_of(const int32_t* sim, int alpha, uint32_t a, uint32_t b) {
    return sim[a * alpha + b];
}

__device__ void extend_generic(const Problem& P, const Unit& u, int32_t* A, int32_t* B,
                               int32_t* Cc, const int32_t* sim, int lane) {
    const int64_t dir = u.side ? -1 : 1;
    auto sim_at = [&](int64_t i, int64_t j) {
        const uint32_t a = residue(P.store, P.alpha, u.h0 + dir * (i - 1));
        const uint32_t b = residue(P.store, P.alpha, u.v0 + dir * (j - 1));
        return sim_of(sim, P.alpha, a, b);
    };
    const SweepOut o = generic_sweep(int64_t(u.m), int64_t(u.n), P.gap, P.X, P.delta, P.zdrop, sim_at, A, B, Cc,
                                     lane);
    if (lane == 0) {
        write_side(P.results, u.pair, u.side, o.best, uint32_t(o.bi), uint32_t(o.bj), o.flags, o.cells);
        atomicAdd(&P.stats[2], 1ull);
        atomicAdd(&P.stats[6], (unsigned long long)o.cells);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(128) k_generic(Problem P, Queues Q, int32_t* scratch,
                                                 uint64_t stride) {
    __shared__ int32_t sim[400];
    for (int t = threadIdx.x; t < P.alpha * P.alpha; t += blockDim.x) sim[t] = P.sim[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
    int32_t* A = scratch + warp * 3 * stride;
    constexpr int G = kGenericQ;
    const uint32_t n_q = *reinterpret_cast<volatile uint32_t*>(&Q.ctr[1 + 2 * G]);
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&Q.ctr[2 + 2 * G], 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n_q) break;
        const uint32_t uidx = Q.q[G][k];
        const Unit u = P.units[uidx];
        const unsigned long long t0 = P.trace ? trace_clock() : 0ull;
        extend_generic(P, u, A, A + stride, A + 2 * stride, sim, lane);
        if (P.trace && lane == 0) trace_visit(P, uidx, kTraceGeneric, t0, 0, 0, 32, 1);
    }
}


// ---------------------------------------------------------------------------------------
// Band tier: NW warps (a block) per side extension, the two previous anti-diagonals in a
// shared memory ring of kBandW slots per row.  Slot s of anti-diagonal d is cell
// i = floor(d/2) + rb + s (the register tiers' layout: the diagonal predecessor is the same
// slot of row d-2, the gap predecessors slots s-1, s (odd d) or s, s+1 (even d) of row
// d-1); slot s lives at ring position (s + base) mod kBandW, so re-centring the window
// only moves base and clears the slots it exposes.  Each anti-diagonal is swept over its
// band only, 32 NW cells at a time; the new anti-diagonal overwrites row d-2 in place, and
// the two slots just outside the band are set to -inf so that the next two anti-diagonals
// read correct neighbours.  The live range and the best cell are reduced per warp, then
// across the block through a double-buffered shared array (one barrier per anti-diagonal).
// Sides reach this tier when their band outgrows every register window (a few very wide
// bands, whose anti-diagonals a whole block shares).  Takes DNA and protein, any band up
// to kBandW - 2 cells, and continues sides from escalation records of the register levels.
constexpr int kBandW = 8192;
constexpr int kBandWarps = 8;

template <int NW>
__device__ __forceinline__ void band_sync() {
    if constexpr (NW == 1) __syncwarp();
    else __syncthreads();
}

__device__ __forceinline__ int32_t band_load_rec(const Problem& P, uint32_t ri, int32_t* R0, int32_t* R1,
                                                 int32_t& rb, int64_t& d, int32_t& L, int32_t& U, int32_t& T,
                                                 int32_t& best, int64_t& bi, int64_t& bj, int64_t& barg,
                                                 uint32_t& flags, uint64_t& cells, int tid, int nt) {
    const int32_t* r = P.rec + ri;
    const int32_t w0 = __ldcg(r + 0);
    const int32_t off = (kBandW - w0) / 2;
    d = __ldcg(r + 1);
    rb = __ldcg(r + 2) - off;
    L = __ldcg(r + 3);
    U = __ldcg(r + 4);
    T = __ldcg(r + 5);
    best = __ldcg(r + 6);
    bi = __ldcg(r + 7);
    bj = __ldcg(r + 8);
    barg = __ldcg(r + 9);
    flags = uint32_t(__ldcg(r + 10));
    cells = uint64_t(uint32_t(__ldcg(r + 11))) | (uint64_t(uint32_t(__ldcg(r + 12))) << 32);
    // record rows: d-1 then d-2, slots 0 .. w0-1
    for (int s = tid; s < w0; s += nt) {
        R0[s + off] = __ldcg(r + 16 + s);
        R1[s + off] = __ldcg(r + 16 + w0 + s);
    }
    return w0;
}

// Returns false when the band outgrew the ring (the side then goes to the generic tier).
// red: 8 NW ints of shared memory for the block reductions.
template <int NW>
__device__ bool extend_band(const Problem& P, const Unit& u, uint32_t uidx, int32_t* R0, int32_t* R1,
                            const int32_t* sim, int32_t* red, int tid) {
    constexpr int W = kBandW;
    constexpr int NT = 32 * NW;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t m = u.m, n = u.n;
    const int64_t dir = u.side ? -1 : 1;
    for (int s = tid; s < W; s += NT) {
        R0[s] = kNeg;
        R1[s] = kNeg;
    }
    band_sync<NW>();
    int32_t* P1 = R0;       // anti-diagonal d-1
    int32_t* P2 = R1;       // anti-diagonal d-2, overwritten by d
    int32_t rb = -W / 2, T = 0, best = 0, L = 0, U = 0;
    int64_t d = 1, bi = 0, bj = 0, barg = 0;
    uint32_t flags = 0, base = 0;
    uint64_t cells = 1;
    const uint32_t ri = P.rec_of ? __ldcg(P.rec_of + uidx) : 0xffffffffu;
    if (ri != 0xffffffffu && __ldcg(P.rec + ri) <= W) {
        band_load_rec(P, ri, R0, R1, rb, d, L, U, T, best, bi, bj, barg, flags, cells, tid, NT);
    } else if (tid == 0) {
        P1[W / 2] = 0;      // S(0,0) = 0 at d = 0 (slot W/2)
    }
    band_sync<NW>();
    const int32_t g = P.gap;
    for (; d <= m + n; d++) {
        int64_t lo = L, hi = int64_t(U) + 1;
        if (d - n > lo) lo = d - n;
        if (lo < 0) lo = 0;
        if (hi > m) hi = m;
        if (hi > d) hi = d;
        if (P.delta && hi - lo + 1 > int64_t(P.delta)) {
            flags |= 1u;
            int64_t start = barg - int64_t(P.delta / 2);
            const int64_t latest = hi - int64_t(P.delta) + 1;
            if (latest < start) start = latest;
            if (start > lo) lo = start;
            hi = lo + int64_t(P.delta) - 1;
        }
        int64_t ib = (d >> 1) + rb;
        int64_t slo = lo - ib, shi = hi - ib;
        if (slo < 1 || shi > W - 2) {
            const int64_t w = hi - lo + 1;
            if (w > W - 2) return false;
            const int64_t k = slo - (1 + (W - 2 - w) / 2);
            // new slot s = old slot s + k: move the ring base, clear the exposed slots
            base = uint32_t((int64_t(base) + k) & (W - 1));
            rb += int32_t(k);
            ib += k;
            slo -= k;
            shi -= k;
            const int64_t ak = k > 0 ? k : -k;
            const int64_t from = ak >= W ? 0 : (k > 0 ? W - k : 0);
            const int64_t cnt = ak >= W ? W : ak;
            for (int64_t t = tid; t < cnt; t += NT) {
                const uint32_t pos = uint32_t((from + t + base) & (W - 1));
                P1[pos] = kNeg;
                P2[pos] = kNeg;
            }
            band_sync<NW>();
        }
        const int32_t thr = max(T - P.X, kDeadLine);
        const bool odd = d & 1;
        int32_t first = INT32_MAX, last = -1, bmax = kNeg, bslot = INT32_MAX;
        for (int64_t s0 = slo; s0 <= shi; s0 += NT) {
            const int64_t s = s0 + tid;
            if (s <= shi) {
                const int64_t i = ib + s, j = d - i;
                const uint32_t ps = uint32_t((s + base) & (W - 1));
                const uint32_t pa = uint32_t((s - 1 + base) & (W - 1)), pb = uint32_t((s + 1 + base) & (W - 1));
                const int32_t up = odd ? P1[pa] : P1[ps];
                const int32_t lf = odd ? P1[ps] : P1[pb];
                int32_t c = max(up, lf) + g;
                if (i >= 1 && j >= 1) {
                    const uint32_t a = residue(P.store, P.alpha, uint64_t(int64_t(u.h0) + dir * (i - 1)));
                    const uint32_t b = residue(P.store, P.alpha, uint64_t(int64_t(u.v0) + dir * (j - 1)));
                    c = max(c, P2[ps] + sim[a * P.alpha + b]);
                }
                if (c < thr) c = kNeg;
                P2[ps] = c;
                if (c != kNeg) {
                    if (first == INT32_MAX) first = int32_t(s);
                    last = int32_t(s);
                    if (c > bmax) {
                        bmax = c;
                        bslot = int32_t(s);
                    }
                }
            }
        }
        if (tid == 0) {
            P2[uint32_t((slo - 1 + base) & (W - 1))] = kNeg;
            P2[uint32_t((shi + 1 + base) & (W - 1))] = kNeg;
        }
        cells += uint64_t(hi - lo + 1);
        first = __reduce_min_sync(0xffffffffu, first);
        last = __reduce_max_sync(0xffffffffu, last);
        int32_t wmax = __reduce_max_sync(0xffffffffu, bmax);
        bslot = __reduce_min_sync(0xffffffffu, bmax == wmax ? bslot : INT32_MAX);
        if constexpr (NW > 1) {
            // across the block: this anti-diagonal's half of the double buffer
            int32_t* rd = red + (d & 1) * 4 * NW;
            if (lane == 0) {
                rd[warp] = first;
                rd[NW + warp] = last;
                rd[2 * NW + warp] = wmax;
                rd[3 * NW + warp] = bslot;
            }
            __syncthreads();
            first = INT32_MAX;
            last = -1;
            wmax = kNeg;
            bslot = INT32_MAX;
#pragma unroll
            for (int w = 0; w < NW; w++) {
                first = min(first, rd[w]);
                last = max(last, rd[NW + w]);
                const int32_t v = rd[2 * NW + w];
                if (v > wmax) {
                    wmax = v;
                    bslot = rd[3 * NW + w];
                } else if (v == wmax) {
                    bslot = min(bslot, rd[3 * NW + w]);
                }
            }
        } else {
            __syncwarp();
        }
        if (first == INT32_MAX) break;
        const int64_t arg = ib + bslot;
        if (wmax > T) {
            T = wmax;
            best = wmax;
            bi = arg;
            bj = d - arg;
        }
        barg = arg;
        if (P.zdrop > 0) {
            // Z-Drop: the anti-diagonal's best cell against the best so far
            const int64_t shift = llabs((arg - bi) - ((d - arg) - bj));
            if (int64_t(best) - wmax > int64_t(P.zdrop) + int64_t(-P.gap) * shift) {
                flags |= 2u;
                break;
            }
        }
        L = int32_t(ib + first);
        U = int32_t(ib + last);
        int32_t* tmp = P2;
        P2 = P1;
        P1 = tmp;
    }
    if (tid == 0) {
        write_side(P.results, u.pair, u.side, best, uint32_t(bi), uint32_t(bj), flags, cells);
        atomicAdd(&P.stats[1], 1ull);
        atomicAdd(&P.stats[5], (unsigned long long)cells);
    }
    band_sync<NW>();
    return true;
}

template <int NW>
__global__ void __launch_bounds__(32 * NW) k_band(Problem P, Queues Q) {
    extern __shared__ int32_t band_smem[];
    int32_t* sim = band_smem;
    int32_t* red = band_smem + 400;                 // 8 NW ints (NW <= 2: within the pad)
    int32_t* R0 = band_smem + 416 + (NW > 2 ? 8 * NW : 0);
    int32_t* R1 = R0 + kBandW;
    __shared__ uint32_t take;
    const int tid = threadIdx.x;
    for (int t = tid; t < P.alpha * P.alpha; t += blockDim.x) sim[t] = P.sim[t];
    if (NW > 2) red = band_smem + 416;
    band_sync<NW>();
    const uint32_t n_q = *reinterpret_cast<volatile uint32_t*>(&Q.ctr[1 + 2 * kBandQ]);
    for (;;) {
        uint32_t k = 0;
        if constexpr (NW == 1) {
            if (tid == 0) k = atomicAdd(&Q.ctr[2 + 2 * kBandQ], 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
        } else {
            if (tid == 0) take = atomicAdd(&Q.ctr[2 + 2 * kBandQ], 1u);
            __syncthreads();
            k = take;
            __syncthreads();
        }
        if (k >= n_q) break;
        const uint32_t uidx = Q.q[kBandQ][k];
        const Unit u = P.units[uidx];
        const unsigned long long t0 = P.trace ? trace_clock() : 0ull;
        const bool fit = extend_band<NW>(P, u, uidx, R0, R1, sim, red, tid);
        if (P.trace && tid == 0) trace_visit(P, uidx, kTraceBand, t0, 0, kBandW, 32 * NW / 8, fit ? 1 : 2);
        if (!fit) {
            if (tid == 0) {
                push_unit(Q, kGenericQ, uidx);
                atomicAdd(&P.stats[3], 1ull);
            }
            band_sync<NW>();
        }
    }
}

// Queue every unit to the generic tier (used when the register tiers are disabled).
__global__ void k_route_all_generic(Queues Q) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < Q.n_units) Q.q[kGenericQ][t] = Q.order[t];
    if (t == 0) Q.ctr[1 + 2 * kGenericQ] = Q.n_units;
}

// ---------------------------------------------------------------------------------------
// a9: pair totals = left + right + sum of Sim over the seed.
__global__ void k_totals(const xd_pair* __restrict__ pairs, uint32_t n_pairs,
                         const uint64_t* __restrict__ offsets, const uint32_t* __restrict__ lengths,
                         uint32_t n_seqs, uint64_t n_res, uint32_t pair_base, uint64_t res_base, Problem P) {
    __shared__ int32_t sim[400];
    for (int t = threadIdx.x; t < P.alpha * P.alpha; t += blockDim.x) sim[t] = P.sim[t];
    __syncthreads();
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    xd_pair e = pairs[p];
    int64_t seed = 0;
    if (e.h_id < n_seqs && e.v_id < n_seqs) {
        uint64_t ho = res_base + offsets[e.h_id] + e.h_seed, vo = res_base + offsets[e.v_id] + e.v_seed;
        // only tuples that k_units accepted: the seed inside its sequence, the sequence
        // inside the store
        if (uint64_t(e.h_seed) + e.seed_len <= lengths[e.h_id] &&
            uint64_t(e.v_seed) + e.seed_len <= lengths[e.v_id] &&
            offsets[e.h_id] + lengths[e.h_id] <= n_res && offsets[e.v_id] + lengths[e.v_id] <= n_res)
            for (uint32_t t = 0; t < e.seed_len; t++)
                seed += sim[residue(P.store, P.alpha, ho + t) * P.alpha + residue(P.store, P.alpha, vo + t)];
    }
    xd_result& r = P.results[pair_base + p];
    r.total = int64_t(r.left.score) + int64_t(r.right.score) + seed;
}

// Adds the per-batch counters into the context's cumulative ones.
__global__ void k_accumulate(const unsigned long long* batch, unsigned long long* total, int n) {
    int t = threadIdx.x;
    if (t < n) total[t] += batch[t];
}

// ---------------------------------------------------------------------------------------
// Host-side launchers.

static int grid_for(uint64_t n, int block, int max_blocks) {
    uint64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > uint64_t(max_blocks)) g = max_blocks;
    return int(g);
}

cudaError_t launch_pack(int alpha, const uint8_t* codes, uint64_t n_codes, uint32_t* store,
                        uint32_t* err, int n_sm, cudaStream_t st) {
    uint64_t per = alpha == 4 ? 16 : 6;
    uint64_t n_words = (n_codes + per - 1) / per;
    if (n_words == 0) return cudaSuccess;
    int grid = grid_for(n_words, 256, n_sm * 16);
    if (alpha == 4) k_pack_dna<<<grid, 256, 0, st>>>(codes, n_codes, store, n_words, err);
    else k_pack_prot<<<grid, 256, 0, st>>>(codes, n_codes, store, n_words, err);
    return cudaGetLastError();
}

cudaError_t launch_units(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                         const uint32_t* lengths, uint32_t n_seqs, uint64_t n_res, int32_t max_abs,
                         uint32_t max_len, uint32_t pair_base, uint64_t res_base, Unit* units,
                         uint32_t* bucket_of, uint32_t* hist, uint32_t* err, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    k_units<<<(n_pairs + 255) / 256, 256, 0, st>>>(pairs, n_pairs, offsets, lengths, n_seqs, n_res,
                                                   max_abs, max_len, pair_base, res_base, units,
                                                   bucket_of, hist, err);
    return cudaGetLastError();
}

cudaError_t launch_order(uint32_t* hist, uint32_t* ctr, int n_ctr, const uint32_t* bucket_of,
                         uint32_t n_units, uint32_t* order, cudaStream_t st) {
    k_bucket_scan<<<1, 32, 0, st>>>(hist, ctr, n_ctr);
    if (n_units)
        k_bucket_scatter<<<(n_units + 255) / 256, 256, 0, st>>>(bucket_of, n_units, hist, order);
    return cudaGetLastError();
}

cudaError_t launch_route_all_generic(const Queues& Q, cudaStream_t st) {
    k_route_all_generic<<<(Q.n_units + 255) / 256 + 1, 256, 0, st>>>(Q);
    return cudaGetLastError();
}

cudaError_t launch_generic(const Problem& P, const Queues& Q, int32_t* scratch,
                           uint64_t stride, int n_blocks, cudaStream_t st) {
    k_generic<<<n_blocks, 128, 0, st>>>(P, Q, scratch, stride);
    return cudaGetLastError();
}

template <int NW>
static cudaError_t launch_band_nw(const Problem& P, const Queues& Q, int n_sm, cudaStream_t st) {
    const size_t smem = (416 + 8 * NW + 2 * size_t(kBandW)) * sizeof(int32_t);
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_band<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_band<NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band<NW>, 32 * NW, smem);
        if (e != cudaSuccess) return e;
        per_sm = per_sm < 1 ? 1 : per_sm;
    }
    // blocks that pull sides from the band queue: as many as fit (the queue decides the work)
    k_band<NW><<<n_sm * per_sm, 32 * NW, smem, st>>>(P, Q);
    return cudaGetLastError();
}

cudaError_t launch_band(const Problem& P, const Queues& Q, int n_sm, int nw, cudaStream_t st) {
    switch (nw) {
        case 1: return launch_band_nw<1>(P, Q, n_sm, st);
        case 2: return launch_band_nw<2>(P, Q, n_sm, st);
        case 4: return launch_band_nw<4>(P, Q, n_sm, st);
        case 16: return launch_band_nw<16>(P, Q, n_sm, st);
        case 32: return launch_band_nw<32>(P, Q, n_sm, st);
        default: return launch_band_nw<kBandWarps>(P, Q, n_sm, st);
    }
}

cudaError_t launch_totals(const xd_pair* pairs, uint32_t n_pairs, const uint64_t* offsets,
                          const uint32_t* lengths, uint32_t n_seqs, uint64_t n_res, uint32_t pair_base,
                          uint64_t res_base, const Problem& P, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    k_totals<<<(n_pairs + 255) / 256, 256, 0, st>>>(pairs, n_pairs, offsets, lengths, n_seqs, n_res,
                                                    pair_base, res_base, P);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const unsigned long long* batch, unsigned long long* total, int n,
                              cudaStream_t st) {
    k_accumulate<<<1, 32, 0, st>>>(batch, total, n);
    return cudaGetLastError();
}

}  // namespace xd
