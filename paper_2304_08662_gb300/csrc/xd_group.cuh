// Register tiers of the X-Drop library: one templated group kernel.
//
// A side extension is owned by a group of G lanes (G = 1 .. 32); lane l of the group holds
// slots [l*CG, (l+1)*CG) of a window of W = G*CG slots per anti-diagonal.  Slot s of
// anti-diagonal d holds cell i = floor(d/2) + rb + s.  In these coordinates the diagonal
// predecessor S(i-1, j-1) sits in the same slot two anti-diagonals back and the two gap
// predecessors sit in slots (s-1, s) on odd d and (s, s+1) on even d, so a band that
// follows the main diagonal does not move in the window; it drifts only with the indels of
// the alignment.  The window is re-centred through shared memory when the band nears its
// edge (one guard slot on each side holds the gap predecessors of the band's end cells).
// A side whose band outgrows the window is appended to the next level's queue with an
// escalation record and continued there in a wider window.  The two anti-diagonals are
// the paper's memory-restricted pair (Gotoh's two-diagonal scheme, Sec. 3): the new
// anti-diagonal overwrites d-2 slot by slot.
//
// Per anti-diagonal (Sec. 3, Algorithm 1): band [first live, last live + 1] of d-1 clipped
// to the matrix and, when restricted, to delta_b cells centred on d-1's best cell; per cell
// the recurrence of Sec. 2.2 as max(S(i-1,j-1) + Sim, max(S(i-1,j), S(i,j-1)) + gap) with
// the DPX add-max, the X-Drop test against T of the completed anti-diagonals; then group
// reductions of the live range and of the best cell (lowest i on ties).
//
// Scores: the template argument A selects the representation, 32-bit slots (A = 4 DNA,
// A = 20 protein: group_step, cells_of) or 16-bit packed slots, two per register (A =
// kDna16, kProt16: group_step16, cells16), described with kDna16 below.
//
// Residues: each lane keeps slices of H and V for its slots (2-bit fields for DNA; for
// protein, 16-bit table offsets, two slots per register).  On odd d the V slice gains one
// residue, on even d the H slice does; residues come from two oriented streams per lane
// whose next store word is always prefetched.
//
// This header holds the templates; xd_tiers.cu instantiates the fused grids,
// xd_tiers_dna.cu / xd_tiers_dna16.cu the DNA level kernels (32-bit / packed) and
// xd_tiers_prot.cu / xd_tiers_prot16.cu the protein ones.
#pragma once
#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "xd_device.cuh"
#include "xd_launch.h"

namespace xd {

// Register levels keep scores in a narrower range so that a (score, slot) key fits 32 bits.
constexpr int32_t kNegR = -(1 << 24);
constexpr int32_t kDeadR = -(1 << 23);
constexpr int64_t kRegLimit = int64_t(1) << 23;

// ---------------------------------------------------------------------------------------
// 16-bit packed scores: representations kDna16 (DNA) and kProt16 (protein) of the group
// kernels (template argument A).
//
// Register p of a lane holds slot p in its low half and slot p + CG/2 in its high half, so
// one 16x2 DPX instruction updates two cells.  A score S of anti-diagonal d is kept as 32 z
// with z = S - (B0 + gap * d).  With the base falling by |gap| per anti-diagonal, the gap
// predecessors (d-1) need no adjustment and the diagonal one (d-2) gains the constant
// -2 gap, which the similarity table already holds: the cell of Sec. 2.2 becomes
// max(max(up, left), diag + 32 (Sim - 2 gap)), two instructions for two cells.  The low
// five bits of a live slot are zero, so one add-max of 31 - slot per register yields the
// best cell of the lane together with its lowest slot (ties: lowest i).  The X-Drop
// threshold T - X of anti-diagonal d sits at z = theta_d; theta starts at theta0 and grows
// by |gap| per anti-diagonal plus the growth of T, and every slot is rebased once theta
// passes theta1.  Dead cells hold -1 (all ones): anything computed from them stays below
// 32 theta, and the live test is the sign of the slot minus 32 theta.
//   theta0 = 2 (|gap| + s_max) + 1: a dead slot plus 32 (Sim - 2 gap) stays below
//            32 theta, and live slots stay positive across a rebase;
//   theta1 = 1022 - X - s_max: live z <= theta + X + s_max, so 32 z + 31 < 2^15.
// A batch takes these levels when theta1 - theta0 >= 64 and -127 <= gap <= 0 (DNA scores
// 1 / -1 / -1: X <= 952; BLOSUM62 with gap -2: X <= 920); other batches take the 32-bit
// levels.
constexpr int kDna16 = 2;
constexpr int kProt16 = 3;
constexpr uint32_t kDead2 = 0xffffffffu;

__host__ __device__ constexpr int alpha_of(int A) { return A == kDna16 ? 4 : A == kProt16 ? 20 : A; }
__host__ __device__ constexpr bool packed_rep(int A) { return A == kDna16 || A == kProt16; }

struct Z16 {
    int32_t th0, th1;
};
__host__ __device__ inline Z16 z16_of(const Problem& P) {
    return Z16{2 * (P.s_max - P.gap) + 1, 1022 - P.X - P.s_max};
}
__host__ __device__ inline bool packed_ok(const Problem& P) {
    if (P.gap > 0 || P.gap < -127 || P.X < 0 || P.X > 1022 || P.s_max < 0 || P.s_max > 127) return false;
    const Z16 z = z16_of(P);
    return z.th1 - z.th0 >= 64;
}

enum { kCont = 0, kDone = 1, kOverflow = 2 };

__device__ __forceinline__ uint32_t ld_word(const uint32_t* store, uint64_t n_words, int64_t w) {
    w = w < 0 ? 0 : w;
    w = w >= int64_t(n_words) ? int64_t(n_words) - 1 : w;
    return __ldg(store + w);
}

// 32 residues from position p: field f (bits 2f, 2f+1) = residue p + f, or p + 31 - f
// when rev.  Positions outside the store read clamped words (only cells outside the band
// ever use them).
__device__ __forceinline__ uint64_t slice_at(const uint32_t* store, uint64_t nw, int64_t p, bool rev) {
    const int64_t w = p >> 4;
    const uint32_t sh = uint32_t(p & 15) * 2u;
    const uint64_t lo = (uint64_t(ld_word(store, nw, w + 1)) << 32) | ld_word(store, nw, w);
    const uint64_t hi = ld_word(store, nw, w + 2);
    uint64_t x = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
    if (rev) {
        x = __brevll(x);
        x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    }
    return x;
}

// Oriented residue stream: next() returns store[p], store[p + dir], store[p + 2 dir], ...
struct Stream {
    int64_t word;      // index of cur
    uint32_t cur, nxt; // current word and the following one (prefetched)
    int32_t off;       // bit offset of the next residue in cur
    int32_t dir;       // +1 or -1
};

__device__ __forceinline__ void stream_init(Stream& s, const uint32_t* store, uint64_t nw, int64_t p, int32_t dir) {
    s.word = p >> 4;
    s.off = int32_t(p & 15) * 2;
    s.dir = dir;
    s.cur = ld_word(store, nw, s.word);
    s.nxt = ld_word(store, nw, s.word + dir);
}

__device__ __forceinline__ uint32_t stream_next(Stream& s, const uint32_t* store, uint64_t nw) {
    const uint32_t c = (s.cur >> s.off) & 3u;
    s.off += 2 * s.dir;
    if (s.off < 0 || s.off > 30) {
        s.word += s.dir;
        s.cur = s.nxt;
        s.nxt = ld_word(store, nw, s.word + s.dir);
        s.off &= 31;
    }
    return c;
}

// Protein residue stream over the 5-bit store (six residues per word, residue k of a word
// in bits 5k .. 5k+4).
struct Stream5 {
    int64_t word;
    uint32_t cur, nxt;
    int32_t off;
    int32_t dir;
};

__device__ __forceinline__ void stream5_init(Stream5& s, const uint32_t* store, uint64_t nw, int64_t p, int32_t dir) {
    const int64_t w = p >= 0 ? p / 6 : -((-p + 5) / 6);   // floor(p / 6)
    s.word = w;
    s.off = int32_t(p - 6 * w) * 5;
    s.dir = dir;
    s.cur = ld_word(store, nw, w);
    s.nxt = ld_word(store, nw, w + dir);
}

__device__ __forceinline__ uint32_t stream5_next(Stream5& s, const uint32_t* store, uint64_t nw) {
    const uint32_t c = (s.cur >> s.off) & 31u;
    s.off += 5 * s.dir;
    if (s.off < 0 || s.off > 25) {
        s.word += s.dir;
        s.cur = s.nxt;
        s.off = s.dir > 0 ? 0 : 25;
    }
    // the next word is re-read on every call, by every lane at once: a load issued only by
    // the lanes that cross a word boundary would leave the register pending for the whole
    // warp until it returns (re-read words hit L1; measured faster for protein, not for DNA)
    s.nxt = ld_word(store, nw, s.word + s.dir);
    return c;
}

// Per-side state, replicated across the lanes of a group (the residue slices live in Res).
struct SideState {
    int64_t h0, v0;
    uint64_t cells;
    int32_t m, n, d, rb, dir;
    int32_t L, U, T, best, bi, bj, barg;
    int32_t B0;                 // kDna16: z = S - (B0 + gap d)
    uint32_t flags, side;
    bool refresh;
};

__device__ __forceinline__ void init_side(SideState& s, const Unit& u, int32_t rb) {
    s.h0 = int64_t(u.h0);
    s.v0 = int64_t(u.v0);
    s.m = int32_t(u.m);
    s.n = int32_t(u.n);
    s.side = u.side;
    s.dir = u.side ? -1 : 1;
    s.rb = rb;
    s.d = 1;
    s.L = s.U = 0;
    s.T = s.best = s.bi = s.bj = s.barg = 0;
    s.flags = 0;
    s.cells = 1;
    s.refresh = true;
}

// Residue slices of a lane's CG slots: slot t pairs H_side[hb + t] with V_side[vb - t],
// where H_side[k] = store[h0 + dir k] (likewise V).
template <int CG, int A>
struct Res;

// DNA: 2-bit fields of one 64-bit word per sequence.
template <int CG>
struct Res<CG, 4> {
    uint64_t hs, vs;
    Stream sh, sv;              // next residue entering the H / V slice

    __device__ __forceinline__ void load(const Problem& P, const SideState& s, int64_t hb, int64_t vb) {
        hs = s.dir > 0 ? slice_at(P.store, P.n_words, s.h0 + hb, false)
                       : slice_at(P.store, P.n_words, s.h0 - hb - 31, true);
        if constexpr (CG < 32) hs &= (1ull << (2 * CG)) - 1ull;   // fields >= CG stay zero while shifting
        vs = s.dir > 0 ? slice_at(P.store, P.n_words, s.v0 + vb - 31, true)
                       : slice_at(P.store, P.n_words, s.v0 - vb, false);
        stream_init(sh, P.store, P.n_words, s.h0 + s.dir * (hb + CG), s.dir);
        stream_init(sv, P.store, P.n_words, s.v0 + s.dir * (vb + 1), s.dir);
    }
    __device__ __forceinline__ void push_h(const Problem& P) {
        const uint64_t c = stream_next(sh, P.store, P.n_words);
        hs = (hs >> 2) | (c << (2 * (CG - 1)));
    }
    __device__ __forceinline__ void push_v(const Problem& P) {
        const uint64_t c = stream_next(sv, P.store, P.n_words);
        vs = (vs << 2) | c;
    }
};

// Protein: byte offsets into the 20 x 20 int32 similarity table in shared memory, H codes
// scaled by 80 and V codes by 4, two slots per register (slot 2k in the low half).  The
// sum of an H and a V register is the table offset of both slots' cells at once (no carry
// crosses the halves: 31 * 80 + 31 * 4 < 2^16).
template <int CG>
struct Res<CG, 20> {
    uint32_t hx[CG / 2], vx[CG / 2];
    Stream5 sh, sv;

    __device__ __forceinline__ void load(const Problem& P, const SideState& s, int64_t hb, int64_t vb) {
        Stream5 t;
        stream5_init(t, P.store, P.n_words, s.h0 + s.dir * hb, s.dir);
#pragma unroll
        for (int k = 0; k < CG / 2; k++) {
            const uint32_t lo = stream5_next(t, P.store, P.n_words) * 80u;
            const uint32_t hi = stream5_next(t, P.store, P.n_words) * 80u;
            hx[k] = lo | (hi << 16);
        }
        // V_side[vb - CG + 1 .. vb] in side order fills the slots from CG - 1 down to 0
        stream5_init(t, P.store, P.n_words, s.v0 + s.dir * (vb - CG + 1), s.dir);
#pragma unroll
        for (int k = CG / 2 - 1; k >= 0; k--) {
            const uint32_t hi = stream5_next(t, P.store, P.n_words) * 4u;
            const uint32_t lo = stream5_next(t, P.store, P.n_words) * 4u;
            vx[k] = lo | (hi << 16);
        }
        stream5_init(sh, P.store, P.n_words, s.h0 + s.dir * (hb + CG), s.dir);
        stream5_init(sv, P.store, P.n_words, s.v0 + s.dir * (vb + 1), s.dir);
    }
    __device__ __forceinline__ void push_h(const Problem& P) {
        const uint32_t c = stream5_next(sh, P.store, P.n_words) * 80u;
#pragma unroll
        for (int k = 0; k < CG / 2 - 1; k++) hx[k] = __funnelshift_r(hx[k], hx[k + 1], 16);
        hx[CG / 2 - 1] = (hx[CG / 2 - 1] >> 16) | (c << 16);
    }
    __device__ __forceinline__ void push_v(const Problem& P) {
        const uint32_t c = stream5_next(sv, P.store, P.n_words) * 4u;
#pragma unroll
        for (int k = CG / 2 - 1; k > 0; k--) vx[k] = __funnelshift_l(vx[k - 1], vx[k], 16);
        vx[0] = (vx[0] << 16) | c;
    }
};

template <int CG, bool ODD, int A>
__device__ __forceinline__ void update_slices(SideState& s, Res<CG, A>& r, const Problem& P, int64_t hb,
                                              int64_t vb) {
    if (s.refresh) {
        r.load(P, s, hb, vb);
        s.refresh = false;
    } else if (!ODD) {
        r.push_h(P);
    } else {
        r.push_v(P);
    }
}

// Band [lo, hi] of anti-diagonal d: [first live, last live + 1] of d-1 clipped to the
// matrix, then to delta_b cells centred on d-1's best cell when restricted.
__device__ __forceinline__ void band_of(SideState& s, const Problem& P, int32_t d, int32_t& lo, int32_t& hi) {
    lo = max(max(s.L, d - s.n), 0);
    hi = min(min(s.U + 1, s.m), d);
    if (P.delta && hi - lo + 1 > int32_t(P.delta)) {
        s.flags |= 1u;
        const int32_t start = min(s.barg - int32_t(P.delta >> 1), hi - int32_t(P.delta) + 1);
        lo = max(lo, start);
        hi = lo + int32_t(P.delta) - 1;
    }
}

// Z-Drop (z > 0; Sec. 1 names the variant, minimap2's definition): after anti-diagonal d,
// whose best live cell is (arg, d - arg) with score wmax, the side stops when the best cell so
// far beats it by more than Z + |gap| times the difference of their diagonals.
__device__ __forceinline__ bool zdrop_stops(const Problem& P, const SideState& s, int32_t wmax, int32_t arg,
                                            int32_t d) {
    const int32_t shift = abs((arg - s.bi) - ((d - arg) - s.bj));
    return int64_t(s.best) - wmax > int64_t(P.zdrop) + int64_t(-P.gap) * shift;
}

// The lane's CG cells.  P1 holds d-1, P2 holds d-2 and receives d.  upb / lfb are the
// neighbours beyond the lane's first / last slot.  tab is the block's similarity table:
// for DNA 256 int4 entries indexed by one byte of the xor of the residue slices (four
// 2-bit fields, zero = match), giving four cells' Sim per load; for protein the 20 x 20
// int32 matrix addressed by the slices' summed byte offsets.  Returns the lane's live mask
// and the maximum key v * 64 + (63 - t) over its cells (dead cells hold kNegR).
template <int CG, bool ODD, int A>
__device__ __forceinline__ void cells_of(int32_t (&P1)[CG], int32_t (&P2)[CG], int32_t upb,
                                         int32_t lfb, const Res<CG, A>& res, uint32_t bm, int32_t thr,
                                         int32_t gap, const int32_t* tab, int32_t& kmax,
                                         uint32_t& lm) {
    static_assert(CG % 4 == 0, "cells come in groups of four");
    kmax = INT32_MIN;
    lm = 0;
#pragma unroll
    for (int q = 0; q < CG / 4; q++) {
        int32_t sg[4];
        if constexpr (A == 4) {
            const uint64_t x = res.hs ^ res.vs;
            const int4 s4 = reinterpret_cast<const int4*>(tab)[uint32_t(x >> (8 * q)) & 0xffu];
            sg[0] = s4.x;
            sg[1] = s4.y;
            sg[2] = s4.z;
            sg[3] = s4.w;
        } else {
            const char* tb = reinterpret_cast<const char*>(tab);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t ix = res.hx[2 * q + h] + res.vx[2 * q + h];
                sg[2 * h] = *reinterpret_cast<const int32_t*>(tb + (ix & 0xffffu));
                sg[2 * h + 1] = *reinterpret_cast<const int32_t*>(tb + (ix >> 16));
            }
        }
        int32_t key[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int t = 4 * q + r;
            const int32_t up = ODD ? (t > 0 ? P1[t - 1] : upb) : P1[t];
            const int32_t lf = ODD ? P1[t] : (t < CG - 1 ? P1[t + 1] : lfb);
            const int32_t raw = __viaddmax_s32(max(up, lf), gap, P2[t] + sg[r]);
            const bool live = raw >= thr && ((bm >> t) & 1u);
            const int32_t v = live ? raw : kNegR;
            P2[t] = v;
            lm |= live ? (1u << t) : 0u;
            key[r] = v * 64 + (63 - t);
        }
        kmax = __vimax3_s32(kmax, key[0], key[1]);
        kmax = __vimax3_s32(kmax, key[2], key[3]);
    }
}

// The block's similarity table at the start of its shared memory.  DNA: entry e holds Sim of
// the four fields (e >> 2f) & 3, f = 0..3 (zero = match).  Protein: Sim row-major, H code
// major.  Entries past the 20 x 20 matrix are zero (offsets of codes >= 20 land there; only
// cells outside the band can carry such codes).
__device__ __forceinline__ void build_table16(int32_t* tab, const Problem& P);
__device__ __forceinline__ void build_table_p16(int32_t* tab, const Problem& P);

template <int A>
__device__ __forceinline__ void build_table(int32_t* tab, const Problem& P) {
    if constexpr (A == kDna16) {
        build_table16(tab, P);
        return;
    } else if constexpr (A == kProt16) {
        build_table_p16(tab, P);
        return;
    } else if constexpr (A == 4) {
        const int32_t mat = P.sim[0], mis = P.sim[1];
        for (int e = threadIdx.x; e < 256; e += blockDim.x) {
            int4 v;
            v.x = (e & 3) ? mis : mat;
            v.y = ((e >> 2) & 3) ? mis : mat;
            v.z = ((e >> 4) & 3) ? mis : mat;
            v.w = ((e >> 6) & 3) ? mis : mat;
            reinterpret_cast<int4*>(tab)[e] = v;
        }
    } else {
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) tab[e] = e < 400 ? int32_t(P.sim[e]) : 0;
    }
    __syncthreads();
}
constexpr int kLutInts = 1024;


// 2-bit field k of the low 32 bits -> bits 4k, 4k + 1.
__device__ __forceinline__ uint64_t spread2(uint64_t s) {
    s = (s | (s << 16)) & 0x0000FFFF0000FFFFull;
    s = (s | (s << 8)) & 0x00FF00FF00FF00FFull;
    s = (s | (s << 4)) & 0x0F0F0F0F0F0F0F0Full;
    s = (s | (s << 2)) & 0x3333333333333333ull;
    return s;
}

// Both halves of a register to all ones where negative, zeros elsewhere (byte permute in
// sign-replicate mode).
__device__ __forceinline__ uint32_t sign_spread(uint32_t u) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %1, 0xBB99;" : "=r"(r) : "r"(u));
    return r;
}

__device__ __forceinline__ uint32_t pack2(int32_t lo, int32_t hi) {
    return (uint32_t(lo) & 0xffffu) | (uint32_t(hi) << 16);
}
__device__ __forceinline__ int32_t lo16(uint32_t v) { return int32_t(int16_t(uint16_t(v & 0xffffu))); }
__device__ __forceinline__ int32_t hi16(uint32_t v) { return int32_t(v) >> 16; }

// DNA residue slices in the register order of kDna16: the field of slot t < CG/2 at bits
// 4t, 4t + 1, that of slot CG/2 + t at bits 4t + 2, 4t + 3, so that byte q of the xor of H
// and V covers registers 2q and 2q + 1.
template <int CG>
struct Res<CG, kDna16> {
    static constexpr int H = CG / 2;
    uint64_t hs, vs;
    Stream sh, sv;

    __device__ __forceinline__ static uint64_t interleave(uint64_t x) {
        const uint64_t m = H == 16 ? 0xffffffffull : ((1ull << (2 * H)) - 1ull);
        return spread2(x & m) | (spread2((x >> (2 * H)) & m) << 2);
    }
    __device__ __forceinline__ void load(const Problem& P, const SideState& s, int64_t hb, int64_t vb) {
        const uint64_t h = s.dir > 0 ? slice_at(P.store, P.n_words, s.h0 + hb, false)
                                     : slice_at(P.store, P.n_words, s.h0 - hb - 31, true);
        const uint64_t v = s.dir > 0 ? slice_at(P.store, P.n_words, s.v0 + vb - 31, true)
                                     : slice_at(P.store, P.n_words, s.v0 - vb, false);
        hs = interleave(h);
        vs = interleave(v);
        stream_init(sh, P.store, P.n_words, s.h0 + s.dir * (hb + CG), s.dir);
        stream_init(sv, P.store, P.n_words, s.v0 + s.dir * (vb + 1), s.dir);
    }
    // slots move down by one, the new residue enters slot CG - 1
    __device__ __forceinline__ void push_h(const Problem& P) {
        const uint64_t c = stream_next(sh, P.store, P.n_words);
        hs = (hs >> 4) | (((hs >> 2) & 3ull) << (4 * (H - 1))) | (c << (4 * (H - 1) + 2));
    }
    // slots move up by one, the new residue enters slot 0
    __device__ __forceinline__ void push_v(const Problem& P) {
        const uint64_t c = stream_next(sv, P.store, P.n_words);
        const uint64_t m = H == 16 ? ~0ull : ((1ull << (4 * H)) - 1ull);
        vs = ((vs << 4) & m) | (((vs >> (4 * (H - 1))) & 3ull) << 2) | c;
    }
};

// The block's table for kDna16: 256 int2 entries; entry e holds 32 (Sim - 2 gap) of the
// four 2-bit fields of e (zero = match), fields 0 / 1 in .x (low / high half), 2 / 3 in .y.
__device__ __forceinline__ void build_table16(int32_t* tab, const Problem& P) {
    const int32_t mat = 32 * (P.sim[0] - 2 * P.gap), mis = 32 * (P.sim[1] - 2 * P.gap);
    for (int e = threadIdx.x; e < 256; e += blockDim.x) {
        const int32_t f0 = (e & 3) ? mis : mat, f1 = ((e >> 2) & 3) ? mis : mat;
        const int32_t f2 = ((e >> 4) & 3) ? mis : mat, f3 = ((e >> 6) & 3) ? mis : mat;
        tab[2 * e] = int32_t(pack2(f0, f1));
        tab[2 * e + 1] = int32_t(pack2(f2, f3));
    }
    __syncthreads();
}

// Protein residue slices in the register order of kProt16: byte offsets into the block's
// 20 x 20 table, slot p in the low half and slot CG/2 + p in the high half (H codes scaled
// by 80, V codes by 4); the sum of an H and a V register addresses both slots' cells.
template <int CG>
struct Res<CG, kProt16> {
    static constexpr int H = CG / 2;
    uint32_t hx[H], vx[H];
    Stream5 sh, sv;

    __device__ __forceinline__ void load(const Problem& P, const SideState& s, int64_t hb, int64_t vb) {
        Stream5 t;
        // slot u pairs H_side[hb + u] with V_side[vb - u]
        stream5_init(t, P.store, P.n_words, s.h0 + s.dir * hb, s.dir);
#pragma unroll
        for (int u = 0; u < CG; u++) {
            const uint32_t c = stream5_next(t, P.store, P.n_words) * 80u;
            if (u < H) hx[u] = c;
            else hx[u - H] |= c << 16;
        }
        stream5_init(t, P.store, P.n_words, s.v0 + s.dir * (vb - CG + 1), s.dir);
#pragma unroll
        for (int u = CG - 1; u >= 0; u--) {
            const uint32_t c = stream5_next(t, P.store, P.n_words) * 4u;
            if (u >= H) vx[u - H] = c << 16;
            else vx[u] |= c;
        }
        stream5_init(sh, P.store, P.n_words, s.h0 + s.dir * (hb + CG), s.dir);
        stream5_init(sv, P.store, P.n_words, s.v0 + s.dir * (vb + 1), s.dir);
    }
    // slots move down by one, the new residue enters slot CG - 1
    __device__ __forceinline__ void push_h(const Problem& P) {
        const uint32_t c = stream5_next(sh, P.store, P.n_words) * 80u;
        const uint32_t s0 = hx[0] >> 16;
#pragma unroll
        for (int p = 0; p < H - 1; p++) hx[p] = hx[p + 1];
        hx[H - 1] = s0 | (c << 16);
    }
    // slots move up by one, the new residue enters slot 0
    __device__ __forceinline__ void push_v(const Problem& P) {
        const uint32_t c = stream5_next(sv, P.store, P.n_words) * 4u;
        const uint32_t sh1 = vx[H - 1] & 0xffffu;
#pragma unroll
        for (int p = H - 1; p > 0; p--) vx[p] = vx[p - 1];
        vx[0] = c | (sh1 << 16);
    }
};

// The block's table for kProt16: 32 (Sim - 2 gap) row-major, H code major (byte offset
// 80 h + 4 v); entries past the 20 x 20 matrix are zero (only cells outside the band can
// carry codes >= 20).
__device__ __forceinline__ void build_table_p16(int32_t* tab, const Problem& P) {
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) tab[e] = e < 400 ? 32 * (int32_t(P.sim[e]) - 2 * P.gap) : 0;
    __syncthreads();
}

// The lane's CG cells in kDna16 / kProt16.  P1 holds d-1, P2 holds d-2 and receives d; upb / lfb are
// the neighbouring lanes' registers holding the slot before the first / after the last
// (kDead2 at the group's ends).  nbv: slots outside the band, slot p at bit p and slot
// CG/2 + p at bit 16 + p.  nth2: -32 theta in both halves.  Returns the packed maximum of
// slot + 31 - lane slot over the new slots (the lane's best cell and its lowest slot; at
// most 30 when none is live) and the dead mask in the layout of nbv.
template <int CG, bool ODD, int A>
__device__ __forceinline__ void cells16(uint32_t (&P1)[CG / 2], uint32_t (&P2)[CG / 2], uint32_t upb,
                                        uint32_t lfb, const Res<CG, A>& res, uint32_t nbv, uint32_t nth2,
                                        const int32_t* tab, uint32_t& mk, uint32_t& dacc) {
    constexpr int H = CG / 2;
    static_assert(CG % 4 == 0 && H <= 16, "slots come in pairs of registers");
    mk = kDead2;
    dacc = 0;
#pragma unroll
    for (int q = 0; q < H / 2; q++) {
        uint32_t sp[2];
        if constexpr (A == kDna16) {
            const uint64_t x = res.hs ^ res.vs;
            const int2 s2 = reinterpret_cast<const int2*>(tab)[uint32_t(x >> (8 * q)) & 0xffu];
            sp[0] = uint32_t(s2.x);
            sp[1] = uint32_t(s2.y);
        } else {
            const char* tb = reinterpret_cast<const char*>(tab);
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const uint32_t ix = res.hx[2 * q + r] + res.vx[2 * q + r];
                const uint32_t a = *reinterpret_cast<const uint32_t*>(tb + (ix & 0xffffu));
                const uint32_t b = *reinterpret_cast<const uint32_t*>(tb + (ix >> 16));
                sp[r] = __byte_perm(a, b, 0x5410);
            }
        }
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int p = 2 * q + r;
            uint32_t up, lf;
            if (ODD) {
                up = p > 0 ? P1[p - 1] : __byte_perm(upb, P1[H - 1], 0x5432);
                lf = P1[p];
            } else {
                up = P1[p];
                lf = p < H - 1 ? P1[p + 1] : __byte_perm(P1[0], lfb, 0x5432);
            }
            const uint32_t raw = __viaddmax_s16x2(P2[p], sp[r], __vmaxs2(up, lf));
            uint32_t u = __viaddmax_s16x2(raw, nth2, 0x80008000u);   // raw - 32 theta
            u |= (nbv << (15 - p)) & 0x80008000u;                   // outside the band: negative
            const uint32_t M = sign_spread(u);
            const uint32_t v = raw | M;
            P2[p] = v;
            dacc |= M & ((1u << p) | (1u << (16 + p)));
            const uint32_t key = uint32_t(31 - p) | (uint32_t(31 - p - H) << 16);
            mk = __viaddmax_s16x2(v, key, mk);
        }
    }
}

template <int G>
__device__ __forceinline__ int32_t gmax(int32_t v, uint32_t gm) {
    if constexpr (G == 32) {
        return __reduce_max_sync(0xffffffffu, v);
    } else {
#pragma unroll
        for (int k = G / 2; k >= 1; k >>= 1) v = max(v, __shfl_xor_sync(gm, v, k));
        return v;
    }
}

template <int G>
__device__ __forceinline__ int32_t gmin(int32_t v, uint32_t gm) {
    if constexpr (G == 32) {
        return __reduce_min_sync(0xffffffffu, v);
    } else {
#pragma unroll
        for (int k = G / 2; k >= 1; k >>= 1) v = min(v, __shfl_xor_sync(gm, v, k));
        return v;
    }
}

__device__ __forceinline__ uint32_t slot_mask(int32_t from, int32_t to, int cw) {
    const int32_t a = max(from, 0), b = min(to + 1, cw);
    if (a >= b) return 0u;
    return uint32_t(((1ull << b) - 1ull) & ~((1ull << a) - 1ull));
}

// One anti-diagonal of the group's side extension.
template <int G, int CG, bool ODD, int A>
__device__ __forceinline__ int group_step(SideState& s, Res<CG, A>& res, int32_t (&P1)[CG], int32_t (&P2)[CG],
                                          const Problem& P, const int32_t* tab, int gl,
                                          uint32_t gm, int32_t* gsm) {
    constexpr int W = G * CG;
    const int32_t d = s.d;
    int32_t ib = (d >> 1) + s.rb;
    int32_t lo, hi;
    band_of(s, P, d, lo, hi);
    int32_t slo = lo - ib, shi = hi - ib;
    if (slo < 1 || shi > W - 2) {
        const int32_t w = hi - lo + 1;
        if (w > W - 2) return kOverflow;
        const int32_t k = slo - (1 + (W - 2 - w) / 2);
        // re-centre: every lane parks its slots in the group's shared row and reads back
        // the slots k positions further
#pragma unroll
        for (int t = 0; t < CG; t++) {
            gsm[gl * CG + t] = P1[t];
            gsm[W + gl * CG + t] = P2[t];
        }
        if (G > 1) __syncwarp(gm);
#pragma unroll
        for (int t = 0; t < CG; t++) {
            const int src = gl * CG + t + k;
            const bool in = src >= 0 && src < W;
            P1[t] = in ? gsm[src] : kNegR;
            P2[t] = in ? gsm[W + src] : kNegR;
        }
        if (G > 1) __syncwarp(gm);
        s.rb += k;
        ib += k;
        slo -= k;
        shi -= k;
        s.refresh = true;
        if (gl == 0) atomicAdd(&P.stats[8], 1ull);
    }
    const int32_t sb = gl * CG;
    update_slices<CG, ODD, A>(s, res, P, int64_t(ib) - 1 + sb, int64_t(d) - ib - 1 - sb);
    const uint32_t bm = slot_mask(slo - sb, shi - sb, CG);
    const int32_t thr = max(s.T - P.X, kDeadR);
    int32_t upb = kNegR, lfb = kNegR;
    if (G > 1) {
        if (ODD) {
            upb = __shfl_up_sync(gm, P1[CG - 1], 1, G);
            if (gl == 0) upb = kNegR;
        } else {
            lfb = __shfl_down_sync(gm, P1[0], 1, G);
            if (gl == G - 1) lfb = kNegR;
        }
    }
    int32_t kmax;
    uint32_t lm;
    cells_of<CG, ODD, A>(P1, P2, upb, lfb, res, bm, thr, P.gap, tab, kmax, lm);
    s.cells += uint64_t(hi - lo + 1);
    const bool any = lm != 0;
    int32_t first = any ? sb + __ffs(lm) - 1 : INT32_MAX;
    int32_t last = any ? sb + 31 - __clz(lm) : -1;
    first = gmin<G>(first, gm);
    if (first == INT32_MAX) return kDone;
    last = gmax<G>(last, gm);
    const int32_t lv = kmax >> 6;
    const int32_t wmax = gmax<G>(lv, gm);
    const int32_t arg = ib + gmin<G>(lv == wmax ? sb + (63 - (kmax & 63)) : INT32_MAX, gm);
    s.L = ib + first;
    s.U = ib + last;
    if (wmax > s.T) {
        s.T = wmax;
        s.best = wmax;
        s.bi = arg;
        s.bj = d - arg;
    }
    s.barg = arg;
    s.d = d + 1;
    if (P.zdrop > 0 && zdrop_stops(P, s, wmax, arg, d)) {
        s.flags |= 2u;
        return kDone;
    }
    return d == s.m + s.n ? kDone : kCont;
}

// One anti-diagonal of the group's side extension in kDna16 / kProt16 (the steps of
// group_step, on packed scores).
template <int G, int CG, bool ODD, int A>
__device__ __forceinline__ int group_step16(SideState& s, Res<CG, A>& res, uint32_t (&P1)[CG / 2],
                                            uint32_t (&P2)[CG / 2], const Problem& P, const Z16& zc,
                                            const int32_t* tab, int gl, uint32_t gm, int32_t* gsm) {
    constexpr int W = G * CG, H = CG / 2;
    const int32_t d = s.d;
    int32_t ib = (d >> 1) + s.rb;
    int32_t lo, hi;
    band_of(s, P, d, lo, hi);
    int32_t slo = lo - ib, shi = hi - ib;
    if (slo < 1 || shi > W - 2) {
        const int32_t w = hi - lo + 1;
        if (w > W - 2) return kOverflow;
        const int32_t k = slo - (1 + (W - 2 - w) / 2);
        // re-centre through the group's shared row, one int per slot in slot order
#pragma unroll
        for (int p = 0; p < H; p++) {
            gsm[gl * CG + p] = lo16(P1[p]);
            gsm[gl * CG + H + p] = hi16(P1[p]);
            gsm[W + gl * CG + p] = lo16(P2[p]);
            gsm[W + gl * CG + H + p] = hi16(P2[p]);
        }
        if (G > 1) __syncwarp(gm);
#pragma unroll
        for (int p = 0; p < H; p++) {
            const int a = gl * CG + p + k, b = a + H;
            const bool ia = a >= 0 && a < W, ibb = b >= 0 && b < W;
            P1[p] = pack2(ia ? gsm[a] : -1, ibb ? gsm[b] : -1);
            P2[p] = pack2(ia ? gsm[W + a] : -1, ibb ? gsm[W + b] : -1);
        }
        if (G > 1) __syncwarp(gm);
        s.rb += k;
        ib += k;
        slo -= k;
        shi -= k;
        s.refresh = true;
        if (gl == 0) atomicAdd(&P.stats[8], 1ull);
    }
    const int32_t sb = gl * CG;
    update_slices<CG, ODD, A>(s, res, P, int64_t(ib) - 1 + sb, int64_t(d) - ib - 1 - sb);
    const uint32_t nb = ~slot_mask(slo - sb, shi - sb, CG);
    const uint32_t nbv = H == 16 ? nb : ((nb & ((1u << H) - 1u)) | ((nb >> H) << 16));
    int32_t zb = s.B0 + P.gap * d;
    int32_t theta = s.T - P.X - zb;
    if (theta > zc.th1) {
        // rebase: every slot falls by 32 delta, dead slots stay at -1
        const int32_t delta = theta - zc.th0;
        const uint32_t nd2 = (uint32_t(-32 * delta) & 0xffffu) * 0x10001u;
#pragma unroll
        for (int p = 0; p < H; p++) {
            P1[p] = __viaddmax_s16x2(P1[p], nd2, kDead2);
            P2[p] = __viaddmax_s16x2(P2[p], nd2, kDead2);
        }
        s.B0 += delta;
        zb += delta;
        theta -= delta;
    }
    const uint32_t nth2 = (uint32_t(-32 * theta) & 0xffffu) * 0x10001u;
    uint32_t upb = kDead2, lfb = kDead2;
    if (G > 1) {
        if (ODD) {
            upb = __shfl_up_sync(gm, P1[H - 1], 1, G);
            if (gl == 0) upb = kDead2;
        } else {
            lfb = __shfl_down_sync(gm, P1[0], 1, G);
            if (gl == G - 1) lfb = kDead2;
        }
    }
    uint32_t mk, dacc;
    cells16<CG, ODD, A>(P1, P2, upb, lfb, res, nbv, nth2, tab, mk, dacc);
    s.cells += uint64_t(hi - lo + 1);
    const uint32_t hm = (1u << H) - 1u;
    const uint32_t lv = ~dacc & (hm * 0x10001u);
    const uint32_t lm = (lv & hm) | ((lv >> 16) << H);
    const bool any = lm != 0;
    int32_t first = any ? sb + __ffs(lm) - 1 : INT32_MAX;
    int32_t last = any ? sb + 31 - __clz(lm) : -1;
    if constexpr (G > 1 && G < 32) {
        // first and last live slot of the group in one shuffle tree of 16x2 maxima:
        // (last + 1, 0xffff - first), a lane without live slots contributing (0, 0)
        uint32_t fl = any ? (uint32_t(last + 1) << 16) | uint32_t(0xffff - first) : 0u;
#pragma unroll
        for (int k = G / 2; k >= 1; k >>= 1) fl = __vmaxu2(fl, __shfl_xor_sync(gm, fl, k));
        if ((fl & 0xffffu) == 0) return kDone;
        first = 0xffff - int32_t(fl & 0xffffu);
        last = int32_t(fl >> 16) - 1;
    } else {
        first = gmin<G>(first, gm);
        if (first == INT32_MAX) return kDone;
        last = gmax<G>(last, gm);
    }
    // best cell of the group: z, then 1023 - window slot (the lowest slot wins ties); a lane
    // without live slots has a lane key <= 30 and loses to every live one (z >= theta0 > 0)
    const int32_t kl = max(lo16(mk), hi16(mk));
    const int32_t gk = gmax<G>(((kl >> 5) << 10) | (1023 - (sb + 31 - (kl & 31))), gm);
    const int32_t wmax = (gk >> 10) + zb;
    const int32_t arg = ib + 1023 - (gk & 1023);
    s.L = ib + first;
    s.U = ib + last;
    if (wmax > s.T) {
        s.T = wmax;
        s.best = wmax;
        s.bi = arg;
        s.bj = d - arg;
    }
    s.barg = arg;
    s.d = d + 1;
    if (P.zdrop > 0 && zdrop_stops(P, s, wmax, arg, d)) {
        s.flags |= 2u;
        return kDone;
    }
    return d == s.m + s.n ? kDone : kCont;
}

// Where a group takes its next side extension from.  A static source is a finished list
// (the cost-ordered units, or a queue filled by an earlier launch).  A live source is a
// queue that producers of the same launch may still append to: slots are reserved with an
// atomic counter and published by storing the unit index over the kNoUnit sentinel.
constexpr uint32_t kNoUnit = 0xffffffffu;
constexpr uint64_t kWaitLimitNs = 10ull * 1000 * 1000 * 1000;   // default: 10 s without progress

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Source {
    const uint32_t* list;
    uint32_t* pull;             // pull counter
    uint32_t n;                 // length of a static source
    bool live;
    uint32_t* reserve;          // live: length counter
    uint32_t* producers_done;   // live: producer warps that have finished
    uint32_t n_producers;
    uint64_t wait_limit_ns;     // live: give up after this long without progress
};

// A consumer's wait on a live source (lane 0 of the group keeps it): its ticket, the queue
// words loaded by the previous poll, and the clock of its wait.  An idle group shares its
// warp's instruction stream with groups that still compute, so a poll never waits on
// memory: it decides on the values loaded by the poll before and issues the loads for the
// next.  (The zero start is a valid, if stale, snapshot.)
struct LiveWait {
    uint32_t ticket = kNoUnit;      // taken ticket (slot index of the queue), or kNoUnit
    uint32_t res = 0, pull = 0, fin = 0, slot = kNoUnit;
    uint32_t sig = 0xffffffffu;     // queue length and finished producers when last changed
    uint32_t t_us = 0;              // globaltimer (microseconds) of that change, 0 = not waiting
};

// Takes the group's next side extension from S without blocking (group-uniform result):
// 1 = uidx holds a unit, 0 = none yet (a live source whose producers still run, or a poll
// in progress), -1 = S is exhausted, or a live wait gave up after S.wait_limit_ns without
// progress (kErrWait).  `progress` is set when the poll took a ticket (the caller then does
// not back off).  LIVE: S is a live queue (else a finished list).
template <int G, bool LIVE>
__device__ __forceinline__ int take_unit(const Source& S, int gl, int lane, uint32_t gm, int chunk,
                                         uint32_t& next, uint32_t& end, uint32_t& uidx, LiveWait& lw,
                                         uint32_t* err, bool& progress) {
    if constexpr (!LIVE) {
        if (next >= end) {
            uint32_t base = 0;
            const uint32_t take = G == 1 ? uint32_t(chunk) : 1u;
            if (gl == 0) base = atomicAdd(S.pull, take);
            if (G > 1) base = __shfl_sync(gm, base, lane - gl);
            if (base >= S.n) return -1;
            next = base;
            end = min(base + take, S.n);
        }
        uidx = S.list[next++];
        return 1;
    }
    int st = 0;
    uint32_t u = kNoUnit;
    if (gl == 0) {
        // plain coherent loads (an idle consumer must not load L2 with atomics); a ticket is
        // taken only when the queue holds a slot nobody has taken
        const volatile uint32_t* reserve = S.reserve;
        const volatile uint32_t* pull = S.pull;
        const volatile uint32_t* done = S.producers_done;
        const volatile uint32_t* list = S.list;
        const uint32_t res = lw.res, fin = lw.fin;   // queue length known to this poll
        bool took = false;
        if (lw.ticket == kNoUnit) {
            if (lw.pull < res) {
                lw.ticket = atomicAdd(S.pull, 1u);   // its slot is loaded by the next poll
                took = true;
            }
        } else if (lw.ticket < res && lw.slot != kNoUnit) {
            u = lw.slot;   // the slot loaded by the previous poll, published
            st = 1;
            lw.ticket = kNoUnit;
            lw.t_us = 0;
        }
        if (st == 0 && !took) {
            if (fin >= S.n_producers) {
                // every producer has counted itself: the queue's length is final
                __threadfence();
                const uint32_t r2 = *reserve;
                if (lw.ticket == kNoUnit ? *pull >= r2 : lw.ticket >= r2) st = -1;
            }
            if (st == 0) {
                const uint32_t now = uint32_t(globaltimer_ns() >> 10);
                const uint32_t sig = res ^ (fin << 20);
                if (lw.t_us == 0 || sig != lw.sig) {
                    lw.sig = sig;
                    lw.t_us = now;
                } else if (uint64_t(now - lw.t_us) << 10 > S.wait_limit_ns) {
                    atomicOr(err, kErrWait);
                    st = -1;
                }
            }
        }
        if (took) lw.t_us = 0;
        progress = took;
        // loads for the next poll; the slot of a held ticket only once the ticket is below
        // a known queue length (tickets past it may lie beyond the queue)
        lw.slot = kNoUnit;
        if (!took && lw.ticket < res) lw.slot = list[lw.ticket];
        lw.res = *reserve;
        lw.pull = *pull;
        lw.fin = *done;
    }
    if (G > 1) {
        st = __shfl_sync(gm, st, lane - gl);
        u = __shfl_sync(gm, u, lane - gl);
        progress = __shfl_sync(gm, progress ? 1 : 0, lane - gl) != 0;
    }
    uidx = u;
    return st;
}

// Record layout: 16 header ints (window, d, rb, L, U, T, best, bi, bj, barg, flags,
// cells lo/hi), then the window's anti-diagonal d-1 and d-2 in slot order.  Records are
// bump-allocated from one int pool; rec_of holds a record's offset in the pool.
constexpr int kRecHeader = 16;

template <int G, int CG>
__device__ __forceinline__ void save_record(const Problem& P, uint32_t ri, const SideState& s,
                                            const int32_t (&P1)[CG], const int32_t (&P2)[CG], int gl) {
    constexpr int W = G * CG;
    int32_t* r = P.rec + ri;
#pragma unroll
    for (int t = 0; t < CG; t++) {
        __stcg(r + kRecHeader + gl * CG + t, P1[t]);
        __stcg(r + kRecHeader + W + gl * CG + t, P2[t]);
    }
    if (gl == 0) {
        __stcg(r + 0, W);
        __stcg(r + 1, s.d);
        __stcg(r + 2, s.rb);
        __stcg(r + 3, s.L);
        __stcg(r + 4, s.U);
        __stcg(r + 5, s.T);
        __stcg(r + 6, s.best);
        __stcg(r + 7, s.bi);
        __stcg(r + 8, s.bj);
        __stcg(r + 9, s.barg);
        __stcg(r + 10, int32_t(s.flags));
        __stcg(r + 11, int32_t(uint32_t(s.cells)));
        __stcg(r + 12, int32_t(uint32_t(s.cells >> 32)));
    }
}

// Continues a side from its record in a window of W >= the record's window (placed in the
// middle).  Returns false if the record does not fit (the side then starts from scratch).
template <int G, int CG>
__device__ __forceinline__ bool load_record(const Problem& P, uint32_t ri, SideState& s, int32_t (&A)[CG],
                                            int32_t (&B)[CG], int gl) {
    constexpr int W = G * CG;
    const int32_t* r = P.rec + ri;
    const int32_t w0 = __ldcg(r + 0);
    if (w0 > W) return false;
    const int32_t off = (W - w0) / 2;
    s.d = __ldcg(r + 1);
    s.rb = __ldcg(r + 2) - off;
    s.L = __ldcg(r + 3);
    s.U = __ldcg(r + 4);
    s.T = __ldcg(r + 5);
    s.best = __ldcg(r + 6);
    s.bi = __ldcg(r + 7);
    s.bj = __ldcg(r + 8);
    s.barg = __ldcg(r + 9);
    s.flags = uint32_t(__ldcg(r + 10));
    s.cells = uint64_t(uint32_t(__ldcg(r + 11))) | (uint64_t(uint32_t(__ldcg(r + 12))) << 32);
    const bool odd = s.d & 1;   // odd d: A holds d-1; even d: B holds d-1
#pragma unroll
    for (int t = 0; t < CG; t++) {
        const int src = gl * CG + t - off;
        const bool in = src >= 0 && src < w0;
        const int32_t v1 = in ? __ldcg(r + kRecHeader + src) : kNegR;
        const int32_t v2 = in ? __ldcg(r + kRecHeader + w0 + src) : kNegR;
        A[t] = odd ? v1 : v2;
        B[t] = odd ? v2 : v1;
    }
    return true;
}

// kDna16 records: the same layout, scores converted to and from S (dead slots: kNegR).
template <int G, int CG>
__device__ __forceinline__ void save_record16(const Problem& P, uint32_t ri, const SideState& s,
                                              const uint32_t (&P1)[CG / 2], const uint32_t (&P2)[CG / 2], int gl) {
    constexpr int W = G * CG, H = CG / 2;
    int32_t* r = P.rec + ri;
    const int32_t z1 = s.B0 + P.gap * (s.d - 1), z2 = s.B0 + P.gap * (s.d - 2);
#pragma unroll
    for (int p = 0; p < H; p++) {
        const int32_t a = lo16(P1[p]), b = hi16(P1[p]), c = lo16(P2[p]), e = hi16(P2[p]);
        __stcg(r + kRecHeader + gl * CG + p, a >= 0 ? (a >> 5) + z1 : kNegR);
        __stcg(r + kRecHeader + gl * CG + H + p, b >= 0 ? (b >> 5) + z1 : kNegR);
        __stcg(r + kRecHeader + W + gl * CG + p, c >= 0 ? (c >> 5) + z2 : kNegR);
        __stcg(r + kRecHeader + W + gl * CG + H + p, e >= 0 ? (e >> 5) + z2 : kNegR);
    }
    if (gl == 0) {
        __stcg(r + 0, W);
        __stcg(r + 1, s.d);
        __stcg(r + 2, s.rb);
        __stcg(r + 3, s.L);
        __stcg(r + 4, s.U);
        __stcg(r + 5, s.T);
        __stcg(r + 6, s.best);
        __stcg(r + 7, s.bi);
        __stcg(r + 8, s.bj);
        __stcg(r + 9, s.barg);
        __stcg(r + 10, int32_t(s.flags));
        __stcg(r + 11, int32_t(uint32_t(s.cells)));
        __stcg(r + 12, int32_t(uint32_t(s.cells >> 32)));
    }
}

template <int G, int CG>
__device__ __forceinline__ bool load_record16(const Problem& P, const Z16& zc, uint32_t ri, SideState& s,
                                              uint32_t (&A)[CG / 2], uint32_t (&B)[CG / 2], int gl) {
    constexpr int W = G * CG, H = CG / 2;
    const int32_t* r = P.rec + ri;
    const int32_t w0 = __ldcg(r + 0);
    if (w0 > W) return false;
    const int32_t off = (W - w0) / 2;
    s.d = __ldcg(r + 1);
    s.rb = __ldcg(r + 2) - off;
    s.L = __ldcg(r + 3);
    s.U = __ldcg(r + 4);
    s.T = __ldcg(r + 5);
    s.best = __ldcg(r + 6);
    s.bi = __ldcg(r + 7);
    s.bj = __ldcg(r + 8);
    s.barg = __ldcg(r + 9);
    s.flags = uint32_t(__ldcg(r + 10));
    s.cells = uint64_t(uint32_t(__ldcg(r + 11))) | (uint64_t(uint32_t(__ldcg(r + 12))) << 32);
    // theta of the next anti-diagonal at theta0
    s.B0 = s.T - P.X - P.gap * s.d - zc.th0;
    const int32_t z1 = s.B0 + P.gap * (s.d - 1), z2 = s.B0 + P.gap * (s.d - 2);
    const bool odd = s.d & 1;   // odd d: A holds d-1; even d: B holds d-1
    int32_t v1[2], v2[2];
#pragma unroll
    for (int p = 0; p < H; p++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int src = gl * CG + p + h * H - off;
            const bool in = src >= 0 && src < w0;
            const int32_t x1 = in ? __ldcg(r + kRecHeader + src) : kNegR;
            const int32_t x2 = in ? __ldcg(r + kRecHeader + w0 + src) : kNegR;
            v1[h] = x1 < kDeadR ? -1 : 32 * (x1 - z1);
            v2[h] = x2 < kDeadR ? -1 : 32 * (x2 - z2);
        }
        const uint32_t a = pack2(v1[0], v1[1]), b = pack2(v2[0], v2[1]);
        A[p] = odd ? a : b;
        B[p] = odd ? b : a;
    }
    return true;
}

// Runs side extensions from S with groups of G lanes until S is exhausted; overflows go to
// q[out_q], carrying an escalation record when the next level is a register level.
// gsm_block: the block's shared rows (2W ints per group).
// smem: the block's similarity table, then one shift area of warp_ints ints per warp (at
// least 64 * CG: 2W ints for each of the warp's 32 / G groups).  The areas belong to warps,
// not to groups, so that warps of one block may run groups of different shapes at the same
// time (the roles of the fused grid) without sharing shift buffers.
template <int G, int CG, int A, bool LIVE>
__device__ __forceinline__ void group_loop(const Problem& P, const Queues& Q, const Source& S, int out_q,
                                           int chunk, int32_t* smem, int stage, int warp_ints, int level) {
    constexpr int W = G * CG;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const uint32_t gm = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
    const int32_t* tab = smem;
    int32_t* gsm = smem + kLutInts + (threadIdx.x >> 5) * warp_ints + ((threadIdx.x & 31) / G) * 2 * W;
    // kDna16: CG/2 registers of two 16-bit slots each, else CG int32 slots
    constexpr bool PK = packed_rep(A);
    constexpr int NR = PK ? CG / 2 : CG;
    const Z16 zc = z16_of(P);
    using Reg = std::conditional_t<PK, uint32_t, int32_t>;
    Reg R0[NR], R1[NR];
    SideState s{};
    Res<CG, A> res;
    uint32_t uidx = 0, pair = 0, next = 0, end = 0;
    bool active = false, done = false, skip_odd = false;
    int32_t d_start = 0;
    uint64_t cells_start = 0;
    unsigned long long t_take = 0;   // tracing: when the group took its side
    LiveWait lw;   // unused (optimised away) for a finished list
    uint32_t pause = 128;
    for (;;) {
        bool took = false;
        if (!active && !done) {
            const int st = take_unit<G, LIVE>(S, gl, lane, gm, chunk, next, end, uidx, lw, P.err, took);
            if (st < 0) done = true;
            if (st > 0) {
                took = true;
                const Unit u = P.units[uidx];
                if ((int64_t(u.m) + u.n) * P.max_abs >= kRegLimit || P.alpha != alpha_of(A) ||
                    (PK && !packed_ok(P))) {
                    if (gl == 0) push_unit(Q, kBandQ, uidx);
                } else {
                    init_side(s, u, -W / 2);
                    pair = u.pair;
                    if (s.m + s.n == 0) {
                        if (gl == 0) {
                            if (P.trace) trace_visit(P, uidx, level, trace_clock(), 0, W, G, 1);
                            write_side(P.results, pair, s.side, 0, 0, 0, 0, 1);
                            atomicAdd(&P.stats[stage], 1ull);
                            atomicAdd(&P.stats[4 + stage], 1ull);
                        }
                    } else {
                        const uint32_t ri = P.rec_of ? __ldcg(P.rec_of + uidx) : kNoUnit;
                        bool resumed = false;
                        if (ri != kNoUnit) {
                            if constexpr (PK) resumed = load_record16<G, CG>(P, zc, ri, s, R0, R1, gl);
                            else resumed = load_record<G, CG>(P, ri, s, R0, R1, gl);
                        }
                        if (!resumed) {
                            // S(0,0) = 0 in the middle of the window, every other cell -inf (Sec. 2.2)
                            if constexpr (PK) {
                                constexpr int t0 = (W / 2) % CG, p0 = t0 % (CG / 2);
                                s.B0 = -P.X - P.gap - zc.th0;   // theta of d = 1 at theta0
                                const int32_t z0 = -32 * s.B0;
#pragma unroll
                                for (int p = 0; p < NR; p++) {
                                    R0[p] = kDead2;
                                    R1[p] = kDead2;
                                }
                                if (gl == (W / 2) / CG) R0[p0] = t0 < CG / 2 ? pack2(z0, -1) : pack2(-1, z0);
                            } else {
#pragma unroll
                                for (int t = 0; t < CG; t++) {
                                    R0[t] = kNegR;
                                    R1[t] = kNegR;
                                }
                                if (gl == (W / 2) / CG) R0[(W / 2) % CG] = 0;
                            }
                        }
                        skip_odd = (s.d & 1) == 0;   // a side continued on an even anti-diagonal
                        active = true;
                        d_start = s.d;
                        cells_start = s.cells;
                        if (P.trace) t_take = trace_clock();
                    }
                }
            }
        }
        if (active) {
            int r = kCont;
            if constexpr (PK) {
                if (!skip_odd) r = group_step16<G, CG, true, A>(s, res, R0, R1, P, zc, tab, gl, gm, gsm);
                skip_odd = false;
                if (r == kCont) r = group_step16<G, CG, false, A>(s, res, R1, R0, P, zc, tab, gl, gm, gsm);
            } else {
                if (!skip_odd) r = group_step<G, CG, true, A>(s, res, R0, R1, P, tab, gl, gm, gsm);
                skip_odd = false;
                if (r == kCont) r = group_step<G, CG, false, A>(s, res, R1, R0, P, tab, gl, gm, gsm);
            }
            if (r != kCont) {
                active = false;
                if (gl == 0) {
                    // window fill of this level: in-band cells against the slots evaluated
                    atomicAdd(&P.stats[9], (unsigned long long)(s.cells - cells_start));
                    atomicAdd(&P.stats[10], (unsigned long long)(s.d + 1 - d_start) * (unsigned long long)W);
                    if (P.trace)
                        trace_visit(P, uidx, level, t_take, uint32_t(s.d + 1 - d_start), W, G, r == kDone ? 1 : 2);
                }
                if (r == kDone) {
                    if (gl == 0) {
                        write_side(P.results, pair, s.side, s.best, uint32_t(s.bi), uint32_t(s.bj), s.flags,
                                   s.cells);
                        atomicAdd(&P.stats[stage], 1ull);
                        atomicAdd(&P.stats[4 + stage], (unsigned long long)s.cells);
                    }
                } else {
                    // overflow: hand the side to the next level, with its state when that level
                    // can take it
                    uint32_t ri = kNoUnit;
                    if (out_q <= kBandQ && P.rec) {
                        // bump-allocate kRecHeader + 2W ints of the record pool
                        const uint32_t need = uint32_t(kRecHeader + 2 * W);
                        if (gl == 0) ri = atomicAdd(P.rec_ctr, need);
                        if (G > 1) ri = __shfl_sync(gm, ri, lane - gl);
                        if (ri <= P.rec_cap && P.rec_cap - ri >= need) {
                            if constexpr (PK) {
                                if (s.d & 1) save_record16<G, CG>(P, ri, s, R0, R1, gl);
                                else save_record16<G, CG>(P, ri, s, R1, R0, gl);
                            } else {
                                if (s.d & 1) save_record<G, CG>(P, ri, s, R0, R1, gl);
                                else save_record<G, CG>(P, ri, s, R1, R0, gl);
                            }
                            if (G > 1) __syncwarp(gm);
                        } else {
                            ri = kNoUnit;
                        }
                    }
                    if (gl == 0) {
                        if (ri != kNoUnit) {
                            __threadfence();
                            __stcg(P.rec_of + uidx, ri);
                            __threadfence();
                        } else {
                            atomicAdd(&P.stats[7], (unsigned long long)s.cells);
                        }
                        push_unit(Q, out_q, uidx);
                        atomicAdd(&P.stats[3], 1ull);
                    }
                }
            }
        }
        // the warp leaves once every group is done (measured faster than leaving group by
        // group); a warp of a live source with no group at work and none that took a ticket
        // backs off before polling again
        if (__all_sync(0xffffffffu, done)) break;
        if constexpr (LIVE) {
            if (__any_sync(0xffffffffu, active || took)) {
                pause = 128;
            } else {
                __nanosleep(pause);
                pause = min(pause * 2u, 8192u);
            }
        }
    }
}


__device__ __forceinline__ Source static_source(const Queues& Q, int in_q) {
    Source S{};
    S.list = in_q < 0 ? Q.order : Q.q[in_q];
    S.pull = in_q < 0 ? &Q.ctr[0] : &Q.ctr[2 + 2 * in_q];
    S.n = in_q < 0 ? Q.n_units : *reinterpret_cast<volatile uint32_t*>(&Q.ctr[1 + 2 * in_q]);
    S.live = false;
    return S;
}

// One register level over a finished list.  in_q < 0: the cost-ordered units, else q[in_q].
template <int G, int CG, int MINB, int A>
__global__ void __launch_bounds__(128, MINB) k_group(Problem P, Queues Q, int in_q, int out_q, int chunk) {
    extern __shared__ __align__(16) int32_t group_smem[];
    build_table<A>(group_smem, P);
    group_loop<G, CG, A, false>(P, Q, static_source(Q, in_q), out_q, chunk, group_smem, in_q < 0 ? 0 : 1,
                                64 * CG, in_q + 1);
}

// The first register levels fused into one persistent, cooperatively launched grid.
// Each warp walks the role sequence 0 -> 1 -> 2: role 0 runs the cost-ordered units with
// groups of G0 lanes and appends overflows to the live queue q[0]; role 1 consumes q[0]
// with groups of G1 lanes and appends its overflows to the live queue q[1]; role 2
// consumes q[1] with groups of G2 lanes, overflows go to q[2] for the later register
// launches, or to the band tier when the chain has no level after the grid.
// Some warps start directly in role 1 or 2, so wider sides begin while narrower levels
// still run.  A warp that leaves role 0 (1) counts itself in done[0] (done[1]); consumers
// stop once their queue is drained and all its producers have counted themselves.
struct RolePlan {
    int every1, every2;         // warp gw starts in role 2 if gw % every2 == every2 - 1,
                                // else in role 1 if gw % every1 == 0, else in role 0
    uint32_t producers0;        // warps that run role 0
    uint32_t producers1;        // warps that run role 0 or 1
    uint32_t n_long;            // units at the head of the cost order taken by the long role
    uint32_t long_warps;        // warps gw < long_warps start in the long role, then role 0
    int out2;                   // queue of role 2's overflows: q[2] when later register levels
                                // follow the grid, else the band tier's queue
    uint64_t wait_limit_ns;     // live-queue waits give up (kErrWait) after this long without
                                // progress
    int every3;                 // four-role grids: warp gw starts in role 3 if
                                // gw % every3 == every3 - 1 (checked first)
    uint32_t producers2;        // four-role grids: warps that run role 0, 1 or 2
};

__host__ __device__ __forceinline__ int start_role(uint32_t gw, int every1, int every2, int every3 = 0) {
    if (every3 > 0 && gw % uint32_t(every3) == uint32_t(every3 - 1)) return 3;
    if (every2 > 0 && gw % uint32_t(every2) == uint32_t(every2 - 1)) return 2;
    if (every1 > 0 && gw % uint32_t(every1) == 0) return 1;
    return 0;
}

__device__ __forceinline__ Source live_source(const Queues& Q, int k, uint32_t* done, uint32_t producers,
                                              uint64_t wait_limit_ns) {
    Source S{};
    S.list = Q.q[k];
    S.pull = &Q.ctr[2 + 2 * k];
    S.live = true;
    S.reserve = &Q.ctr[1 + 2 * k];
    S.producers_done = done;
    S.n_producers = producers;
    S.wait_limit_ns = wait_limit_ns;
    return S;
}

__device__ __forceinline__ void signal_done(uint32_t* done) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        atomicAdd(done, 1u);
    }
    __syncwarp();
}

// Shift-area ints per warp of a fused grid: 64 x the largest slots per lane of its roles.
template <int C0, int C1, int C2, int CL>
__host__ __device__ constexpr int fused_warp_ints() {
    int c = C0 > C1 ? C0 : C1;
    c = c > C2 ? c : C2;
    c = c > CL ? c : CL;
    return 64 * c;
}

// GL x CL (GL = 0: none) is the long role: the first R.long_warps warps take the R.n_long
// longest sides (the head of the cost order) with GL-lane groups, whose anti-diagonals take
// less time than a single lane's, so that the longest serial chains do not set the
// makespan; those warps then join role 0 on the rest of the order.
template <int G0, int C0, int G1, int C1, int G2, int C2, int MINB, int A, int GL, int CL>
__global__ void __launch_bounds__(128, MINB) k_fused(Problem P, Queues Q, RolePlan R, int chunk) {
    constexpr int kWarpInts = fused_warp_ints<C0, C1, C2, CL>();
    extern __shared__ __align__(16) int32_t group_smem[];
    build_table<A>(group_smem, P);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t* done0 = &Q.ctr[1 + 2 * kLevels];
    uint32_t* done1 = &Q.ctr[2 + 2 * kLevels];
    const bool long_role = GL > 0 && gw < R.long_warps;
    const int role = long_role ? 0 : start_role(gw, R.every1, R.every2);
    if constexpr (GL > 0) {
        if (long_role) {
            Source SL = static_source(Q, -1);
            SL.pull = &Q.ctr[kLongPull];
            SL.n = R.n_long;
            group_loop<GL, CL, A, false>(P, Q, SL, 0, 1, group_smem, 0, kWarpInts, kTraceLong);
        }
    }
    if (role == 0) {
        Source S0 = static_source(Q, -1);
        S0.list = Q.order + R.n_long;
        S0.n = Q.n_units - R.n_long;
        group_loop<G0, C0, A, false>(P, Q, S0, 0, chunk, group_smem, 0, kWarpInts, 0);
        signal_done(done0);
    }
    if (role <= 1) {
        group_loop<G1, C1, A, true>(P, Q, live_source(Q, 0, done0, R.producers0, R.wait_limit_ns), 1, 1, group_smem, 0,
                              kWarpInts, 1);
        signal_done(done1);
    }
    group_loop<G2, C2, A, true>(P, Q, live_source(Q, 1, done1, R.producers1, R.wait_limit_ns), R.out2, 1, group_smem, 0,
                          kWarpInts, 2);
}

// Four roles: k_fused with a fourth level.  Role 2 appends its overflows to the live queue
// q[2], which role 3 consumes; role 3's overflows go to R.out2 (q[3] when later register
// levels follow the grid, else the band tier).  A warp that leaves role 2 counts itself in
// done[2].
template <int G0, int C0, int G1, int C1, int G2, int C2, int G3, int C3, int MINB, int A, int GL, int CL>
__global__ void __launch_bounds__(128, MINB) k_fused4(Problem P, Queues Q, RolePlan R, int chunk) {
    constexpr int kC13 = C1 > C3 ? C1 : C3;
    constexpr int kWarpInts = fused_warp_ints<C0, kC13, C2, CL>();
    extern __shared__ __align__(16) int32_t group_smem[];
    build_table<A>(group_smem, P);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t* done0 = &Q.ctr[1 + 2 * kLevels];
    uint32_t* done1 = &Q.ctr[2 + 2 * kLevels];
    uint32_t* done2 = &Q.ctr[kDone2];
    const bool long_role = GL > 0 && gw < R.long_warps;
    const int role = long_role ? 0 : start_role(gw, R.every1, R.every2, R.every3);
    if constexpr (GL > 0) {
        if (long_role) {
            Source SL = static_source(Q, -1);
            SL.pull = &Q.ctr[kLongPull];
            SL.n = R.n_long;
            group_loop<GL, CL, A, false>(P, Q, SL, 0, 1, group_smem, 0, kWarpInts, kTraceLong);
        }
    }
    if (role == 0) {
        Source S0 = static_source(Q, -1);
        S0.list = Q.order + R.n_long;
        S0.n = Q.n_units - R.n_long;
        group_loop<G0, C0, A, false>(P, Q, S0, 0, chunk, group_smem, 0, kWarpInts, 0);
        signal_done(done0);
    }
    if (role <= 1) {
        group_loop<G1, C1, A, true>(P, Q, live_source(Q, 0, done0, R.producers0, R.wait_limit_ns), 1, 1, group_smem, 0,
                              kWarpInts, 1);
        signal_done(done1);
    }
    if (role <= 2) {
        group_loop<G2, C2, A, true>(P, Q, live_source(Q, 1, done1, R.producers1, R.wait_limit_ns), 2, 1, group_smem, 0,
                              kWarpInts, 2);
        signal_done(done2);
    }
    group_loop<G3, C3, A, true>(P, Q, live_source(Q, 2, done2, R.producers2, R.wait_limit_ns), R.out2, 1, group_smem, 0,
                          kWarpInts, 3);
}

template <int G, int CG, int MINB, int A>
static cudaError_t launch_group(const Problem& P, const Queues& Q, int in_q, int out_q, int blocks,
                                int chunk, cudaStream_t st) {
    const size_t smem = (size_t(kLutInts) + size_t(128 / G) * 2 * G * CG) * sizeof(int32_t);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_group<G, CG, MINB, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        // the largest shared-memory carveout, so that the blocks the registers allow fit
        e = cudaFuncSetAttribute(k_group<G, CG, MINB, A>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_group<G, CG, MINB, A><<<blocks, 128, smem, st>>>(P, Q, in_q, out_q, chunk);
    return cudaGetLastError();
}

template <int G, int CG>
constexpr size_t group_smem_bytes() {
    return (size_t(kLutInts) + size_t(128 / G) * 2 * G * CG) * sizeof(int32_t);
}

template <int G0, int C0, int G1, int C1, int G2, int C2, int MINB, int A, int GL = 0, int CL = 4>
static cudaError_t launch_fused(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                cudaStream_t st) {
    constexpr int kCL = (GL > 0) ? CL : 4;
    const size_t smem = (size_t(kLutInts) + 4 * size_t(fused_warp_ints<C0, C1, C2, kCL>())) * sizeof(int32_t);
    auto fn = k_fused<G0, C0, G1, C1, G2, C2, MINB, A, GL, kCL>;
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 128, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
    }
    // every block must be resident at once: consumers wait for producers of the same grid
    const int blocks = n_sm * occ;
    const uint32_t n_warps = uint32_t(blocks) * 4;
    RolePlan R{cfg.every1, cfg.every2, 0, 0, 0, 0, cfg.n_levels > 3 ? 2 : kBandQ,
               cfg.wait_limit_ms > 0 ? uint64_t(cfg.wait_limit_ms) * 1000000ull : kWaitLimitNs};
    if (GL > 0 && cfg.long_permille > 0) {
        R.n_long = uint32_t(uint64_t(Q.n_units) * uint32_t(cfg.long_permille) / 1000u);
        R.long_warps = std::min(R.n_long, n_warps / 4);   // at most a quarter of the grid
    }
    for (uint32_t w = 0; w < n_warps; w++) {
        const int r = w < R.long_warps ? 0 : start_role(w, R.every1, R.every2);
        R.producers0 += r == 0;
        R.producers1 += r <= 1;
    }
    if (R.producers0 == 0) return cudaErrorInvalidValue;   // nobody would take the ordered units
    // failure-detection test: a role-0 producer that never finishes, so that the role-1
    // consumers' waits run out (bounded) and the batch reports kErrWait
    R.producers0 += cfg.phantom_producer ? 1u : 0u;
    R.producers1 += cfg.phantom_producer ? 1u : 0u;
    Problem p = P;
    Queues q = Q;
    int ch = cfg.chunk;
    void* args[] = {&p, &q, &R, &ch};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3(blocks), dim3(128), args, smem, st);
}

template <int G0, int C0, int G1, int C1, int G2, int C2, int G3, int C3, int MINB, int A, int GL, int CL>
static cudaError_t launch_fused4(const Problem& P, const Queues& Q, const TierConfig& cfg, int n_sm,
                                 cudaStream_t st) {
    constexpr int kC13 = C1 > C3 ? C1 : C3;
    const size_t smem = (size_t(kLutInts) + 4 * size_t(fused_warp_ints<C0, kC13, C2, CL>())) * sizeof(int32_t);
    auto fn = k_fused4<G0, C0, G1, C1, G2, C2, G3, C3, MINB, A, GL, CL>;
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 128, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
    }
    // every block must be resident at once: consumers wait for producers of the same grid
    const int blocks = n_sm * occ;
    const uint32_t n_warps = uint32_t(blocks) * 4;
    RolePlan R{cfg.every1, cfg.every2, 0, 0, 0, 0, cfg.n_levels > 4 ? 3 : kBandQ,
               cfg.wait_limit_ms > 0 ? uint64_t(cfg.wait_limit_ms) * 1000000ull : kWaitLimitNs, cfg.every3, 0};
    if (GL > 0 && cfg.long_permille > 0) {
        R.n_long = uint32_t(uint64_t(Q.n_units) * uint32_t(cfg.long_permille) / 1000u);
        R.long_warps = std::min(R.n_long, n_warps / 4);   // at most a quarter of the grid
    }
    for (uint32_t w = 0; w < n_warps; w++) {
        const int r = w < R.long_warps ? 0 : start_role(w, R.every1, R.every2, R.every3);
        R.producers0 += r == 0;
        R.producers1 += r <= 1;
        R.producers2 += r <= 2;
    }
    if (R.producers0 == 0) return cudaErrorInvalidValue;   // nobody would take the ordered units
    // failure-detection test: a role-0 producer that never finishes
    R.producers0 += cfg.phantom_producer ? 1u : 0u;
    R.producers1 += cfg.phantom_producer ? 1u : 0u;
    R.producers2 += cfg.phantom_producer ? 1u : 0u;
    Problem p = P;
    Queues q = Q;
    int ch = cfg.chunk;
    void* args[] = {&p, &q, &R, &ch};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3(blocks), dim3(128), args, smem, st);
}

}  // namespace xd
