// Internal device-side definitions of the X-Drop library (shared by its two translation
// units, never by the CPU oracle).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "xdrop.h"

namespace xd {

// -inf for scores: dead cells hold exactly kNeg.  Thresholds are clamped to kDeadLine, so
// anything computed from a dead predecessor (kNeg plus at most a few small scores) is
// pruned, while every real score (|S| < 2^29, checked at admission) is compared exactly.
constexpr int32_t kNeg = -(1 << 30);
constexpr int32_t kDeadLine = -(1 << 29);
constexpr int64_t kScoreLimit = int64_t(1) << 29;

// Error word bits (also documented in xdrop.h, xd_device_status).
constexpr uint32_t kErrCode = 1u;       // residue code outside the alphabet
constexpr uint32_t kErrSeed = 2u;       // seed outside its sequence / bad sequence id
constexpr uint32_t kErrRange = 4u;      // score range or reserved length exceeded
constexpr uint32_t kErrWait = 8u;       // a bounded device wait gave up

// One side extension (Sec. 4.1.2 LR splitting: each side is its own unit of work).
// H_side[t] = packed[h0 + hdir * t] (hdir = +1 right side, -1 left side), same for V.
struct Unit {
    uint64_t h0, v0;
    uint32_t m, n;
    uint32_t pair;
    uint32_t side;      // 0 = right, 1 = left
};
static_assert(sizeof(Unit) == 32, "unit layout");

// Everything a tier kernel needs about the batch.
struct Problem {
    const uint32_t* store;      // packed residues of the whole codes buffer
    uint64_t n_words;           // words in store
    const Unit* units;
    xd_result* results;         // per pair
    uint32_t* err;              // validation / wait error word
    unsigned long long* stats;  // per batch: [0..2] units finished per stage, [3] escalations,
                                // [4..6] cells per stage, [7] cells discarded by escalation,
                                // [8] window re-centrings, [9] / [10] in-band cells and
                                // slots evaluated by the register levels.  Stage 0: the first register
                                // launch (fused grid or level 0); 1: later register levels
                                // and the band tier; 2: the generic tier
    int32_t alpha;              // 4 or 20
    int32_t gap;
    int32_t X;
    uint32_t delta;             // 0 = unrestricted
    int32_t max_abs;            // largest |score| of one step (similarity or gap)
    int32_t s_max;              // largest similarity, at least 0
    // Escalation records: a side that outgrows a register level's window saves its two
    // anti-diagonals and band state so that the next level continues instead of restarting.
    int32_t* rec;               // record pool of rec_cap ints
    uint32_t* rec_of;           // per unit: offset of its record, or 0xffffffff (start from scratch)
    uint32_t* rec_ctr;          // pool allocation counter (ints)
    uint32_t rec_cap;
    int8_t sim[400];            // alpha x alpha similarity, row-major with stride alpha
};

// Queue state of one batch.  The first register level pulls the cost-ordered unit list;
// a side whose band does not fit a level's window is appended to the next level's queue.
// q[kBandQ] feeds the shared-memory band tier, q[kGenericQ] the generic tier.
constexpr int kLevels = 7;
constexpr int kBandQ = kLevels - 2;
constexpr int kGenericQ = kLevels - 1;

struct Queues {
    const uint32_t* order;      // all units, most expensive first (first level's input)
    uint32_t n_units;
    uint32_t* q[kLevels];
    uint32_t* ctr;              // [0] order pull; [1 + 2k] length of q[k]; [2 + 2k] pull of q[k]
};

__device__ __forceinline__ void push_unit(const Queues& Q, int k, uint32_t unit) {
    Q.q[k][atomicAdd(&Q.ctr[1 + 2 * k], 1u)] = unit;
}

// Residue at absolute position pos of the packed store.
// DNA: 16 residues of 2 bits per word.  Protein: 6 residues of 5 bits per word.
__device__ __forceinline__ uint32_t residue(const uint32_t* store, int alpha, uint64_t pos) {
    if (alpha == 4) return (__ldg(store + (pos >> 4)) >> (uint32_t(pos & 15) * 2u)) & 3u;
    uint64_t w = pos / 6;
    uint32_t r = uint32_t(pos - w * 6);
    return (__ldg(store + w) >> (5u * r)) & 31u;
}

__device__ __forceinline__ void write_side(xd_result* res, uint32_t pair, uint32_t side,
                                           int32_t score, uint32_t hi, uint32_t vj,
                                           uint32_t flags, uint64_t cells) {
    xd_side* s = side ? &res[pair].left : &res[pair].right;
    s->score = score;
    s->h_ext = hi;
    s->v_ext = vj;
    s->flags = flags;
    s->cells = cells;
}

}  // namespace xd
