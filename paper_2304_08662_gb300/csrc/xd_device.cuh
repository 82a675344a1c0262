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

// Per-side timeline (tracing, off unless the host asks for it): one record per side
// extension and level that worked on it.  Visit slot: register levels 0 .. 4 (the fused
// grid's roles are levels 0 .. 3), 5 the band tier, 6 the generic tier, 7 the fused grid's
// long-side role.
using TraceRec = xd_trace_rec;   // layout in xdrop.h
static_assert(sizeof(TraceRec) == 24, "trace record layout");
constexpr int kTraceVisits = 8;
constexpr int kTraceLong = 7, kTraceBand = 5, kTraceGeneric = 6;

__device__ __forceinline__ unsigned long long trace_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t trace_smid() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

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
    int32_t zdrop;              // 0 = X-Drop alone, > 0: Z-Drop with Z = zdrop
    int32_t max_abs;            // largest |score| of one step (similarity or gap)
    int32_t s_max;              // largest similarity, at least 0
    // Escalation records: a side that outgrows a register level's window saves its two
    // anti-diagonals and band state so that the next level continues instead of restarting.
    int32_t* rec;               // record pool of rec_cap ints
    uint32_t* rec_of;           // per unit: offset of its record, or 0xffffffff (start from scratch)
    uint32_t* rec_ctr;          // pool allocation counter (ints)
    uint32_t rec_cap;
    TraceRec* trace;            // per unit kTraceVisits records, or null (no tracing)
    int8_t sim[400];            // alpha x alpha similarity, row-major with stride alpha
};

__device__ __forceinline__ void trace_visit(const Problem& P, uint32_t unit, int level, unsigned long long t0,
                                            uint32_t diags, int window, int lanes, int outcome) {
    TraceRec r;
    r.start_ns = t0;
    const unsigned long long t1 = trace_clock();
    r.dur_ns = uint32_t(t1 - t0 < 0xffffffffull ? t1 - t0 : 0xffffffffull);
    r.diags = diags;
    r.window = uint16_t(window);
    r.smid = uint16_t(trace_smid());
    r.lanes = uint8_t(lanes);
    r.level = uint8_t(level);
    r.outcome = uint16_t(outcome);
    P.trace[size_t(unit) * kTraceVisits + level] = r;
}

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
