// Host runtime behind the C ABI of xdrop.h: contexts, validation, memory admission,
// pinned staging, the request dispatcher (continuous batching over in-flight slots with
// their own streams), tickets, and the device pipeline that runs one batch.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "xdrop.h"
#include "xd_device.cuh"
#include "xd_launch.h"

namespace {

using namespace xd;

// NVTX range over a host-side scope (visible to timeline profilers; free without one).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

cudaError_t grow(DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t n = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, n);
    if (e == cudaSuccess) b.cap = n;
    return e;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

struct HostBuf {
    void* p = nullptr;
    size_t cap = 0;
};

cudaError_t grow_pinned(HostBuf& b, size_t bytes) {
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t n = std::max<size_t>(bytes, 4096);
    cudaError_t e = cudaHostAlloc(&b.p, n, cudaHostAllocDefault);
    if (e == cudaSuccess) b.cap = n;
    return e;
}

// Device working memory of one batch in flight.
struct Scratch {
    DevBuf store, units, bucket, order, ctr, hist, err, generic, bstats, rec, rec_of;
    DevBuf q[kLevels];           // escalation queues, one per register level plus generic
};

void release(Scratch& s) {
    for (DevBuf* b : {&s.store, &s.units, &s.bucket, &s.order, &s.ctr, &s.hist, &s.err, &s.generic,
                      &s.bstats, &s.rec, &s.rec_of})
        release(*b);
    for (DevBuf& q : s.q) release(q);
}

// A batch as the device pipeline sees it (device pointers).
struct BatchView {
    int alpha = 4;
    uint32_t n_seqs = 0;
    uint64_t n_codes = 0;
    const uint8_t* codes = nullptr;
    const uint64_t* offsets = nullptr;
    const uint32_t* lengths = nullptr;
    uint32_t n_pairs = 0;
    const xd_pair* pairs = nullptr;
    int8_t sim[400] = {};
    int32_t gap = 0, X = 0, max_abs = 1, zdrop = 0;
    uint32_t delta = 0, max_len = 0;
    const uint32_t* packed = nullptr;   // resident store: residues already packed (no codes)
    uint64_t packed_words = 0;
};

// One submitted host batch (a request).  Its inputs are copied to a pinned buffer at
// submit, laid out codes | offsets | lengths | pairs; results are copied out of the slot
// that ran it when that slot finishes.
struct Request {
    enum State { kPending, kLaunched, kDone, kFailed };
    uint64_t ticket = 0;
    State state = kPending;
    xd_status status = XD_OK;
    std::string err;
    BatchView v;                 // parameters and sizes; pointers unused
    HostBuf in;
    size_t o_offs = 0, o_lens = 0, o_pairs = 0, in_bytes = 0;
    size_t n_words = 0;          // packed residue words at the start of its pinned buffer
    size_t need = 0;             // device bytes admitted for it
    bool pairs_only = false;     // seed tuples on the resident sequence store
    std::vector<xd_result> out;
};

// Parameter sets (alphabet, scoring, X, delta_b, Z) one launch may carry.
constexpr int kSlotGroups = 4;

// An in-flight launch: one or more requests merged into one upload and one result copy; the
// requests of each parameter set form one batch of the hot path (the first on the slot's
// stream, the others on streams of their own that fork after the upload and join before
// the result copy).
struct Slot {
    bool busy = false;
    uint32_t n_pairs = 0;
    int n_groups = 0;                  // parameter sets of the in-flight launch
    std::vector<Request*> reqs;
    std::vector<uint32_t> pair_base;   // first result of each request in the merged batch
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t uploaded = nullptr;    // created at the first launch of several sets
    Scratch s;
    struct Side {                      // the second and later parameter sets
        cudaStream_t stream = nullptr;
        cudaEvent_t joined = nullptr;
        Scratch s;
    } side[kSlotGroups - 1];
    DevBuf d_in, d_results;
    HostBuf h_stage, h_out;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Residue check of one block: true if every byte is below alpha.  Eight bytes at a time.
bool codes_valid(const uint8_t* p, size_t n, int alpha) {
    size_t t = 0;
    if (alpha == 4) {
        uint64_t bad = 0;
        for (; t + 8 <= n; t += 8) {
            uint64_t w;
            std::memcpy(&w, p + t, 8);
            bad |= w & 0xFCFCFCFCFCFCFCFCull;
        }
        if (bad) return false;
    } else {
        for (; t + 8 <= n; t += 8) {
            uint64_t w;
            std::memcpy(&w, p + t, 8);
            // a byte b >= 20 has bit 7 set in b or in b + 108 (a carry out of a byte that is
            // itself >= 148 can only add to an already invalid word)
            if ((w | (w + 0x6C6C6C6C6C6C6C6Cull)) & 0x8080808080808080ull) return false;
        }
    }
    for (; t < n; t++)
        if (p[t] >= alpha) return false;
    return true;
}

// Copies n bytes to dst with up to 16 host threads; when alpha > 0 also checks that every
// byte is a residue code below alpha (each block is checked right after it is copied, while
// it is still in cache).  Returns the index of a block holding an invalid code, or SIZE_MAX.
size_t par_copy_check(void* dst, const void* src, size_t n, int alpha) {
    const size_t kBlock = size_t(256) << 10;
    const size_t kMinParallel = size_t(32) << 20;
    auto run = [&](size_t a, size_t b, std::atomic<size_t>* bad) {
        for (size_t s = a; s < b; s += kBlock) {
            const size_t e = std::min(b, s + kBlock);
            std::memcpy(static_cast<char*>(dst) + s, static_cast<const char*>(src) + s, e - s);
            if (alpha > 0 && !codes_valid(static_cast<const uint8_t*>(dst) + s, e - s, alpha)) {
                size_t cur = bad->load();
                while (s < cur && !bad->compare_exchange_weak(cur, s)) {
                }
            }
        }
    };
    std::atomic<size_t> bad{SIZE_MAX};
    if (n < kMinParallel) {
        run(0, n, &bad);
        return bad.load();
    }
    unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    size_t per = align_up((n + hw - 1) / hw, kBlock);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < hw; t++) {
        size_t a = t * per;
        if (a >= n) break;
        size_t b = std::min(n, a + per);
        th.emplace_back(run, a, b, &bad);
    }
    for (auto& t : th) t.join();
    return bad.load();
}

void par_memcpy(void* dst, const void* src, size_t n) { par_copy_check(dst, src, n, 0); }

// Host packing of residue codes in the device store's layout, while they are staged:
// DNA word w holds codes 16w .. 16w + 15, code t at bits 2t; protein word w holds codes
// 6w .. 6w + 5, code t at bits 5t.  8 DNA codes (one byte each, 0..3) to 16 bits: pair the
// bytes of each 16-bit lane, then the nibbles of each 32-bit lane, then the bytes.
inline uint32_t pack8_dna(uint64_t x) {
    x = (x | (x >> 6)) & 0x000F000F000F000Full;
    x = (x | (x >> 12)) & 0x000000FF000000FFull;
    return uint32_t((x | (x >> 24)) & 0xFFFFull);
}

size_t packed_words(uint64_t n_codes, int alpha) {
    const uint64_t per = alpha == 4 ? 16 : 6;
    return size_t((n_codes + per - 1) / per);
}

// Packs words [w0, w1) of n codes from src into dst; false if a code is outside the alphabet.
bool pack_range(uint32_t* dst, const uint8_t* src, uint64_t n, int alpha, size_t w0, size_t w1) {
    bool ok = true;
    if (alpha == 4) {
        for (size_t w = w0; w < w1; w++) {
            const uint64_t base = uint64_t(w) * 16;
            if (base + 16 <= n) {
                uint64_t a, b;
                std::memcpy(&a, src + base, 8);
                std::memcpy(&b, src + base + 8, 8);
                ok &= ((a | b) & 0xFCFCFCFCFCFCFCFCull) == 0;
                dst[w] = pack8_dna(a) | (pack8_dna(b) << 16);
            } else {
                uint32_t word = 0;
                for (uint64_t t = 0; base + t < n; t++) {
                    const uint8_t c = src[base + t];
                    ok &= c < 4;
                    word |= uint32_t(c & 3u) << (2 * t);
                }
                dst[w] = word;
            }
        }
    } else {
        for (size_t w = w0; w < w1; w++) {
            const uint64_t base = uint64_t(w) * 6;
            uint32_t word = 0;
            for (uint64_t t = 0; t < 6 && base + t < n; t++) {
                const uint8_t c = src[base + t];
                ok &= c < 20;
                word |= uint32_t(c & 31u) << (5 * t);
            }
            dst[w] = word;
        }
    }
    return ok;
}

// Packs n codes into dst (packed_words(n, alpha) words) with up to 16 host threads; false if
// any code is outside the alphabet.
bool par_pack_check(uint32_t* dst, const uint8_t* src, uint64_t n, int alpha) {
    const size_t words = packed_words(n, alpha);
    const size_t kMinParallel = size_t(2) << 20;   // words
    if (words < kMinParallel) return pack_range(dst, src, n, alpha, 0, words);
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t per = (words + hw - 1) / hw;
    std::atomic<bool> ok{true};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < hw; t++) {
        const size_t a = t * per;
        if (a >= words) break;
        const size_t b = std::min(words, a + per);
        th.emplace_back([&, a, b]() {
            if (!pack_range(dst, src, n, alpha, a, b)) ok = false;
        });
    }
    for (auto& x : th) x.join();
    return ok.load();
}

}  // namespace

// Everything a captured pipeline bakes in: device pointers, sizes, parameters, scratch.
struct GraphKey {
    int alpha;
    uint32_t n_seqs, n_pairs, max_len, delta;
    int32_t zdrop;
    uint64_t n_codes;
    const void *codes, *offsets, *lengths, *pairs, *out, *stream;
    int32_t gap, X;
    int8_t sim[400];
    const void* scratch[11 + kLevels];
    const void* tiers;
};

// One tuned configuration: the register-level chain and its launch parameters for batches of
// one alphabet, X bucket and length bucket.
struct TuneEntry {
    int alpha = 4, xb = 0, lb = 0, sb = 2, db = 0;
    TierConfig cfg{};
    float ms = 0;
};

// The resident sequence store of one alphabet: sequences packed once on the device and kept
// across batches (the paper's detached sequence set, Sec. 4.1.1), deduplicated by content.
struct SeqStore {
    DevBuf words;                        // packed residues
    uint64_t used_words = 0;
    std::vector<uint64_t> off;           // residue position of each sequence
    std::vector<uint32_t> len;
    DevBuf d_off, d_len;                 // the same tables on the device
    std::vector<uint8_t> codes;          // host copy of every stored sequence (exact dedup)
    std::vector<uint64_t> host_off;
    std::unordered_map<uint64_t, std::vector<uint32_t>> by_hash;
};

struct xd_ctx {
    int device = 0;
    int n_sm = 1;
    uint64_t cap = 0;
    uint64_t admitted = 0;       // device bytes of requests not yet finished
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    Scratch dev;                 // scratch of xd_run_device
    uint32_t reserved_len = 0;
    cudaStream_t dev_stream = nullptr;
    bool generic_only = false;
    TierConfig tiers{}, tiers_tiny_x{}, tiers_small_x{}, tiers_large_x{}, tiers_protein{};
    TierConfig tiers_latency{}, tiers_latency_mid{}, tiers_latency_prot{};
    TierConfig tiers_huge{}, tiers_huge_tiny_x{}, tiers_huge_small_x{}, tiers_huge_large_x{};   // DNA launches
                                                                                           // of >= huge_units sides
    uint32_t latency_units = 0;        // batches with fewer side extensions use tiers_latency
    uint32_t huge_units = 0;           // launches with at least this many use tiers_huge
    std::vector<TuneEntry> tuned;      // autotuned configurations by (alphabet, X, length) bucket
    const TierConfig* force_tiers = nullptr;   // set while the autotuner times a candidate
    DevBuf stats;                // uint64 [16]: cumulative per-batch counters (see Problem::stats)
    uint64_t batches = 0, pairs = 0, launches = 0;
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 8>> ev_sets;   // one set per timed batch
    size_t ev_used = 0;
    uint64_t stats_at_enable[16] = {};
    uint64_t launches_at_enable = 0;
    std::string err;
    std::mutex mu;
    // request dispatcher
    bool merge = true;           // merge waiting requests with identical parameters
    uint32_t max_batch_pairs = 1u << 20;
    uint64_t max_batch_codes = uint64_t(24) << 30;   // residue bytes of one merged launch
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> requests;
    std::vector<HostBuf> pinned_cache;
    uint64_t pinned_cached = 0;
    std::condition_variable wake;      // dispatcher: new request or stop
    std::condition_variable finished;  // pollers: a request finished
    std::thread dispatcher;
    bool stop = false;
    bool stop_timed_out = false;
    uint64_t merged_launches = 0, merged_requests = 0, mixed_launches = 0;
    int mix_groups = kSlotGroups;      // parameter sets per launch (1: one set per launch)
    // the fused persistent kernel's blocks wait on one another, so two of them never run at
    // the same time: each waits for the previous one through this event
    cudaEvent_t coop_done = nullptr;
    SeqStore store[2];                 // DNA, protein
    // CUDA graph of the device entry point: a batch that repeats the previous call's
    // arguments exactly is captured once and then replayed
    bool graphs = true;
    GraphKey last_key{}, graph_key{};
    bool have_last = false;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_launches = 0;       // kernels per replay
    uint64_t graph_replays = 0, graph_captures = 0;
    // per-side timeline of xd_run_device batches (xd_set_trace / xd_get_trace)
    bool tracing = false;
    DevBuf trace;
    uint64_t trace_units = 0;          // units of the last traced batch (0: none yet)
    cudaStream_t trace_stream = nullptr;
};

namespace {

thread_local std::string g_create_error;

xd_status fail(xd_ctx* c, xd_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

xd_status cuda_fail(xd_ctx* c, cudaError_t e, const char* what) {
    return fail(c, XD_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

#define XD_CUDA(ctx, call)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int32_t score_max_abs(const int8_t* sim, int alpha, int32_t gap) {
    int32_t m = std::abs(gap);
    for (int t = 0; t < alpha * alpha; t++) m = std::max(m, std::abs(int32_t(sim[t])));
    return std::max(m, 1);
}

// Fill sim / gap / X / delta of a view from the ABI scoring; validates parameters that do
// not need the sequences.
xd_status scoring_view(xd_ctx* c, const xd_batch* b, BatchView& v) {
    if (b->alpha != XD_DNA2 && b->alpha != XD_PROT5) return fail(c, XD_EINVAL, "unknown alphabet");
    if (b->X < 0) return fail(c, XD_EINVAL, "X must be >= 0");
    v.alpha = b->alpha == XD_DNA2 ? 4 : 20;
    if (v.alpha == 4) {
        if (std::abs(b->scoring.match) > 127 || std::abs(b->scoring.mismatch) > 127)
            return fail(c, XD_EINVAL, "DNA scores must lie in [-127, 127]");
        for (int a = 0; a < 4; a++)
            for (int q = 0; q < 4; q++)
                v.sim[a * 4 + q] = int8_t(a == q ? b->scoring.match : b->scoring.mismatch);
    } else {
        if (!b->scoring.matrix20x20) return fail(c, XD_EINVAL, "protein batch without substitution matrix");
        std::memcpy(v.sim, b->scoring.matrix20x20, 400);
    }
    if (b->scoring.gap > 0 || b->scoring.gap < -(1 << 20)) return fail(c, XD_EINVAL, "gap must be a negative score (or 0)");
    v.gap = b->scoring.gap;
    v.X = b->X;
    v.delta = b->delta_b;
    if (b->z_drop < 0) return fail(c, XD_EINVAL, "z_drop must be >= 0");
    v.zdrop = b->z_drop;
    v.max_abs = score_max_abs(v.sim, v.alpha, v.gap);
    v.n_seqs = b->n_seqs;
    v.n_codes = b->n_codes;
    v.n_pairs = b->n_pairs;
    return XD_OK;
}

// Full host-side validation of a host batch; returns max side length on H.
xd_status validate_host(xd_ctx* c, const xd_batch* b, const BatchView& v, uint32_t* max_len) {
    if (b->n_pairs && (!b->pairs || !b->seq_offsets || !b->seq_lengths))
        return fail(c, XD_EINVAL, "null pointer in batch");
    if (b->n_codes && !b->seq_codes) return fail(c, XD_EINVAL, "null seq_codes");
    // residue codes are checked while they are staged (par_copy_check)
    for (uint32_t s = 0; s < b->n_seqs; s++)
        if (b->seq_offsets[s] + b->seq_lengths[s] > b->n_codes)
            return fail(c, XD_EINVAL, "sequence " + std::to_string(s) + " extends past n_codes");
    uint32_t ml = 0;
    for (uint32_t p = 0; p < b->n_pairs; p++) {
        const xd_pair& e = b->pairs[p];
        if (e.h_id >= b->n_seqs || e.v_id >= b->n_seqs)
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": sequence id out of range");
        uint64_t lh = b->seq_lengths[e.h_id], lv = b->seq_lengths[e.v_id];
        if (uint64_t(e.h_seed) + e.seed_len > lh || uint64_t(e.v_seed) + e.seed_len > lv)
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": seed outside its sequence");
        uint64_t rm = lh - e.h_seed - e.seed_len, rn = lv - e.v_seed - e.seed_len;
        if (int64_t(rm + rn) * v.max_abs >= kScoreLimit || int64_t(e.h_seed + e.v_seed) * v.max_abs >= kScoreLimit)
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": scores could exceed 2^29 in magnitude");
        ml = std::max<uint32_t>(ml, uint32_t(std::max<uint64_t>(rm, e.h_seed)));
    }
    *max_len = ml;
    return XD_OK;
}

// Escalation-record pool: 256 ints per unit on average (a 32-slot record takes 80, a
// 512-slot one 1040), at most 256 Mi ints (1 GiB, reached by launches of several batches).
constexpr uint64_t kRecIntsPerUnit = 256;
constexpr uint64_t kRecPoolMax = uint64_t(1) << 28;

struct ScratchPlan {
    size_t store, units, bucket, order, q, generic, rec, rec_of;
    uint32_t rec_cap;
    uint64_t generic_stride;
    int generic_blocks;
};

ScratchPlan plan_scratch(const xd_ctx* c, int alpha, uint64_t n_codes, uint32_t n_pairs, uint32_t max_len) {
    ScratchPlan p{};
    uint64_t per = alpha == 4 ? 16 : 6;
    p.store = ((n_codes + per - 1) / per + 4) * 4;
    uint64_t nu = uint64_t(n_pairs) * 2;
    p.units = nu * sizeof(Unit);
    p.bucket = nu * 4;
    p.order = nu * 4;
    p.q = nu * 4;
    p.rec_cap = uint32_t(std::min<uint64_t>(nu * kRecIntsPerUnit, kRecPoolMax));
    p.rec = size_t(p.rec_cap) * 4;
    p.rec_of = nu * 4;
    p.generic_blocks = c->n_sm * 2;
    p.generic_stride = align_up(uint64_t(max_len) + 1, 32);
    p.generic = size_t(p.generic_blocks) * 4 * 3 * p.generic_stride * 4;
    return p;
}

size_t plan_bytes(const ScratchPlan& p) {
    return p.store + p.units + p.bucket + p.order + kLevels * p.q + p.generic + p.rec + p.rec_of + 4096;
}

cudaError_t ensure_scratch(Scratch& s, const ScratchPlan& p) {
    cudaError_t e;
    if ((e = grow(s.store, p.store)) != cudaSuccess) return e;
    if ((e = grow(s.units, p.units)) != cudaSuccess) return e;
    if ((e = grow(s.bucket, p.bucket)) != cudaSuccess) return e;
    if ((e = grow(s.order, p.order)) != cudaSuccess) return e;
    for (DevBuf& q : s.q)
        if ((e = grow(q, p.q)) != cudaSuccess) return e;
    if ((e = grow(s.ctr, kNumCtr * 4)) != cudaSuccess) return e;
    if ((e = grow(s.hist, 64 * 4)) != cudaSuccess) return e;
    if ((e = grow(s.err, 16)) != cudaSuccess) return e;
    if ((e = grow(s.bstats, 16 * 8)) != cudaSuccess) return e;
    if ((e = grow(s.rec, p.rec)) != cudaSuccess) return e;
    if ((e = grow(s.rec_of, p.rec_of)) != cudaSuccess) return e;
    return grow(s.generic, p.generic);
}

int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

// Register-level chains.  The first level's window should hold the typical live band of
// the batch's X (a few tens of cells for X up to ~30 with DNA scoring); wider bands escalate.
void set_chain(TierConfig& t, std::initializer_list<int> vs) {
    t.n_levels = 0;
    for (int v : vs) t.variant[t.n_levels++] = v;
}

// Comma-separated variant ids into a chain; false if the list is empty.
bool parse_chain(const char* ch, TierConfig& t) {
    int n = 0;
    for (const char* q = ch; *q && n < kLevels - 2;) {
        const int v = std::atoi(q);
        if (v < 0 || v >= kNumGroupVariants) return false;
        t.variant[n++] = v;
        while (*q && *q != ',') q++;
        if (*q == ',') q++;
    }
    if (n == 0) return false;
    t.n_levels = n;
    return true;
}

// Batches with fewer side extensions than this cannot fill the GPU with one lane per side:
// their time is the serial anti-diagonal chain of their longest sides, so they run with a
// full warp per side from the first level (lower latency per anti-diagonal).
constexpr uint32_t kLatencyUnits = 65536;
// Launches with this many side extensions or more (several batches in one pass, or one very
// large batch) are bound by the total work, not by the serial chains of their longest sides
// (the bulk of the others overlaps them), so their wide levels use the fewest lanes per
// side: 4 x 32 and 8 x 32 slots instead of 16 x 16 and 32 x 16.
constexpr uint32_t kHugeUnits = 1u << 20;

void default_tiers(xd_ctx* c) {
    TierConfig& t = c->tiers;
    for (int v = 0; v < kNumGroupVariants; v++) t.blocks_per_sm[v] = 3;
    for (int v : {kG1C32, kG32C32, kG4C32, kG8C32, kG16C32, kG2C32}) t.blocks_per_sm[v] = 2;
    // 8- and 16-slot levels: 128 registers (four blocks per SM) in the packed builds; the
    // 32-bit builds of the 16-slot levels hold three, the rest of their grid runs after
    for (int v : {kG4C8, kG8C8, kG16C8, kG32C8, kG1C16, kG2C16, kG4C16, kG8C16, kG16C16, kG32C16})
        t.blocks_per_sm[v] = 4;
    t.chunk = std::max(1, env_int("XD_CHUNK", 1));
    t.fused = env_int("XD_FUSED", 1) != 0;
    t.every1 = std::max(0, env_int("XD_EVERY1", 8));
    t.every2 = std::max(0, env_int("XD_EVERY2", 32));
    t.every3 = std::max(0, env_int("XD_EVERY3", 64));
    if (t.every1 == 1) t.every1 = 2;   // every warp in role 1 would leave the ordered units to nobody
    if (t.every2 == 1) t.every2 = 2;
    if (t.every3 == 1) t.every3 = 2;
    t.fused_minb = env_int("XD_FUSED_MINB", 2);
    // the longest 0.2% of the sides first, with 8 lanes x 4 slots (measured +3-4% at X = 20)
    t.long_permille = std::max(0, std::min(250, env_int("XD_LONG_PERMILLE", 2)));
    t.long_shape = std::max(0, std::min(2, env_int("XD_LONG_SHAPE", 1)));
    // failure-detection tests: a short wait limit and a producer that never finishes
    t.wait_limit_ms = std::max(0, env_int("XD_TEST_WAIT_MS", 0));
    t.phantom_producer = env_int("XD_TEST_PHANTOM_PRODUCER", 0) != 0;
    t.band_warps = env_int("XD_BAND_WARPS", 8);
    t.fused4 = env_int("XD_FUSED4", 1) != 0;
    set_chain(t, {kG1C32, kG16C16, kG32C16, kG32C32});
    // X <= 15: narrower first windows (measured at X = 10: 20 slots 195, 24 slots 184,
    // 32 slots 152 GCUPS); 20 slots up to X = 12, 24 slots up to X = 15
    c->tiers_small_x = t;
    set_chain(c->tiers_small_x, {kG1C24, kG16C16, kG32C16, kG32C32});
    c->tiers_tiny_x = t;
    set_chain(c->tiers_tiny_x, {kG1C20, kG16C16, kG32C16, kG32C32});
    c->tiers_large_x = t;
    set_chain(c->tiers_large_x, {kG4C16, kG16C16, kG32C32});
    // measured at X = 50: three blocks per SM for its 16-slot levels ahead of four (~1%)
    for (int v : {kG4C16, kG16C16}) c->tiers_large_x.blocks_per_sm[v] = 3;
    c->tiers_large_x.every1 = std::max(0, env_int("XD_EVERY1", 4));
    c->tiers_large_x.every2 = std::max(0, env_int("XD_EVERY2", 16));
    if (c->tiers_large_x.every1 == 1) c->tiers_large_x.every1 = 2;
    if (c->tiers_large_x.every2 == 1) c->tiers_large_x.every2 = 2;
    // X > 30: one launch per level measured faster than the fused grid (451 vs 376 GCUPS at
    // X = 50 on the long-read batch)
    c->tiers_large_x.fused = env_int("XD_FUSED_LARGE", 0) != 0 && t.fused;
    c->tiers_protein = t;
    if (env_int("XD_FUSED_PROT", 1) != 0 && t.fused) {
        // measured on two 1,000,000-pair protein batches per launch: the persistent grid of the
        // 16-slot levels 4 x 16 -> 8 x 16 -> 16 x 16 (128 registers, four blocks per SM), every
        // warp starting in the first level, then 32 x 32: 366 GCUPS against 355 for one launch
        // per level of 4 x 16 -> 8 x 16 -> 32 x 32 (242 with one warp in 8 starting in the second
        // level, 159 with the 32 x 32 level as a fourth role)
        set_chain(c->tiers_protein, {kG4C16, kG8C16, kG16C16, kG32C32});
        c->tiers_protein.fused4 = false;
        c->tiers_protein.every1 = 0;
        c->tiers_protein.every2 = 0;
    } else {
        // one launch per level: 4 x 16 -> 8 x 16 -> 32 x 32 (268 GCUPS on the 32-bit build) ahead
        // of 4 x 16 -> 16 x 16 -> 32 x 32 (248)
        set_chain(c->tiers_protein, {kG4C16, kG8C16, kG32C32});
        c->tiers_protein.fused = false;
    }
    // small batches (measured on long-read and protein batches of 1,000 - 30,000 pairs):
    // DNA below half the threshold 32 lanes x 16 slots, above it 16 x 8 first; protein 32 x 8
    c->tiers_latency = t;
    set_chain(c->tiers_latency, {kG32C16, kG32C32});
    c->tiers_latency.fused = false;
    c->tiers_latency_mid = c->tiers_latency;
    set_chain(c->tiers_latency_mid, {kG16C8, kG32C16, kG32C32});
    c->tiers_latency_prot = c->tiers_latency;
    set_chain(c->tiers_latency_prot, {kG32C8, kG32C32});
    // small batches: the 32 x 16 level with three blocks per SM, as measured for serving
    for (TierConfig* tc : {&c->tiers_latency, &c->tiers_latency_mid, &c->tiers_latency_prot})
        tc->blocks_per_sm[kG32C16] = 3;
    c->latency_units = uint32_t(std::max(0, env_int("XD_LATENCY_UNITS", int(kLatencyUnits))));
    c->huge_units = uint32_t(std::max(0, env_int("XD_HUGE_UNITS", int(kHugeUnits))));
    // huge DNA launches: 1 x 32 -> 4 x 32 -> 8 x 32 in the four-block grid, then 32 x 32 and
    // the band tier (measured on ten long-read batches per launch, X = 10 and 20)
    c->tiers_huge = t;
    set_chain(c->tiers_huge, {kG1C32, kG4C32, kG8C32, kG32C32});
    // four blocks per SM (128 registers, 16 warps per SM): measured 1,019-1,021 GCUPS against
    // 958-967 with three blocks (168 registers) on ten long-read batches per launch, X = 20
    c->tiers_huge.fused_minb = env_int("XD_FUSED_MINB", 4);
    // the 32 x 32 level as a separate launch: a fourth role in the grid (XD_FUSED4_HUGE=1)
    // measured level with it (951 - 984 against 963 GCUPS at X = 20, box noise), and the
    // grid's own rate drops by the wide level's lower fill
    c->tiers_huge.fused4 = env_int("XD_FUSED4_HUGE", 0) != 0 && t.fused4;
    // every warp starts in the first level (the wide sides wait for the bulk of the narrow ones;
    // the other batches of the launch cover their chains)
    c->tiers_huge.every1 = std::max(0, env_int("XD_EVERY1", 0));
    c->tiers_huge.every2 = std::max(0, env_int("XD_EVERY2", 0));
    for (int* e : {&c->tiers_huge.every1, &c->tiers_huge.every2})
        if (*e == 1) *e = 2;
    c->tiers_huge_small_x = c->tiers_huge;
    set_chain(c->tiers_huge_small_x, {kG1C24, kG4C32, kG8C32, kG32C32});
    c->tiers_huge_tiny_x = c->tiers_huge;
    set_chain(c->tiers_huge_tiny_x, {kG1C20, kG4C32, kG8C32, kG32C32});
    // X > 30: the chain of large batches (measured faster than the 32-slot wide levels at X = 50)
    c->tiers_huge_large_x = t;
    // measured on ten long-read batches per launch at X = 50, one launch per level:
    // 4 x 16 -> 8 x 32 -> 16 x 32 -> 32 x 32 (four blocks per SM for the first level) 899 GCUPS,
    // against 708 for the chain of large batches (4 x 16 -> 16 x 16 -> 32 x 32) and 660 for the
    // four-block wide grid of X <= 30
    set_chain(c->tiers_huge_large_x, {kG4C16, kG8C32, kG16C32, kG32C32});
    c->tiers_huge_large_x.fused = false;
    // overrides for experiments: comma-separated variant ids
    if (const char* ch = std::getenv("XD_CHAIN_PROT")) parse_chain(ch, c->tiers_protein);
    if (const char* ch = std::getenv("XD_CHAIN_SMALL")) {
        parse_chain(ch, c->tiers_latency);
        parse_chain(ch, c->tiers_latency_mid);
        parse_chain(ch, c->tiers_latency_prot);
    }
    if (const char* ch = std::getenv("XD_CHAIN_HUGE")) {
        parse_chain(ch, c->tiers_huge);
        c->tiers_huge_small_x = c->tiers_huge_tiny_x = c->tiers_huge;
    }
    if (const char* ch = std::getenv("XD_CHAIN")) {
        TierConfig forced = t;
        if (parse_chain(ch, forced))
            c->tiers = c->tiers_tiny_x = c->tiers_small_x = c->tiers_large_x = c->tiers_huge =
                c->tiers_huge_tiny_x = c->tiers_huge_small_x = c->tiers_huge_large_x = forced;
    }
}

int x_bucket(int32_t X) { return X <= 15 ? 0 : X <= 30 ? 1 : 2; }
int len_bucket(uint32_t max_len) { return max_len <= 2048 ? 0 : max_len <= 20000 ? 1 : 2; }
// Memory-restricted window: 0 unrestricted, 1 up to 512 cells, 2 up to 2048, 3 wider.
int delta_bucket(uint32_t delta) { return delta == 0 ? 0 : delta <= 512 ? 1 : delta <= 2048 ? 2 : 3; }
int size_bucket(uint32_t n_pairs) {
    const uint64_t u = uint64_t(n_pairs) * 2;
    return u < 8192 ? 0 : u < kLatencyUnits ? 1 : u < kHugeUnits ? 2 : 3;
}

const TierConfig& tiers_for(const xd_ctx* c, const BatchView& b) {
    if (c->force_tiers) return *c->force_tiers;
    const int xb = x_bucket(b.X), lb = len_bucket(b.max_len), sb = size_bucket(b.n_pairs);
    const int db = delta_bucket(uint32_t(b.delta));
    for (const TuneEntry& t : c->tuned)
        if (t.alpha == b.alpha && t.xb == xb && t.lb == lb && t.sb == sb && t.db == db) return t.cfg;
    const uint64_t units = uint64_t(b.n_pairs) * 2;
    if (units < c->latency_units) {
        if (b.alpha == 20) return c->tiers_latency_prot;
        return units < c->latency_units / 2 ? c->tiers_latency : c->tiers_latency_mid;
    }
    if (b.alpha == 20) return c->tiers_protein;
    if (units >= c->huge_units)
        return b.X <= 12 ? c->tiers_huge_tiny_x : b.X <= 15 ? c->tiers_huge_small_x
               : b.X <= 30 ? c->tiers_huge : c->tiers_huge_large_x;
    if (b.X <= 12) return c->tiers_tiny_x;
    if (b.X <= 15) return c->tiers_small_x;
    if (b.X <= 30) return c->tiers;
    return c->tiers_large_x;
}

// The hot path of nb batches that share alphabet, scoring, X and delta_b (Sec. 3 method on
// every side extension), all on stream st and in one set of launches: the batches' residues
// are packed into one store (each batch from a word boundary), their side extensions form
// one cost-ordered unit list for the tiers, and batch k's results land at d_out + its first
// pair (the batches' pairs in order).  One batch is the common case (nb = 1).
// chain: an event that orders the fused persistent launches of the context (may be null).
xd_status run_pipeline(xd_ctx* c, Scratch& s, const BatchView* bs, int nb, xd_result* d_out, cudaStream_t st,
                       cudaEvent_t chain) {
    Range range("xd.pipeline");
    const BatchView& b0 = bs[0];
    const uint64_t per_word = b0.alpha == 4 ? 16 : 6;
    // per batch: first pair, first store word; totals over the batches
    std::vector<uint32_t> pair_base(nb);
    std::vector<uint64_t> word_base(nb);
    uint64_t n_pairs_all = 0, words_all = 0, codes_all = 0;
    uint32_t max_len = 0;
    for (int k = 0; k < nb; k++) {
        pair_base[k] = uint32_t(n_pairs_all);
        word_base[k] = words_all;
        n_pairs_all += bs[k].n_pairs;
        words_all += (bs[k].n_codes + per_word - 1) / per_word;
        codes_all += bs[k].n_codes;
        max_len = std::max(max_len, bs[k].max_len);
    }
    if (n_pairs_all >= (uint64_t(1) << 31)) return fail(c, XD_EINVAL, "too many pairs in one launch");
    BatchView b = b0;                  // the parameters, with the sizes of all batches
    b.n_pairs = uint32_t(n_pairs_all);
    b.n_codes = words_all * per_word;
    b.max_len = max_len;
    ScratchPlan plan = plan_scratch(c, b.alpha, b.n_codes, b.n_pairs, b.max_len);
    XD_CUDA(c, ensure_scratch(s, plan));
    bool timed = c->timing && c->ev_used < 4096;
    cudaEvent_t* ev = nullptr;
    if (timed) {
        if (c->ev_used == c->ev_sets.size()) {
            std::array<cudaEvent_t, 8> set{};
            for (auto& e : set) XD_CUDA(c, cudaEventCreate(&e));
            c->ev_sets.push_back(set);
        }
        ev = c->ev_sets[c->ev_used++].data();
    }
    auto mark = [&](int k) -> cudaError_t { return timed ? cudaEventRecord(ev[k], st) : cudaSuccess; };
    XD_CUDA(c, mark(0));
    XD_CUDA(c, cudaMemsetAsync(s.hist.p, 0, 64 * 4, st));
    XD_CUDA(c, cudaMemsetAsync(s.err.p, 0, 4, st));
    XD_CUDA(c, cudaMemsetAsync(s.bstats.p, 0, 16 * 8, st));
    auto* err = static_cast<uint32_t*>(s.err.p);
    const uint32_t* store = b.packed ? b.packed : static_cast<const uint32_t*>(s.store.p);
    if (!b.packed)
        for (int k = 0; k < nb; k++)
            XD_CUDA(c, launch_pack(b.alpha, bs[k].codes, bs[k].n_codes,
                                   static_cast<uint32_t*>(s.store.p) + word_base[k], err, c->n_sm, st));
    XD_CUDA(c, mark(1));
    Problem P{};
    P.store = store;
    P.n_words = b.packed ? std::max<uint64_t>(1, b.packed_words)
                         : std::max<uint64_t>(1, (b.n_codes + (b.alpha == 4 ? 15 : 5)) / (b.alpha == 4 ? 16 : 6));
    P.max_abs = b.max_abs;
    P.s_max = 0;
    for (int e = 0; e < (b.alpha == 4 ? 16 : 400); e++) P.s_max = std::max<int32_t>(P.s_max, b.sim[e]);
    P.units = static_cast<const Unit*>(s.units.p);
    P.results = d_out;
    P.err = err;
    P.stats = static_cast<unsigned long long*>(s.bstats.p);
    P.rec = static_cast<int32_t*>(s.rec.p);
    P.rec_of = static_cast<uint32_t*>(s.rec_of.p);
    P.rec_ctr = static_cast<uint32_t*>(s.ctr.p) + (3 + 2 * kLevels);
    P.rec_cap = plan.rec_cap;
    P.trace = nullptr;
    if (c->tracing && &s == &c->dev && b.n_pairs) {
        const size_t tb = size_t(2) * b.n_pairs * kTraceVisits * sizeof(TraceRec);
        XD_CUDA(c, grow(c->trace, tb));
        XD_CUDA(c, cudaMemsetAsync(c->trace.p, 0, tb, st));
        P.trace = static_cast<TraceRec*>(c->trace.p);
        c->trace_units = uint64_t(2) * b.n_pairs;
        c->trace_stream = st;
    }
    if (b.n_pairs) XD_CUDA(c, cudaMemsetAsync(s.rec_of.p, 0xff, size_t(2) * b.n_pairs * 4, st));
    P.alpha = b.alpha;
    P.gap = b.gap;
    P.X = b.X;
    P.delta = b.delta;
    P.zdrop = b.zdrop;
    std::memcpy(P.sim, b.sim, sizeof(P.sim));
    // residues each batch may address (a resident-store batch: the whole store)
    auto n_res_of = [&](int k) { return b.packed ? b.packed_words * per_word : bs[k].n_codes; };
    for (int k = 0; k < nb; k++)
        XD_CUDA(c, launch_units(bs[k].pairs, bs[k].n_pairs, bs[k].offsets, bs[k].lengths, bs[k].n_seqs, n_res_of(k),
                                b.max_abs, b.max_len, pair_base[k], word_base[k] * per_word,
                                static_cast<Unit*>(s.units.p), static_cast<uint32_t*>(s.bucket.p),
                                static_cast<uint32_t*>(s.hist.p), err, st));
    XD_CUDA(c, mark(2));
    Queues Q{};
    Q.order = static_cast<const uint32_t*>(s.order.p);
    Q.n_units = 2 * b.n_pairs;
    for (int k = 0; k < kLevels; k++) {
        Q.q[k] = static_cast<uint32_t*>(s.q[k].p);
        if (!Q.q[k]) return fail(c, XD_EDEVICE, "escalation queue not allocated");
    }
    Q.ctr = static_cast<uint32_t*>(s.ctr.p);
    XD_CUDA(c, launch_order(static_cast<uint32_t*>(s.hist.p), Q.ctr, kNumCtr,
                            static_cast<const uint32_t*>(s.bucket.p), Q.n_units,
                            static_cast<uint32_t*>(s.order.p), st));
    XD_CUDA(c, mark(3));
    uint64_t launches = 1 + (b.n_pairs ? 1 : 0);   // scan, scatter (with pairs), plus per batch below
    for (int k = 0; k < nb; k++) launches += (bs[k].n_codes ? 1 : 0) + (bs[k].n_pairs ? 1 : 0);   // pack, units
    if (b.n_pairs) {
        if (c->generic_only) {
            XD_CUDA(c, launch_route_all_generic(Q, st));
            launches += 1;
            XD_CUDA(c, mark(4));
            XD_CUDA(c, mark(5));
        } else {
            const TierConfig& tc = tiers_for(c, b);
            int lv = 0;
            const int roles = packed_batch(P) ? fused_roles(tc, b.alpha) : 0;
            if (roles) {
                // the live queues' slots start unpublished
                for (int k = 0; k < roles - 1; k++)
                    XD_CUDA(c, cudaMemsetAsync(Q.q[k], 0xff, sizeof(uint32_t) * size_t(Q.n_units), st));
                if (chain) XD_CUDA(c, cudaStreamWaitEvent(st, chain, 0));
                XD_CUDA(c, launch_fused_levels(P, Q, tc, c->n_sm, st));
                if (chain) XD_CUDA(c, cudaEventRecord(chain, st));
                XD_CUDA(c, mark(4));
                lv = roles;
                launches += 1;
            }
            for (; lv < tc.n_levels; lv++) {
                XD_CUDA(c, launch_level(P, Q, tc, lv, c->n_sm, st));
                if (lv == 0) XD_CUDA(c, mark(4));
                launches += 1;
            }
            XD_CUDA(c, launch_band(P, Q, c->n_sm, tc.band_warps, st));
            launches += 1;
            XD_CUDA(c, mark(5));
        }
        XD_CUDA(c, launch_generic(P, Q, static_cast<int32_t*>(s.generic.p), plan.generic_stride,
                                  plan.generic_blocks, st));
        XD_CUDA(c, mark(6));
        for (int k = 0; k < nb; k++)
            XD_CUDA(c, launch_totals(bs[k].pairs, bs[k].n_pairs, bs[k].offsets, bs[k].lengths, bs[k].n_seqs,
                                     n_res_of(k), pair_base[k], word_base[k] * per_word, P, st));
        launches += 1 + nb;
    } else {
        XD_CUDA(c, mark(4));
        XD_CUDA(c, mark(5));
        XD_CUDA(c, mark(6));
    }
    XD_CUDA(c, mark(7));
    XD_CUDA(c, launch_accumulate(static_cast<const unsigned long long*>(s.bstats.p),
                                 static_cast<unsigned long long*>(c->stats.p), 16, st));
    launches += 1;
    c->launches += launches;
    c->batches += 1;
    c->pairs += b.n_pairs;
    return XD_OK;
}

xd_status run_pipeline(xd_ctx* c, Scratch& s, const BatchView& b, xd_result* d_out, cudaStream_t st,
                       cudaEvent_t chain) {
    return run_pipeline(c, s, &b, 1, d_out, st, chain);
}

// ---------------------------------------------------------------- request dispatcher

constexpr size_t kMaxRequests = 1u << 16;
constexpr uint64_t kPinnedCacheMax = uint64_t(16) << 30;
constexpr size_t kGatherBelow = size_t(1) << 20;   // smaller code arrays are gathered on the host

// Pinned buffers are cached across requests (page-locking memory is slow), in power-of-two
// size classes from 64 KiB.
cudaError_t take_pinned(xd_ctx* c, size_t bytes, HostBuf& out) {
    size_t cls = size_t(1) << 16;
    while (cls < bytes) cls <<= 1;
    for (size_t k = 0; k < c->pinned_cache.size(); k++) {
        if (c->pinned_cache[k].cap != cls) continue;
        out = c->pinned_cache[k];
        c->pinned_cached -= out.cap;
        c->pinned_cache[k] = c->pinned_cache.back();
        c->pinned_cache.pop_back();
        return cudaSuccess;
    }
    out = HostBuf{};
    cudaError_t e = cudaHostAlloc(&out.p, cls, cudaHostAllocDefault);
    if (e == cudaSuccess) out.cap = cls;
    else out.p = nullptr;
    return e;
}

void give_pinned(xd_ctx* c, HostBuf& b) {
    if (!b.p) return;
    c->pinned_cache.push_back(b);
    c->pinned_cached += b.cap;
    b = HostBuf{};
    while (c->pinned_cached > kPinnedCacheMax && !c->pinned_cache.empty()) {
        auto big = std::max_element(c->pinned_cache.begin(), c->pinned_cache.end(),
                                    [](const HostBuf& x, const HostBuf& y) { return x.cap < y.cap; });
        c->pinned_cached -= big->cap;
        cudaFreeHost(big->p);
        c->pinned_cache.erase(big);
    }
}

// Two requests can share a launch when the kernels see the same parameters.
bool same_params(const BatchView& a, const BatchView& b) {
    return a.alpha == b.alpha && a.gap == b.gap && a.X == b.X && a.delta == b.delta && a.zdrop == b.zdrop &&
           std::memcmp(a.sim, b.sim, size_t(a.alpha) * a.alpha) == 0;
}

void finish_request(xd_ctx* c, Request* r, xd_status st, const std::string& msg) {
    r->state = st == XD_OK ? Request::kDone : Request::kFailed;
    r->status = st;
    r->err = msg;
    give_pinned(c, r->in);
    c->admitted -= std::min(c->admitted, uint64_t(r->need));
}

// Launch the oldest waiting request on a free slot, together with later waiting requests
// while the launch stays under the size caps: every request with the oldest one's
// parameters, and requests with other parameters (another alphabet, scoring, X, delta_b or
// Z) as further parameter sets, up to kSlotGroups sets per launch.  The launch has one
// upload and one result copy; each parameter set is one batch of the hot path on a stream of
// its own, so the sets' kernels run side by side on the device (fused persistent grids still
// take turns through coop_done).  Called with the context lock held.
void launch_merged(xd_ctx* c, Slot& slot) {
    Range range("xd.launch");
    struct Group {
        const Request* first = nullptr;
        std::vector<Request*> reqs;
        uint64_t words = 0, seqs = 0, pairs = 0, codes = 0;
        uint32_t max_len = 0;
    };
    std::vector<Group> groups;
    uint64_t n_codes = 0, n_seqs = 0, n_pairs = 0, n_words = 0;
    for (auto it = c->pending.begin(); it != c->pending.end();) {
        Request* r = *it;
        int g = -1;
        bool fits = groups.empty();
        if (!fits && c->merge && n_pairs + r->v.n_pairs <= c->max_batch_pairs &&
            n_codes + r->v.n_codes <= c->max_batch_codes && n_seqs + r->v.n_seqs <= 0xffffffffull) {
            for (size_t k = 0; k < groups.size() && g < 0; k++)
                if (same_params(r->v, groups[k].first->v) && r->pairs_only == groups[k].first->pairs_only) g = int(k);
            fits = g >= 0 || int(groups.size()) < c->mix_groups;
        }
        if (fits) {
            if (g < 0) {
                groups.emplace_back();
                groups.back().first = r;
                g = int(groups.size()) - 1;
            }
            Group& G = groups[size_t(g)];
            G.reqs.push_back(r);
            G.words += r->n_words;
            G.seqs += r->v.n_seqs;
            G.pairs += r->v.n_pairs;
            G.codes += r->v.n_codes;
            G.max_len = std::max(G.max_len, r->v.max_len);
            n_codes += r->v.n_codes;
            n_words += r->n_words;
            n_seqs += r->v.n_seqs;
            n_pairs += r->v.n_pairs;
            it = c->pending.erase(it);
        } else {
            ++it;
        }
        if (!c->merge) break;
    }
    // the requests in launch order: parameter set by parameter set, each set's requests in
    // arrival order, so that every set's words, sequences and pairs are contiguous
    std::vector<Request*> take;
    for (const Group& G : groups) take.insert(take.end(), G.reqs.begin(), G.reqs.end());
    // the requests' packed residues one after the other (each from a word boundary), then the
    // sequence tables and the seed tuples
    const size_t o_offs = align_up(4 * n_words, 256);
    const size_t o_lens = o_offs + align_up(8 * n_seqs, 256);
    const size_t o_pairs = o_lens + align_up(4 * n_seqs, 256);
    const size_t in_bytes = o_pairs + align_up(sizeof(xd_pair) * n_pairs, 256);
    const size_t out_bytes = sizeof(xd_result) * n_pairs + 16;
    cudaStream_t st = slot.stream;
    auto fail_all = [&](xd_status code, const std::string& msg) {
        for (Request* r : take) finish_request(c, r, code, msg);
        c->finished.notify_all();
    };
    auto cuda_err = [&](cudaError_t e, const char* what) {
        fail_all(XD_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = grow(slot.d_in, in_bytes)) != cudaSuccess) return cuda_err(e, "device input buffer");
    if ((e = grow(slot.d_results, out_bytes)) != cudaSuccess) return cuda_err(e, "device result buffer");
    if ((e = grow_pinned(slot.h_out, out_bytes)) != cudaSuccess) return cuda_err(e, "pinned result buffer");
    for (size_t g = 1; g < groups.size(); g++) {
        Slot::Side& sd = slot.side[g - 1];
        if (!sd.stream && (e = cudaStreamCreateWithFlags(&sd.stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_err(e, "parameter-set stream");
        if (!sd.joined && (e = cudaEventCreateWithFlags(&sd.joined, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_err(e, "parameter-set event");
    }
    if (groups.size() > 1 && !slot.uploaded &&
        (e = cudaEventCreateWithFlags(&slot.uploaded, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_err(e, "upload event");
    char* d = static_cast<char*>(slot.d_in.p);
    if (take.size() == 1) {
        // one request: its pinned buffer already has the device layout
        e = cudaMemcpyAsync(d, take[0]->in.p, take[0]->in_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
    } else {
        // small code arrays and all metadata go through the slot's stage buffer, laid out
        // like the device buffer; large code arrays are copied from the requests' buffers
        if ((e = grow_pinned(slot.h_stage, in_bytes)) != cudaSuccess) return cuda_err(e, "pinned stage buffer");
        char* h = static_cast<char*>(slot.h_stage.p);
        uint64_t word_base = 0, seq_base = 0, pair_base = 0;
        size_t run_a = 0, run_b = 0;   // staged word bytes not yet copied
        auto flush_run = [&]() -> cudaError_t {
            cudaError_t e2 = cudaSuccess;
            if (run_b > run_a) e2 = cudaMemcpyAsync(d + run_a, h + run_a, run_b - run_a, cudaMemcpyHostToDevice, st);
            run_a = run_b;
            return e2;
        };
        for (const Group& G : groups) {
            // positions and sequence ids count from the parameter set's first word and sequence
            const uint64_t per_word = G.first->v.alpha == 4 ? 16 : 6;
            const uint64_t g_word0 = word_base, g_seq0 = seq_base;
            for (Request* r : G.reqs) {
                const char* src = static_cast<const char*>(r->in.p);
                const size_t nb = 4 * r->n_words, at = 4 * word_base;
                if (nb >= kGatherBelow) {
                    if ((e = flush_run()) != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
                    e = cudaMemcpyAsync(d + at, src, nb, cudaMemcpyHostToDevice, st);
                    if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
                    run_a = run_b = at + nb;
                } else {
                    std::memcpy(h + at, src, nb);
                    run_b = at + nb;
                }
                const uint64_t code_base = (word_base - g_word0) * per_word;
                auto* offs = reinterpret_cast<uint64_t*>(h + o_offs) + seq_base;
                const auto* r_offs = reinterpret_cast<const uint64_t*>(src + r->o_offs);
                for (uint32_t q = 0; q < r->v.n_seqs; q++) offs[q] = r_offs[q] + code_base;
                std::memcpy(reinterpret_cast<uint32_t*>(h + o_lens) + seq_base, src + r->o_lens, 4ull * r->v.n_seqs);
                auto* prs = reinterpret_cast<xd_pair*>(h + o_pairs) + pair_base;
                const auto* r_prs = reinterpret_cast<const xd_pair*>(src + r->o_pairs);
                const uint32_t id_base = uint32_t(seq_base - g_seq0);
                for (uint32_t q = 0; q < r->v.n_pairs; q++) {
                    prs[q] = r_prs[q];
                    prs[q].h_id += id_base;
                    prs[q].v_id += id_base;
                }
                word_base += r->n_words;
                seq_base += r->v.n_seqs;
                pair_base += r->v.n_pairs;
            }
        }
        if ((e = flush_run()) != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
        e = cudaMemcpyAsync(d + o_offs, h + o_offs, in_bytes - o_offs, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
    }
    if (groups.size() > 1 && (e = cudaEventRecord(slot.uploaded, st)) != cudaSuccess)
        return cuda_err(e, "cudaEventRecord");
    auto* d_res = static_cast<xd_result*>(slot.d_results.p);
    uint64_t word_base = 0, seq_base = 0, pair_base = 0;
    for (size_t g = 0; g < groups.size(); g++) {
        const Group& G = groups[g];
        BatchView v = G.first->v;
        v.n_codes = 0;
        v.n_seqs = uint32_t(G.seqs);
        v.n_pairs = uint32_t(G.pairs);
        v.max_len = G.max_len;
        // packed on the host: the pipeline reads the words directly (no packing kernel)
        v.codes = nullptr;
        v.packed = reinterpret_cast<const uint32_t*>(d + 4 * word_base);
        v.packed_words = std::max<uint64_t>(1, G.words);
        v.offsets = reinterpret_cast<const uint64_t*>(d + o_offs) + seq_base;
        v.lengths = reinterpret_cast<const uint32_t*>(d + o_lens) + seq_base;
        v.pairs = reinterpret_cast<const xd_pair*>(d + o_pairs) + pair_base;
        if (G.first->pairs_only) {
            // seed tuples on the resident store: its packed residues and tables, no upload
            const SeqStore& ss = c->store[v.alpha == 4 ? 0 : 1];
            v.packed = static_cast<const uint32_t*>(ss.words.p);
            v.packed_words = ss.used_words;
            v.offsets = static_cast<const uint64_t*>(ss.d_off.p);
            v.lengths = static_cast<const uint32_t*>(ss.d_len.p);
            v.n_seqs = uint32_t(ss.off.size());
        }
        cudaStream_t gs = g == 0 ? st : slot.side[g - 1].stream;
        Scratch& sc = g == 0 ? slot.s : slot.side[g - 1].s;
        if (g > 0 && (e = cudaStreamWaitEvent(gs, slot.uploaded, 0)) != cudaSuccess)
            return cuda_err(e, "cudaStreamWaitEvent");
        xd_status ps = run_pipeline(c, sc, v, d_res + pair_base, gs, c->coop_done);
        if (ps != XD_OK) return fail_all(ps, c->err);
        // the set's validation word after the results (one word per set)
        e = cudaMemcpyAsync(static_cast<char*>(slot.h_out.p) + out_bytes - 16 + 4 * g, sc.err.p, 4,
                            cudaMemcpyDeviceToHost, gs);
        if (e == cudaSuccess && g > 0) e = cudaEventRecord(slot.side[g - 1].joined, gs);
        if (e == cudaSuccess && g > 0) e = cudaStreamWaitEvent(st, slot.side[g - 1].joined, 0);
        if (e != cudaSuccess) return cuda_err(e, "parameter-set join");
        word_base += G.words;
        seq_base += G.seqs;
        pair_base += G.pairs;
    }
    if ((e = cudaMemcpyAsync(slot.h_out.p, d_res, sizeof(xd_result) * n_pairs, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaEventRecord(slot.done, st)) != cudaSuccess)
        return cuda_err(e, "result copy");
    slot.busy = true;
    slot.n_pairs = uint32_t(n_pairs);
    slot.n_groups = int(groups.size());
    slot.reqs = take;
    slot.pair_base.clear();
    uint32_t base = 0;
    for (Request* r : take) {
        r->state = Request::kLaunched;
        slot.pair_base.push_back(base);
        base += r->v.n_pairs;
    }
    c->merged_launches += 1;
    c->merged_requests += take.size();
    c->mixed_launches += groups.size() > 1 ? 1 : 0;
}

// Copy a finished slot's results to its requests.  Context lock held.
void retire_slot(xd_ctx* c, Slot& slot, cudaError_t status) {
    const size_t out_bytes = sizeof(xd_result) * size_t(slot.n_pairs) + 16;
    uint32_t flags = 0;
    for (int g = 0; status == cudaSuccess && g < slot.n_groups; g++) {
        uint32_t f = 0;
        std::memcpy(&f, static_cast<char*>(slot.h_out.p) + out_bytes - 16 + 4 * g, 4);
        flags |= f;
    }
    for (size_t k = 0; k < slot.reqs.size(); k++) {
        Request* r = slot.reqs[k];
        if (status != cudaSuccess) {
            finish_request(c, r, XD_EDEVICE, std::string("batch failed: ") + cudaGetErrorString(status));
        } else if (flags) {
            finish_request(c, r, XD_EDEVICE, "device validation flags " + std::to_string(flags));
        } else {
            r->out.resize(r->v.n_pairs);
            if (r->v.n_pairs)
                std::memcpy(r->out.data(), static_cast<const xd_result*>(slot.h_out.p) + slot.pair_base[k],
                            sizeof(xd_result) * r->v.n_pairs);
            finish_request(c, r, XD_OK, "");
        }
    }
    slot.reqs.clear();
    slot.busy = false;
}

// The dispatcher thread: retires finished slots and launches waiting requests whenever a
// slot is free, so requests that arrive while others run join the next launch.
void dispatch_loop(xd_ctx* c) {
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(c->mu);
    std::chrono::steady_clock::time_point stop_at{};
    bool stopping = false;
    for (;;) {
        if (c->stop && !stopping) {
            stopping = true;
            stop_at = std::chrono::steady_clock::now();
        }
        bool any_busy = false, retired = false;
        for (Slot& sl : c->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            retire_slot(c, sl, q);
            retired = true;
        }
        if (retired) c->finished.notify_all();
        if (c->stop && !any_busy) break;
        if (stopping && std::chrono::steady_clock::now() - stop_at > std::chrono::seconds(60)) {
            for (Slot& sl : c->slots)
                if (sl.busy) retire_slot(c, sl, cudaErrorLaunchTimeout);
            c->stop_timed_out = true;
            break;
        }
        if (!c->stop) {
            for (Slot& sl : c->slots) {
                if (c->pending.empty()) break;
                if (sl.busy) continue;
                launch_merged(c, sl);
                any_busy = any_busy || sl.busy;
            }
        }
        if (any_busy) c->wake.wait_for(lk, std::chrono::microseconds(40));
        else if (c->pending.empty() && !c->stop) c->wake.wait_for(lk, std::chrono::milliseconds(50));
    }
    // stopping: requests that never launched fail
    for (Request* r : c->pending) finish_request(c, r, XD_EDEVICE, "context destroyed");
    c->pending.clear();
    c->finished.notify_all();
}

// ---------------------------------------------------------------- tuning table

// One line per entry:  alpha=4 xb=1 lb=1 sb=2 db=0 chain=1,4,5,6 chunk=1 fused=1 every1=4 every2=16 every3=0
// minb=2 long=2 band=8 ms=63.2
std::string format_entry(const TuneEntry& t) {
    std::string chain;
    for (int k = 0; k < t.cfg.n_levels; k++) chain += (k ? "," : "") + std::to_string(t.cfg.variant[k]);
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "alpha=%d xb=%d lb=%d sb=%d db=%d chain=%s chunk=%d fused=%d every1=%d every2=%d every3=%d minb=%d "
                  "long=%d band=%d ms=%.4f",
                  t.alpha, t.xb, t.lb, t.sb, t.db, chain.c_str(), t.cfg.chunk, t.cfg.fused ? 1 : 0, t.cfg.every1,
                  t.cfg.every2, t.cfg.every3, t.cfg.fused_minb, t.cfg.long_permille, t.cfg.band_warps, double(t.ms));
    return buf;
}

// Parses one entry over the defaults `base`; false (with a reason) on a malformed line.
bool parse_entry(const std::string& line, const TierConfig& base, TuneEntry& out, std::string& why) {
    out = TuneEntry{};
    out.cfg = base;
    bool have_chain = false;
    size_t p = 0;
    while (p < line.size()) {
        while (p < line.size() && line[p] == ' ') p++;
        size_t e = line.find(' ', p);
        if (e == std::string::npos) e = line.size();
        const std::string tok = line.substr(p, e - p);
        p = e;
        if (tok.empty()) continue;
        const size_t eq = tok.find('=');
        if (eq == std::string::npos) { why = "token without '=': " + tok; return false; }
        const std::string k = tok.substr(0, eq), v = tok.substr(eq + 1);
        if (k == "chain") {
            out.cfg.n_levels = 0;
            for (size_t q = 0; q < v.size();) {
                if (out.cfg.n_levels >= kLevels - 2) { why = "chain too long"; return false; }
                const int id = std::atoi(v.c_str() + q);
                if (id < 0 || id >= kNumGroupVariants) { why = "unknown variant " + std::to_string(id); return false; }
                out.cfg.variant[out.cfg.n_levels++] = id;
                while (q < v.size() && v[q] != ',') q++;
                if (q < v.size()) q++;
            }
            have_chain = out.cfg.n_levels > 0;
        } else {
            const int x = std::atoi(v.c_str());
            if (k == "alpha") out.alpha = x;
            else if (k == "xb") out.xb = x;
            else if (k == "lb") out.lb = x;
            else if (k == "sb") out.sb = x;
            else if (k == "db") out.db = x;
            else if (k == "chunk") out.cfg.chunk = std::max(1, std::min(x, 64));
            else if (k == "fused") out.cfg.fused = x != 0;
            else if (k == "every1") out.cfg.every1 = x == 1 ? 2 : std::max(0, x);   // 1: no warp in role 0
            else if (k == "every2") out.cfg.every2 = x == 1 ? 2 : std::max(0, x);
            else if (k == "every3") out.cfg.every3 = x == 1 ? 2 : std::max(0, x);
            else if (k == "minb") out.cfg.fused_minb = x;
            else if (k == "long") out.cfg.long_permille = std::max(0, std::min(250, x));
            else if (k == "band") out.cfg.band_warps = x;
            else if (k == "ms") out.ms = float(std::atof(v.c_str()));
        }
    }
    if (!have_chain) { why = "entry without chain"; return false; }
    if (out.alpha != 4 && out.alpha != 20) { why = "alpha must be 4 or 20"; return false; }
    if (out.xb < 0 || out.xb > 2 || out.lb < 0 || out.lb > 2 || out.sb < 0 || out.sb > 3 || out.db < 0 ||
        out.db > 3) {
        why = "bucket out of range";
        return false;
    }
    if (out.alpha == 20)
        for (int k = 0; k < out.cfg.n_levels; k++) {
            const int v = out.cfg.variant[k];
            if (!(v == kG1C16 || v == kG4C16 || v == kG8C16 || v == kG16C16 || v == kG32C16 || v == kG32C32 ||
                  v == kG8C8 || v == kG32C8 || v == kG1C32 || v == kG1C24 || v == kG4C8 || v == kG2C32 ||
                  v == kG2C16)) {
                why = "variant " + std::to_string(v) + " is not compiled for protein";
                return false;
            }
        }
    if (out.cfg.fused && fused_roles(out.cfg, out.alpha) == 0) out.cfg.fused = false;
    return true;
}

xd_status load_table(xd_ctx* c, const char* path, std::vector<TuneEntry>& out) {
    out.clear();
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(c, XD_EINVAL, std::string("cannot open tuning table ") + path);
    char buf[1024];
    int ln = 0;
    xd_status st = XD_OK;
    while (std::fgets(buf, sizeof(buf), f)) {
        ln++;
        std::string line(buf);
        while (!line.empty() && (line.back() == '\n' || line.back() == '\r')) line.pop_back();
        if (line.empty() || line[0] == '#') continue;
        TuneEntry t;
        std::string why;
        if (!parse_entry(line, c->tiers, t, why)) {
            st = fail(c, XD_EINVAL, std::string(path) + ":" + std::to_string(ln) + ": " + why);
            break;
        }
        out.push_back(t);
    }
    std::fclose(f);
    return st;
}

void put_entry(std::vector<TuneEntry>& v, const TuneEntry& t) {
    for (TuneEntry& e : v)
        if (e.alpha == t.alpha && e.xb == t.xb && e.lb == t.lb && e.sb == t.sb && e.db == t.db) {
            e = t;
            return;
        }
    v.push_back(t);
}

// Lanes per side extension of a variant (the threads per alignment of its level).
int tier_group_of(int v) {
    switch (v) {
        case kG1C16: case kG1C32: case kG1C24: case kG1C20: return 1;
        case kG2C32: case kG2C16: return 2;
        case kG4C16: case kG4C32: case kG4C8: return 4;
        case kG8C16: case kG8C32: case kG8C8: return 8;
        case kG16C16: case kG16C32: case kG16C8: return 16;
        default: return 32;
    }
}

// Candidate configurations of the autotuner, in stages: the register chain (lanes per side
// and window of every level: the threads per alignment and band tile width), then the
// queue chunk of single-lane levels, then the fused grid's role mix.
std::vector<TierConfig> chain_candidates(const TierConfig& base, int alpha) {
    std::vector<std::vector<int>> chains;
    if (alpha == 4)
        chains = {{kG1C32, kG16C16, kG32C16, kG32C32}, {kG1C16, kG4C16, kG16C16, kG32C32},
                  {kG1C32, kG8C16, kG32C16, kG32C32}, {kG1C32, kG4C32, kG8C32, kG32C32},
                  {kG4C16, kG16C16, kG32C32},         {kG1C16, kG8C16, kG32C16, kG32C32},
                  {kG1C32, kG8C16, kG16C16, kG32C32}, {kG32C16, kG32C32},
                  {kG32C8, kG32C32},                  {kG16C8, kG32C16, kG32C32},
                  {kG8C16, kG32C32},                  {kG1C24, kG16C16, kG32C16, kG32C32},
                  {kG1C32, kG8C16, kG16C16, kG32C16, kG32C32}};
    else
        chains = {{kG4C16, kG16C16, kG32C32}, {kG1C16, kG4C16, kG16C16, kG32C32}, {kG4C16, kG8C16, kG16C16, kG32C32},
                  {kG8C16, kG32C16, kG32C32}, {kG4C16, kG8C16, kG32C16, kG32C32},
                  {kG32C16, kG32C32},         {kG32C8, kG32C32},
                  {kG8C8, kG32C32}};
    std::vector<TierConfig> out;
    for (const auto& ch : chains)
        for (int fused = 1; fused >= 0; fused--) {
            TierConfig t = base;
            t.n_levels = 0;
            for (int v : ch) t.variant[t.n_levels++] = v;
            t.fused = fused != 0;
            if (t.fused && fused_roles(t, alpha) == 0) continue;
            out.push_back(t);
        }
    return out;
}

}  // namespace

extern "C" {

const char* xd_version(void) { return "xdrop-gb300 0.1 (sm_103a)"; }

const char* xd_last_error(const xd_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

xd_status xd_create(const xd_config* cfg, xd_ctx** out) {
    if (!out) return fail(nullptr, XD_EINVAL, "out is NULL");
    *out = nullptr;
    int dev = cfg ? cfg->device : 0;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return fail(nullptr, XD_EDEVICE, "no CUDA device");
    if (dev < 0 || dev >= count) return fail(nullptr, XD_EDEVICE, "device ordinal out of range");
    cudaDeviceProp prop{};
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
        return fail(nullptr, XD_EDEVICE, cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
        return fail(nullptr, XD_EDEVICE, "this build targets sm_103a (GB300); found sm_" +
                                             std::to_string(prop.major) + std::to_string(prop.minor));
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return fail(nullptr, XD_EDEVICE, cudaGetErrorString(e));
    auto* c = new xd_ctx();
    c->device = dev;
    c->n_sm = prop.multiProcessorCount;
    c->cap = cfg && cfg->store_bytes_cap ? cfg->store_bytes_cap : (uint64_t(64) << 30);
    int inflight = cfg && cfg->max_inflight > 0 ? cfg->max_inflight : 3;
    c->slots.resize(inflight);
    c->merge = !(cfg && cfg->batching < 0);
    c->mix_groups = std::max(1, std::min(kSlotGroups, env_int("XD_MIX_GROUPS", kSlotGroups)));
    c->graphs = env_int("XD_GRAPHS", 1) != 0;
    if (cfg && cfg->max_batch_pairs) c->max_batch_pairs = cfg->max_batch_pairs;
    const char* mode = std::getenv("XD_TIERS");
    c->generic_only = mode && std::strcmp(mode, "generic") == 0;
    default_tiers(c);
    if ((e = cudaStreamCreateWithFlags(&c->dev_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->coop_done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = grow(c->stats, 128)) != cudaSuccess || (e = cudaMemset(c->stats.p, 0, 128)) != cudaSuccess) {
        delete c;
        return fail(nullptr, XD_EDEVICE, cudaGetErrorString(e));
    }
    for (Slot& s : c->slots) {
        if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess) {
            delete c;
            return fail(nullptr, XD_EDEVICE, cudaGetErrorString(e));
        }
    }
    if (cfg && cfg->tune_table) {
        std::vector<TuneEntry> t;
        if (load_table(c, cfg->tune_table, t) != XD_OK) {
            const std::string msg = c->err;
            xd_destroy(c);
            return fail(nullptr, XD_EINVAL, msg);
        }
        c->tuned = t;
    }
    c->dispatcher = std::thread(dispatch_loop, c);
    *out = c;
    return XD_OK;
}

xd_status xd_reserve(xd_ctx* c, uint64_t n_codes, uint32_t n_seqs, uint32_t n_pairs, uint32_t max_seq_len) {
    if (!c) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    (void)n_seqs;
    XD_CUDA(c, cudaSetDevice(c->device));
    c->reserved_len = std::max(c->reserved_len, max_seq_len);
    // reserve for the larger alphabet footprint (DNA packs 16 residues per word, protein 6)
    ScratchPlan p = plan_scratch(c, 20, n_codes, n_pairs, c->reserved_len);
    XD_CUDA(c, ensure_scratch(c->dev, p));
    return XD_OK;
}

xd_status xd_run_device(xd_ctx* c, const xd_batch* b, xd_result* d_out, void* stream) {
    if (!c || !b) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    BatchView v;
    xd_status s = scoring_view(c, b, v);
    if (s != XD_OK) return s;
    if (b->n_pairs && (!b->pairs || !b->seq_offsets || !b->seq_lengths || !d_out))
        return fail(c, XD_EINVAL, "null device pointer in batch");
    if (b->n_codes && !b->seq_codes) return fail(c, XD_EINVAL, "null seq_codes");
    v.codes = b->seq_codes;
    v.offsets = b->seq_offsets;
    v.lengths = b->seq_lengths;
    v.pairs = b->pairs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (c->reserved_len == 0 && b->n_seqs) {
        // no reservation: size the generic scratch from the actual lengths (synchronous)
        std::vector<uint32_t> lens(b->n_seqs);
        XD_CUDA(c, cudaMemcpyAsync(lens.data(), b->seq_lengths, 4ull * b->n_seqs, cudaMemcpyDeviceToHost, st));
        XD_CUDA(c, cudaStreamSynchronize(st));
        v.max_len = *std::max_element(lens.begin(), lens.end());
    } else {
        v.max_len = c->reserved_len;
    }
    // order the fused launch after the host batches' ones (not possible inside a capture,
    // where the caller orders its graphs)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    XD_CUDA(c, cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return run_pipeline(c, c->dev, v, d_out, st, nullptr);
    if (!c->graphs || c->timing || c->tracing || st == nullptr)
        return run_pipeline(c, c->dev, v, d_out, st, c->coop_done);
    // the scratch must be in place before a capture (no allocation inside one)
    const ScratchPlan plan = plan_scratch(c, v.alpha, v.n_codes, v.n_pairs, v.max_len);
    XD_CUDA(c, ensure_scratch(c->dev, plan));
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.alpha = v.alpha;
    k.n_seqs = v.n_seqs;
    k.n_pairs = v.n_pairs;
    k.max_len = v.max_len;
    k.delta = v.delta;
    k.zdrop = v.zdrop;
    k.n_codes = v.n_codes;
    k.codes = v.codes;
    k.offsets = v.offsets;
    k.lengths = v.lengths;
    k.pairs = v.pairs;
    k.out = d_out;
    k.stream = st;
    k.gap = v.gap;
    k.X = v.X;
    std::memcpy(k.sim, v.sim, sizeof(k.sim));
    const Scratch& sc = c->dev;
    const void* bufs[11] = {sc.store.p, sc.units.p, sc.bucket.p, sc.order.p, sc.ctr.p, sc.hist.p,
                            sc.err.p, sc.generic.p, sc.bstats.p, sc.rec.p, sc.rec_of.p};
    std::memcpy(k.scratch, bufs, sizeof(bufs));
    for (int q = 0; q < kLevels; q++) k.scratch[11 + q] = sc.q[q].p;
    k.tiers = &tiers_for(c, v);
    if (c->graph_exec && std::memcmp(&k, &c->graph_key, sizeof(k)) == 0) {
        XD_CUDA(c, cudaStreamWaitEvent(st, c->coop_done, 0));
        XD_CUDA(c, cudaGraphLaunch(c->graph_exec, st));
        XD_CUDA(c, cudaEventRecord(c->coop_done, st));
        c->graph_replays += 1;
        c->launches += c->graph_launches;
        c->batches += 1;
        c->pairs += v.n_pairs;
        return XD_OK;
    }
    const bool repeat = c->have_last && std::memcmp(&k, &c->last_key, sizeof(k)) == 0;
    c->last_key = k;
    c->have_last = true;
    if (!repeat) return run_pipeline(c, c->dev, v, d_out, st, c->coop_done);
    // the second identical call: capture the pipeline, then launch the graph
    const uint64_t launches0 = c->launches, batches0 = c->batches, pairs0 = c->pairs;
    XD_CUDA(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const xd_status ps = run_pipeline(c, c->dev, v, d_out, st, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    cudaGraphExec_t exec = nullptr;
    if (ps == XD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    c->batches = batches0;
    c->pairs = pairs0;
    const uint64_t per = c->launches - launches0;
    c->launches = launches0;
    if (ps != XD_OK || e != cudaSuccess) {
        // this pipeline cannot be captured here: keep launching it directly
        cudaGetLastError();
        c->graphs = false;
        return run_pipeline(c, c->dev, v, d_out, st, c->coop_done);
    }
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = exec;
    c->graph_key = k;
    c->graph_launches = per;
    c->graph_captures += 1;
    XD_CUDA(c, cudaStreamWaitEvent(st, c->coop_done, 0));
    XD_CUDA(c, cudaGraphLaunch(exec, st));
    XD_CUDA(c, cudaEventRecord(c->coop_done, st));
    c->launches += per;
    c->batches += 1;
    c->pairs += v.n_pairs;
    return XD_OK;
}

xd_status xd_run_device_many(xd_ctx* c, uint32_t n_batches, const xd_batch* batches, xd_result* d_out,
                             void* stream) {
    if (!c || (n_batches && !batches)) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    if (n_batches == 0) return XD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<BatchView> vs(n_batches);
    uint64_t pairs = 0;
    for (uint32_t k = 0; k < n_batches; k++) {
        const xd_batch* b = &batches[k];
        BatchView& v = vs[k];
        xd_status s = scoring_view(c, b, v);
        if (s != XD_OK) return s;
        if (k > 0 && !same_params(vs[0], v))
            return fail(c, XD_EINVAL, "the batches of one call must share alphabet, scoring, X, delta_b and z_drop");
        if (b->n_pairs && (!b->pairs || !b->seq_offsets || !b->seq_lengths || !d_out))
            return fail(c, XD_EINVAL, "null device pointer in batch " + std::to_string(k));
        if (b->n_codes && !b->seq_codes) return fail(c, XD_EINVAL, "null seq_codes in batch " + std::to_string(k));
        v.codes = b->seq_codes;
        v.offsets = b->seq_offsets;
        v.lengths = b->seq_lengths;
        v.pairs = b->pairs;
        pairs += b->n_pairs;
        if (c->reserved_len == 0 && b->n_seqs) {
            // no reservation: size the generic scratch from the actual lengths (synchronous)
            std::vector<uint32_t> lens(b->n_seqs);
            XD_CUDA(c, cudaMemcpyAsync(lens.data(), b->seq_lengths, 4ull * b->n_seqs, cudaMemcpyDeviceToHost, st));
            XD_CUDA(c, cudaStreamSynchronize(st));
            v.max_len = *std::max_element(lens.begin(), lens.end());
        } else {
            v.max_len = c->reserved_len;
        }
    }
    if (pairs >= (uint64_t(1) << 31)) return fail(c, XD_EINVAL, "too many pairs in one call");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    XD_CUDA(c, cudaStreamIsCapturing(st, &cs));
    return run_pipeline(c, c->dev, vs.data(), int(n_batches), d_out, st,
                        cs != cudaStreamCaptureStatusNone ? nullptr : c->coop_done);
}

xd_status xd_device_status(xd_ctx* c, uint32_t* flags) {
    if (!c || !flags) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    XD_CUDA(c, cudaDeviceSynchronize());
    *flags = 0;
    if (c->dev.err.p) XD_CUDA(c, cudaMemcpy(flags, c->dev.err.p, 4, cudaMemcpyDeviceToHost));
    return XD_OK;
}

xd_status xd_store_add(xd_ctx* c, xd_alphabet alpha, uint32_t n_seqs, uint64_t n_codes, const uint8_t* seq_codes,
                       const uint64_t* seq_offsets, const uint32_t* seq_lengths, uint32_t* handles) {
    if (!c || (n_seqs && (!seq_offsets || !seq_lengths || !handles)) || (n_codes && !seq_codes)) return XD_EINVAL;
    if (alpha != XD_DNA2 && alpha != XD_PROT5) return fail(c, XD_EINVAL, "unknown alphabet");
    std::unique_lock<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    const int A = alpha == XD_DNA2 ? 4 : 20;
    const uint64_t per = A == 4 ? 16 : 6;
    SeqStore& ss = c->store[alpha == XD_DNA2 ? 0 : 1];
    for (uint32_t q = 0; q < n_seqs; q++)
        if (seq_offsets[q] + seq_lengths[q] > n_codes)
            return fail(c, XD_EINVAL, "sequence " + std::to_string(q) + " extends past n_codes");
    if (!codes_valid(seq_codes, n_codes, A)) return fail(c, XD_EINVAL, "residue code outside the alphabet");
    // deduplicate by content (hash, then exact comparison with the host copy)
    std::vector<uint8_t> fresh;
    std::vector<std::pair<uint32_t, uint64_t>> placed;   // new id, offset in fresh
    const uint32_t first_new = uint32_t(ss.off.size());
    std::vector<uint32_t> out(n_seqs);
    std::unordered_map<uint64_t, std::vector<uint32_t>> pending_hash;   // within this call
    for (uint32_t q = 0; q < n_seqs; q++) {
        const uint8_t* src = seq_codes + seq_offsets[q];
        const uint32_t L = seq_lengths[q];
        uint64_t h = 1469598103934665603ull ^ L;
        for (uint32_t t = 0; t < L; t++) h = (h ^ src[t]) * 1099511628211ull;
        int64_t found = -1;
        if (auto it = ss.by_hash.find(h); it != ss.by_hash.end())
            for (uint32_t id : it->second)
                if (ss.len[id] == L && std::memcmp(ss.codes.data() + ss.host_off[id], src, L) == 0) { found = id; break; }
        if (found < 0)
            if (auto it = pending_hash.find(h); it != pending_hash.end())
                for (uint32_t id : it->second) {
                    const uint64_t o = placed[id - first_new].second;
                    if (ss.len[id] == L && std::memcmp(fresh.data() + o, src, L) == 0) { found = id; break; }
                }
        if (found < 0) {
            const uint32_t id = uint32_t(ss.off.size());
            placed.push_back({id, uint64_t(fresh.size())});
            fresh.insert(fresh.end(), src, src + L);
            ss.len.push_back(L);
            ss.off.push_back(0);           // set below
            ss.host_off.push_back(0);
            pending_hash[h].push_back(id);
            found = id;
        }
        out[q] = uint32_t(found);
    }
    const uint32_t n_new = uint32_t(ss.off.size()) - first_new;
    if (n_new) {
        const uint64_t words = (fresh.size() + per - 1) / per;
        const uint64_t add_bytes = words * 4 + 12ull * n_new;
        if (c->admitted + add_bytes > c->cap) {
            ss.len.resize(first_new);
            ss.off.resize(first_new);
            ss.host_off.resize(first_new);
            return fail(c, XD_ENOMEM, "the resident store would exceed the device memory cap");
        }
        c->admitted += add_bytes;   // the store stays admitted for the context's lifetime
        // growing a device buffer frees the old one: wait for every launch that may read it
        auto grow_keep = [&](DevBuf& b, size_t need, size_t keep) -> cudaError_t {
            if (need <= b.cap) return cudaSuccess;
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return e;
            DevBuf nb;
            e = grow(nb, std::max(need, 2 * b.cap));
            if (e == cudaSuccess && keep) e = cudaMemcpy(nb.p, b.p, keep, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) {
                release(nb);
                return e;
            }
            release(b);
            b = nb;
            return cudaSuccess;
        };
        const uint64_t base_word = ss.used_words;
        XD_CUDA(c, grow_keep(ss.words, (base_word + words + 4) * 4, base_word * 4));
        XD_CUDA(c, grow_keep(ss.d_off, ss.off.size() * 8, first_new * 8ull));
        XD_CUDA(c, grow_keep(ss.d_len, ss.len.size() * 4, first_new * 4ull));
        for (const auto& pl : placed) {
            ss.off[pl.first] = base_word * per + pl.second;
            ss.host_off[pl.first] = ss.codes.size() + pl.second;
        }
        ss.codes.insert(ss.codes.end(), fresh.begin(), fresh.end());
        for (auto& kv : pending_hash)
            for (uint32_t id : kv.second) ss.by_hash[kv.first].push_back(id);
        // upload and pack the new residues behind the stored ones
        DevBuf tmp, terr;
        cudaError_t e = grow(tmp, fresh.size() + 16);
        if (e == cudaSuccess) e = grow(terr, 16);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.p, fresh.data(), fresh.size(), cudaMemcpyHostToDevice, c->dev_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(terr.p, 0, 4, c->dev_stream);
        if (e == cudaSuccess && !fresh.empty())
            e = launch_pack(A, static_cast<const uint8_t*>(tmp.p), fresh.size(),
                            static_cast<uint32_t*>(ss.words.p) + base_word, static_cast<uint32_t*>(terr.p),
                            c->n_sm, c->dev_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<uint64_t*>(ss.d_off.p) + first_new, ss.off.data() + first_new,
                                8ull * n_new, cudaMemcpyHostToDevice, c->dev_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<uint32_t*>(ss.d_len.p) + first_new, ss.len.data() + first_new,
                                4ull * n_new, cudaMemcpyHostToDevice, c->dev_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->dev_stream);
        release(tmp);
        release(terr);
        XD_CUDA(c, e);
        ss.used_words = base_word + words;
    }
    std::memcpy(handles, out.data(), 4ull * n_seqs);
    return XD_OK;
}

xd_status xd_store_info(const xd_ctx* c, xd_alphabet alpha, uint64_t* n_seqs, uint64_t* device_bytes) {
    if (!c || (alpha != XD_DNA2 && alpha != XD_PROT5)) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(const_cast<xd_ctx*>(c)->mu);
    const SeqStore& ss = c->store[alpha == XD_DNA2 ? 0 : 1];
    if (n_seqs) *n_seqs = ss.off.size();
    if (device_bytes) *device_bytes = ss.words.cap + ss.d_off.cap + ss.d_len.cap;
    return XD_OK;
}

xd_status xd_submit_pairs(xd_ctx* c, const xd_pairs_batch* pb, uint64_t* ticket) {
    if (!c || !pb || !ticket) return XD_EINVAL;
    if (pb->n_pairs && !pb->pairs) return fail(c, XD_EINVAL, "null pairs");
    std::unique_lock<std::mutex> lk(c->mu);
    xd_batch b{};
    b.alpha = pb->alpha;
    b.n_pairs = pb->n_pairs;
    b.pairs = pb->pairs;
    b.scoring = pb->scoring;
    b.X = pb->X;
    b.delta_b = pb->delta_b;
    b.z_drop = pb->z_drop;
    BatchView v;
    xd_status s = scoring_view(c, &b, v);
    if (s != XD_OK) return s;
    const SeqStore& ss = c->store[v.alpha == 4 ? 0 : 1];
    uint32_t ml = 0;
    for (uint32_t p = 0; p < pb->n_pairs; p++) {
        const xd_pair& e = pb->pairs[p];
        if (e.h_id >= ss.len.size() || e.v_id >= ss.len.size())
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": handle not in the resident store");
        const uint64_t lh = ss.len[e.h_id], lv = ss.len[e.v_id];
        if (uint64_t(e.h_seed) + e.seed_len > lh || uint64_t(e.v_seed) + e.seed_len > lv)
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": seed outside its sequence");
        const uint64_t rm = lh - e.h_seed - e.seed_len, rn = lv - e.v_seed - e.seed_len;
        if (int64_t(rm + rn) * v.max_abs >= kScoreLimit || int64_t(e.h_seed + e.v_seed) * v.max_abs >= kScoreLimit)
            return fail(c, XD_EINVAL, "pair " + std::to_string(p) + ": scores could exceed 2^29 in magnitude");
        ml = std::max<uint32_t>(ml, uint32_t(std::max<uint64_t>(rm, e.h_seed)));
    }
    v.max_len = ml;
    v.n_seqs = 0;
    v.n_codes = 0;
    const size_t in_bytes = align_up(sizeof(xd_pair) * pb->n_pairs, 256);
    const size_t out_bytes = sizeof(xd_result) * size_t(pb->n_pairs) + 16;
    const ScratchPlan plan = plan_scratch(c, v.alpha, 0, pb->n_pairs, ml);
    const size_t need = in_bytes + out_bytes + plan_bytes(plan) - plan.generic;
    if (c->admitted + need > c->cap) return fail(c, XD_ENOMEM, "batch does not fit the device memory cap now");
    if (c->requests.size() >= kMaxRequests) return fail(c, XD_ENOMEM, "too many requests outstanding");
    auto* r = new Request();
    r->v = v;
    r->pairs_only = true;
    r->o_offs = r->o_lens = r->o_pairs = 0;
    r->in_bytes = in_bytes;
    r->n_words = 0;
    r->need = need;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = take_pinned(c, in_bytes, r->in);
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(c, e, "pinned staging buffer");
    }
    std::memcpy(r->in.p, pb->pairs, sizeof(xd_pair) * pb->n_pairs);
    c->admitted += need;
    r->ticket = c->next_ticket++;
    c->requests[r->ticket] = r;
    c->pending.push_back(r);
    *ticket = r->ticket;
    c->wake.notify_one();
    return XD_OK;
}

xd_status xd_submit_batch(xd_ctx* c, const xd_batch* b, uint64_t* ticket) {
    if (!c || !b || !ticket) return XD_EINVAL;
    Range range("xd.submit");
    std::unique_lock<std::mutex> lk(c->mu);
    BatchView v;
    xd_status s = scoring_view(c, b, v);
    if (s != XD_OK) return s;
    uint32_t max_len = 0;
    if ((s = validate_host(c, b, v, &max_len)) != XD_OK) return s;
    v.max_len = max_len;
    // the residues are packed while they are staged (the device store's layout), so the
    // upload is a quarter (DNA) or five eighths (protein) of the codes
    const size_t words = packed_words(b->n_codes, v.alpha);
    // admission by device memory: inputs, results and the scratch of a batch this size
    const size_t o_offs = align_up(4 * words, 256);
    const size_t o_lens = o_offs + align_up(8ull * b->n_seqs, 256);
    const size_t o_pairs = o_lens + align_up(4ull * b->n_seqs, 256);
    const size_t in_bytes = o_pairs + align_up(sizeof(xd_pair) * b->n_pairs, 256);
    const size_t out_bytes = sizeof(xd_result) * size_t(b->n_pairs) + 16;
    // (the band rows of the generic tier belong to the launch slot, not to the batch)
    const ScratchPlan plan = plan_scratch(c, v.alpha, b->n_codes, b->n_pairs, max_len);
    const size_t need = in_bytes + out_bytes + plan_bytes(plan) - plan.generic;
    if (c->admitted + need > c->cap)
        return fail(c, XD_ENOMEM, "batch needs " + std::to_string(need) + " device bytes; " +
                                      std::to_string(c->cap - std::min(c->cap, c->admitted)) + " available under the cap");
    if (c->requests.size() >= kMaxRequests) return fail(c, XD_ENOMEM, "too many requests outstanding");
    auto* r = new Request();
    r->v = v;
    r->o_offs = o_offs;
    r->o_lens = o_lens;
    r->o_pairs = o_pairs;
    r->in_bytes = in_bytes;
    r->n_words = words;
    r->need = need;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = take_pinned(c, in_bytes, r->in);
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(c, e, "pinned staging buffer");
    }
    c->admitted += need;
    // copy (and check the residue codes) without the lock: the caller may free its arrays
    // when this returns
    lk.unlock();
    char* h = static_cast<char*>(r->in.p);
    const bool codes_ok = par_pack_check(reinterpret_cast<uint32_t*>(h), b->seq_codes, b->n_codes, v.alpha);
    if (codes_ok) {
        std::memcpy(h + o_offs, b->seq_offsets, 8ull * b->n_seqs);
        std::memcpy(h + o_lens, b->seq_lengths, 4ull * b->n_seqs);
        std::memcpy(h + o_pairs, b->pairs, sizeof(xd_pair) * b->n_pairs);
    }
    lk.lock();
    if (!codes_ok) {
        size_t t = 0;
        while (t < b->n_codes && b->seq_codes[t] < v.alpha) t++;
        finish_request(c, r, XD_EINVAL, "");
        delete r;
        return fail(c, XD_EINVAL, "residue code outside the alphabet at byte " + std::to_string(t));
    }
    r->ticket = c->next_ticket++;
    c->requests[r->ticket] = r;
    c->pending.push_back(r);
    *ticket = r->ticket;
    c->wake.notify_one();
    return XD_OK;
}

xd_status xd_poll(xd_ctx* c, uint64_t ticket, xd_result* out, int32_t wait_ms) {
    if (!c) return XD_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->requests.find(ticket);
    if (it == c->requests.end()) return fail(c, XD_ENOTFOUND, "unknown ticket " + std::to_string(ticket));
    Request* r = it->second;
    auto finished = [&]() { return r->state == Request::kDone || r->state == Request::kFailed; };
    if (!finished()) {
        if (wait_ms == 0) return XD_PENDING;
        if (wait_ms < 0) {
            c->finished.wait(lk, finished);
        } else if (!c->finished.wait_for(lk, std::chrono::milliseconds(wait_ms), finished)) {
            return fail(c, XD_ETIMEDOUT, "batch still running");
        }
    }
    c->requests.erase(it);
    if (r->state == Request::kFailed) {
        xd_status st = r->status;
        std::string msg = r->err;
        delete r;
        return fail(c, st, msg);
    }
    lk.unlock();
    if (out && !r->out.empty()) par_memcpy(out, r->out.data(), sizeof(xd_result) * r->out.size());
    delete r;
    return XD_OK;
}

xd_status xd_get_stats(const xd_ctx* c, xd_stats* out) {
    if (!c || !out) return XD_EINVAL;
    std::memset(out, 0, sizeof(*out));
    uint64_t dev[16] = {};
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->stats.p) cudaMemcpy(dev, c->stats.p, 128, cudaMemcpyDeviceToHost);
    std::lock_guard<std::mutex> lk(const_cast<xd_ctx*>(c)->mu);
    out->batches = c->batches;
    out->pairs = c->pairs;
    out->units_tier[0] = dev[0];
    out->units_tier[1] = dev[1];
    out->units_tier[2] = dev[2];
    out->escalations = dev[3];
    out->cells = dev[4] + dev[5] + dev[6];
    out->kernel_launches = c->launches;
    out->host_launches = c->merged_launches;
    out->host_requests = c->merged_requests;
    out->graph_captures = c->graph_captures;
    out->graph_replays = c->graph_replays;
    out->mixed_launches = c->mixed_launches;
    return XD_OK;
}

xd_status xd_set_timing(xd_ctx* c, int32_t enable) {
    if (!c) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    if (enable) {
        XD_CUDA(c, cudaDeviceSynchronize());
        XD_CUDA(c, cudaMemcpy(c->stats_at_enable, c->stats.p, 128, cudaMemcpyDeviceToHost));
        c->launches_at_enable = c->launches;
        c->ev_used = 0;
    }
    c->timing = enable != 0;
    return XD_OK;
}

xd_status xd_get_timing(xd_ctx* c, xd_timing* out) {
    if (!c || !out) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->ev_used == 0) return fail(c, XD_ENOTFOUND, "no timed batch");
    XD_CUDA(c, cudaSetDevice(c->device));
    XD_CUDA(c, cudaDeviceSynchronize());
    std::memset(out, 0, sizeof(*out));
    float* stage[7] = {&out->pack_ms, &out->units_ms, &out->order_ms, &out->tier_ms[0],
                       &out->tier_ms[1], &out->tier_ms[2], &out->totals_ms};
    for (size_t b = 0; b < c->ev_used; b++) {
        const auto& ev = c->ev_sets[b];
        for (int k = 1; k < 8; k++) {
            float t = 0;
            XD_CUDA(c, cudaEventElapsedTime(&t, ev[k - 1], ev[k]));
            *stage[k - 1] += t;
        }
        float t = 0;
        XD_CUDA(c, cudaEventElapsedTime(&t, ev[0], ev[7]));
        out->total_ms += t;
    }
    out->batches = c->ev_used;
    uint64_t d[16] = {};
    XD_CUDA(c, cudaMemcpy(d, c->stats.p, 128, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 16; k++) d[k] -= c->stats_at_enable[k];
    for (int k = 0; k < 3; k++) {
        out->tier_units[k] = d[k];
        out->tier_cells[k] = d[4 + k];
    }
    out->escalations = d[3];
    out->discarded_cells = d[7];
    out->window_shifts = d[8];
    out->register_band_cells = d[9];
    out->register_slot_cells = d[10];
    out->launches = c->launches - c->launches_at_enable;
    return XD_OK;
}

xd_status xd_set_trace(xd_ctx* c, int32_t enable) {
    if (!c) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->tracing = enable != 0;
    return XD_OK;
}

xd_status xd_get_trace(xd_ctx* c, void* out, uint64_t capacity, uint64_t* n_units) {
    if (!c || (capacity && !out)) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->trace_units == 0) return fail(c, XD_ENOTFOUND, "no traced batch");
    XD_CUDA(c, cudaSetDevice(c->device));
    XD_CUDA(c, cudaStreamSynchronize(c->trace_stream));
    const uint64_t bytes = c->trace_units * kTraceVisits * sizeof(TraceRec);
    if (n_units) *n_units = c->trace_units;
    if (capacity) XD_CUDA(c, cudaMemcpy(out, c->trace.p, std::min(bytes, capacity), cudaMemcpyDeviceToHost));
    return XD_OK;
}

xd_status xd_probe(xd_ctx* c, int32_t op, double* rate) {
    if (!c || !rate) return XD_EINVAL;
    if (!((op >= 0 && op <= 10) || (op >= 100 && op <= 103))) return fail(c, XD_EINVAL, "unknown probe op");
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    XD_CUDA(c, cudaDeviceSynchronize());
    float ms = 0;
    XD_CUDA(c, probe_rate(op, c->n_sm, rate, &ms));
    return XD_OK;
}

xd_status xd_autotune(xd_ctx* c, const xd_batch* b, const char* path, float* best_ms) {
    if (!c || !b) return XD_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    BatchView v;
    xd_status s = scoring_view(c, b, v);
    if (s != XD_OK) return s;
    uint32_t max_len = 0;
    if ((s = validate_host(c, b, v, &max_len)) != XD_OK) return s;
    if (b->n_pairs == 0) return fail(c, XD_EINVAL, "empty tuning sample");
    for (uint64_t t = 0; t < b->n_codes; t++)
        if (b->seq_codes[t] >= v.alpha) return fail(c, XD_EINVAL, "residue code outside the alphabet");
    v.max_len = max_len;
    // the sample on the device, with its own scratch and stream
    const size_t o_offs = align_up(b->n_codes, 256);
    const size_t o_lens = o_offs + align_up(8ull * b->n_seqs, 256);
    const size_t o_pairs = o_lens + align_up(4ull * b->n_seqs, 256);
    const size_t in_bytes = o_pairs + align_up(sizeof(xd_pair) * b->n_pairs, 256);
    const size_t out_bytes = sizeof(xd_result) * size_t(b->n_pairs);
    DevBuf d_in, d_out;
    Scratch sc;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<char> h(in_bytes);
    std::vector<xd_result> ref(b->n_pairs), got(b->n_pairs);
    std::memcpy(h.data(), b->seq_codes, b->n_codes);
    std::memcpy(h.data() + o_offs, b->seq_offsets, 8ull * b->n_seqs);
    std::memcpy(h.data() + o_lens, b->seq_lengths, 4ull * b->n_seqs);
    std::memcpy(h.data() + o_pairs, b->pairs, sizeof(xd_pair) * b->n_pairs);
    auto cleanup = [&]() {
        c->force_tiers = nullptr;
        if (st) cudaStreamSynchronize(st);
        release(d_in);
        release(d_out);
        release(sc);
        if (st) cudaStreamDestroy(st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    auto cuda_bail = [&](cudaError_t e, const char* what) {
        cleanup();
        return cuda_fail(c, e, what);
    };
    cudaError_t e;
    if ((e = grow(d_in, in_bytes)) != cudaSuccess || (e = grow(d_out, out_bytes)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_in.p, h.data(), in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_bail(e, "autotune setup");
    char* d = static_cast<char*>(d_in.p);
    v.codes = reinterpret_cast<const uint8_t*>(d);
    v.offsets = reinterpret_cast<const uint64_t*>(d + o_offs);
    v.lengths = reinterpret_cast<const uint32_t*>(d + o_lens);
    v.pairs = reinterpret_cast<const xd_pair*>(d + o_pairs);
    auto* res = static_cast<xd_result*>(d_out.p);
    const bool timing = c->timing;
    c->timing = false;
    bool have_ref = false;
    // time one candidate: a warm-up run, then the best of two; results must not change
    auto run = [&](const TierConfig& cand, float& ms) -> xd_status {
        c->force_tiers = &cand;
        ms = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaError_t ee = cudaEventRecord(e0, st);
            if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaEventRecord");
            xd_status ps = run_pipeline(c, sc, v, res, st, c->coop_done);
            if (ps != XD_OK) return ps;
            if ((ee = cudaEventRecord(e1, st)) != cudaSuccess || (ee = cudaEventSynchronize(e1)) != cudaSuccess)
                return cuda_fail(c, ee, "autotune run");
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
        }
        uint32_t flags = 0;
        cudaError_t ee = cudaMemcpy(&flags, sc.err.p, 4, cudaMemcpyDeviceToHost);
        if (ee == cudaSuccess)
            ee = cudaMemcpy(have_ref ? got.data() : ref.data(), res, out_bytes, cudaMemcpyDeviceToHost);
        if (ee != cudaSuccess) return cuda_fail(c, ee, "autotune copy");
        if (flags) return fail(c, XD_EDEVICE, "device flags " + std::to_string(flags) + " while tuning");
        if (have_ref && std::memcmp(got.data(), ref.data(), out_bytes) != 0)
            return fail(c, XD_EDEVICE, "a tuning candidate changed the results");
        have_ref = true;
        return XD_OK;
    };
    const TierConfig base = tiers_for(c, v);
    TuneEntry best;
    best.alpha = v.alpha;
    best.xb = x_bucket(v.X);
    best.lb = len_bucket(v.max_len);
    best.sb = size_bucket(v.n_pairs);
    best.db = delta_bucket(uint32_t(v.delta));
    best.cfg = base;
    best.ms = 1e30f;
    auto consider = [&](const TierConfig& cand) -> xd_status {
        float ms = 0;
        xd_status r = run(cand, ms);
        if (r == XD_OK && ms < best.ms) {
            best.ms = ms;
            best.cfg = cand;
        }
        return r;
    };
    xd_status r = consider(base);
    for (const TierConfig& cand : chain_candidates(base, v.alpha))
        if (r == XD_OK) r = consider(cand);
    if (r == XD_OK && tier_group_of(best.cfg.variant[0]) == 1)
        for (int ch : {2, 4, 8, 16, 32, 64}) {
            TierConfig cand = best.cfg;
            cand.chunk = ch;
            if (r == XD_OK) r = consider(cand);
        }
    // the band tier's warps per side: 32 - 1024 threads per alignment of the widest bands
    if (r == XD_OK)
        for (int nw : {1, 2, 4, 16, 32}) {
            TierConfig cand = best.cfg;
            cand.band_warps = nw;
            if (r == XD_OK) r = consider(cand);
        }
    if (r == XD_OK && best.cfg.fused)
        for (int lp : {2, 5, 10}) {
            TierConfig cand = best.cfg;
            cand.long_permille = lp;
            if (r == XD_OK) r = consider(cand);
        }
    if (r == XD_OK && best.cfg.fused)
        for (auto mix : {std::pair<int, int>{2, 8}, {4, 16}, {8, 32}, {4, 8}, {8, 16}, {0, 16}, {4, 0}, {3, 6}}) {
            TierConfig cand = best.cfg;
            cand.every1 = mix.first;
            cand.every2 = mix.second;
            if (r == XD_OK) r = consider(cand);
        }
    c->timing = timing;
    if (r != XD_OK) {
        const std::string msg = c->err;
        cleanup();
        return fail(c, r, msg);
    }
    cleanup();
    put_entry(c->tuned, best);
    if (best_ms) *best_ms = best.ms;
    if (path && *path) {
        std::vector<TuneEntry> table;
        if (FILE* f = std::fopen(path, "r")) {
            std::fclose(f);
            if (load_table(c, path, table) != XD_OK) return XD_EINVAL;
        }
        put_entry(table, best);
        FILE* f = std::fopen(path, "w");
        if (!f) return fail(c, XD_EINVAL, std::string("cannot write tuning table ") + path);
        std::fprintf(f, "# xdrop-gb300 tuning table: alpha (4 DNA, 20 protein), X bucket (0: X <= 15, 1: <= 30,\n"
                        "# 2: more), length bucket (0: longest side <= 2048, 1: <= 20000, 2: more), size bucket\n"
                        "# (0: < 8192 side extensions, 1: < 65536, 2: < 1048576, 3: more), window bucket (0:\n"
                        "# unrestricted, 1: delta_b <= 512, 2: <= 2048, 3: more), chain of register-level variants,\n"
                        "# queue chunk, fused grid and its role mix, band-tier warps per side, measured ms\n");
        for (const TuneEntry& t : table) std::fprintf(f, "%s\n", format_entry(t).c_str());
        std::fclose(f);
    }
    return XD_OK;
}

xd_status xd_destroy(xd_ctx* c) {
    if (!c) return XD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->wake.notify_all();
    if (c->dispatcher.joinable()) c->dispatcher.join();   // waits (bounded) for in-flight slots
    cudaSetDevice(c->device);
    const xd_status rc = c->stop_timed_out ? XD_ETIMEDOUT : XD_OK;
    if (rc == XD_OK) cudaDeviceSynchronize();
    for (auto& kv : c->requests) {
        if (kv.second->in.p) cudaFreeHost(kv.second->in.p);
        delete kv.second;
    }
    for (HostBuf& b : c->pinned_cache) cudaFreeHost(b.p);
    for (Slot& s : c->slots) {
        release(s.s);
        release(s.d_in);
        release(s.d_results);
        if (s.h_stage.p) cudaFreeHost(s.h_stage.p);
        if (s.h_out.p) cudaFreeHost(s.h_out.p);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.uploaded) cudaEventDestroy(s.uploaded);
        for (Slot::Side& sd : s.side) {
            release(sd.s);
            if (sd.stream) cudaStreamDestroy(sd.stream);
            if (sd.joined) cudaEventDestroy(sd.joined);
        }
    }
    release(c->dev);
    release(c->stats);
    release(c->trace);
    for (SeqStore& ss : c->store) {
        release(ss.words);
        release(ss.d_off);
        release(ss.d_len);
    }
    for (auto& set : c->ev_sets)
        for (cudaEvent_t ev : set) cudaEventDestroy(ev);
    if (c->dev_stream) cudaStreamDestroy(c->dev_stream);
    if (c->coop_done) cudaEventDestroy(c->coop_done);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    delete c;
    return rc;
}

}  // extern "C"
