// Host runtime behind the C ABI of xdrop.h: contexts, validation, memory admission,
// pinned staging, in-flight slots with their own streams, tickets, and the device
// pipeline that runs one batch.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "xdrop.h"
#include "xd_device.cuh"
#include "xd_launch.h"

namespace {

using namespace xd;

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
    int32_t gap = 0, X = 0, max_abs = 1;
    uint32_t delta = 0, max_len = 0;
};

struct Slot {
    bool busy = false;
    uint64_t ticket = 0;
    uint32_t n_pairs = 0;
    uint64_t bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Scratch s;
    DevBuf d_in, d_results;
    HostBuf h_in, h_out;
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

}  // namespace

struct xd_ctx {
    int device = 0;
    int n_sm = 1;
    uint64_t cap = 0;
    uint64_t in_flight = 0;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    Scratch dev;                 // scratch of xd_run_device
    uint32_t reserved_len = 0;
    cudaStream_t dev_stream = nullptr;
    bool generic_only = false;
    TierConfig tiers{}, tiers_small_x{}, tiers_large_x{};
    DevBuf stats;                // uint64 [16]: cumulative per-batch counters (see Problem::stats)
    uint64_t batches = 0, pairs = 0, launches = 0;
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 8>> ev_sets;   // one set per timed batch
    size_t ev_used = 0;
    uint64_t stats_at_enable[16] = {};
    uint64_t launches_at_enable = 0;
    std::string err;
    std::mutex mu;
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
// 512-slot one 1040), at most 64 Mi ints.
constexpr uint64_t kRecIntsPerUnit = 256;
constexpr uint64_t kRecPoolMax = uint64_t(1) << 26;

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

void default_tiers(xd_ctx* c) {
    TierConfig& t = c->tiers;
    for (int v = 0; v < kNumGroupVariants; v++) t.blocks_per_sm[v] = 3;
    for (int v : {kG1C32, kG32C32, kG4C32, kG8C32, kG16C32}) t.blocks_per_sm[v] = 2;
    t.chunk = std::max(1, env_int("XD_CHUNK", 1));
    t.fused = env_int("XD_FUSED", 1) != 0;
    t.every1 = std::max(0, env_int("XD_EVERY1", 4));
    t.every2 = std::max(0, env_int("XD_EVERY2", 16));
    t.fused_minb = env_int("XD_FUSED_MINB", 2);
    set_chain(t, {kG1C32, kG16C16, kG32C16, kG32C32});
    c->tiers_small_x = t;
    set_chain(c->tiers_small_x, {kG1C32, kG16C16, kG32C16, kG32C32});
    c->tiers_large_x = t;
    set_chain(c->tiers_large_x, {kG4C16, kG16C16, kG32C32});
    if (const char* ch = std::getenv("XD_CHAIN")) {
        // comma-separated variant ids, used for every X
        TierConfig forced = t;
        forced.n_levels = 0;
        for (const char* q = ch; *q && forced.n_levels < kLevels - 2;) {
            forced.variant[forced.n_levels++] = std::atoi(q);
            while (*q && *q != ',') q++;
            if (*q == ',') q++;
        }
        c->tiers = c->tiers_small_x = c->tiers_large_x = forced;
    }
}

const TierConfig& tiers_for(const xd_ctx* c, const BatchView& b) {
    if (b.X <= 15) return c->tiers_small_x;
    if (b.X <= 30) return c->tiers;
    return c->tiers_large_x;
}

// The hot path of one batch (Sec. 3 method on every side extension), all on stream st.
xd_status run_pipeline(xd_ctx* c, Scratch& s, const BatchView& b, xd_result* d_out, cudaStream_t st) {
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
    auto* store = static_cast<uint32_t*>(s.store.p);
    XD_CUDA(c, launch_pack(b.alpha, b.codes, b.n_codes, store, err, c->n_sm, st));
    XD_CUDA(c, mark(1));
    Problem P{};
    P.store = store;
    P.n_words = std::max<uint64_t>(1, (b.n_codes + (b.alpha == 4 ? 15 : 5)) / (b.alpha == 4 ? 16 : 6));
    P.max_abs = b.max_abs;
    P.units = static_cast<const Unit*>(s.units.p);
    P.results = d_out;
    P.err = err;
    P.stats = static_cast<unsigned long long*>(s.bstats.p);
    P.rec = static_cast<int32_t*>(s.rec.p);
    P.rec_of = static_cast<uint32_t*>(s.rec_of.p);
    P.rec_ctr = static_cast<uint32_t*>(s.ctr.p) + (3 + 2 * kLevels);
    P.rec_cap = plan.rec_cap;
    if (b.n_pairs) XD_CUDA(c, cudaMemsetAsync(s.rec_of.p, 0xff, size_t(2) * b.n_pairs * 4, st));
    P.alpha = b.alpha;
    P.gap = b.gap;
    P.X = b.X;
    P.delta = b.delta;
    std::memcpy(P.sim, b.sim, sizeof(P.sim));
    XD_CUDA(c, launch_units(b.pairs, b.n_pairs, b.offsets, b.lengths, b.n_seqs, b.max_abs, b.max_len,
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
    uint64_t launches = b.n_pairs ? 4 : 3;   // pack (when codes exist), units, scan, scatter
    if (b.n_codes == 0) launches -= 1;
    if (b.n_pairs) {
        if (c->generic_only) {
            XD_CUDA(c, launch_route_all_generic(Q, st));
            launches += 1;
            XD_CUDA(c, mark(4));
            XD_CUDA(c, mark(5));
        } else {
            const TierConfig& tc = tiers_for(c, b);
            int lv = 0;
            if (tc.fused && fused_supported(tc)) {
                // the live queues' slots start unpublished
                XD_CUDA(c, cudaMemsetAsync(Q.q[0], 0xff, sizeof(uint32_t) * size_t(Q.n_units), st));
                XD_CUDA(c, cudaMemsetAsync(Q.q[1], 0xff, sizeof(uint32_t) * size_t(Q.n_units), st));
                XD_CUDA(c, launch_fused_levels(P, Q, tc, c->n_sm, st));
                XD_CUDA(c, mark(4));
                lv = 3;
                launches += 1;
            }
            for (; lv < tc.n_levels; lv++) {
                XD_CUDA(c, launch_level(P, Q, tc, lv, c->n_sm, st));
                if (lv == 0) XD_CUDA(c, mark(4));
                launches += 1;
            }
            XD_CUDA(c, launch_band(P, Q, c->n_sm, st));
            launches += 1;
            XD_CUDA(c, mark(5));
        }
        XD_CUDA(c, launch_generic(P, Q, static_cast<int32_t*>(s.generic.p), plan.generic_stride,
                                  plan.generic_blocks, st));
        XD_CUDA(c, mark(6));
        XD_CUDA(c, launch_totals(b.pairs, b.n_pairs, b.offsets, b.lengths, b.n_seqs, P, st));
        launches += 2;
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
    int inflight = cfg && cfg->max_inflight > 0 ? cfg->max_inflight : 8;
    c->slots.resize(inflight);
    const char* mode = std::getenv("XD_TIERS");
    c->generic_only = mode && std::strcmp(mode, "generic") == 0;
    default_tiers(c);
    if ((e = cudaStreamCreateWithFlags(&c->dev_stream, cudaStreamNonBlocking)) != cudaSuccess ||
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
    return run_pipeline(c, c->dev, v, d_out, st);
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

xd_status xd_submit_batch(xd_ctx* c, const xd_batch* b, uint64_t* ticket) {
    if (!c || !b || !ticket) return XD_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    BatchView v;
    xd_status s = scoring_view(c, b, v);
    if (s != XD_OK) return s;
    uint32_t max_len = 0;
    if ((s = validate_host(c, b, v, &max_len)) != XD_OK) return s;
    v.max_len = max_len;
    // admission by device memory
    size_t in_bytes = align_up(b->n_codes, 256) + align_up(8ull * b->n_seqs, 256) +
                      align_up(4ull * b->n_seqs, 256) + align_up(sizeof(xd_pair) * b->n_pairs, 256);
    size_t out_bytes = sizeof(xd_result) * size_t(b->n_pairs) + 16;
    size_t need = in_bytes + out_bytes + plan_bytes(plan_scratch(c, v.alpha, b->n_codes, b->n_pairs, max_len));
    if (c->in_flight + need > c->cap)
        return fail(c, XD_ENOMEM, "batch needs " + std::to_string(need) + " device bytes; " +
                                      std::to_string(c->cap - std::min(c->cap, c->in_flight)) + " available under the cap");
    Slot* slot = nullptr;
    for (Slot& q : c->slots)
        if (!q.busy) { slot = &q; break; }
    if (!slot) return fail(c, XD_ENOMEM, "no free in-flight slot");
    // stage inputs in pinned memory (the caller may free its buffers on return)
    size_t o_codes = 0, o_offs = align_up(b->n_codes, 256);
    size_t o_lens = o_offs + align_up(8ull * b->n_seqs, 256);
    size_t o_pairs = o_lens + align_up(4ull * b->n_seqs, 256);
    XD_CUDA(c, cudaEventSynchronize(slot->done));   // the slot's previous copies are finished
    XD_CUDA(c, grow_pinned(slot->h_in, in_bytes));
    XD_CUDA(c, grow_pinned(slot->h_out, out_bytes));
    char* h = static_cast<char*>(slot->h_in.p);
    const size_t bad_block = par_copy_check(h + o_codes, b->seq_codes, b->n_codes, v.alpha);
    if (bad_block != SIZE_MAX) {
        size_t t = bad_block;
        while (t < b->n_codes && b->seq_codes[t] < v.alpha) t++;
        return fail(c, XD_EINVAL, "residue code outside the alphabet at byte " + std::to_string(t));
    }
    std::memcpy(h + o_offs, b->seq_offsets, 8ull * b->n_seqs);
    std::memcpy(h + o_lens, b->seq_lengths, 4ull * b->n_seqs);
    std::memcpy(h + o_pairs, b->pairs, sizeof(xd_pair) * b->n_pairs);
    XD_CUDA(c, grow(slot->d_in, in_bytes));
    XD_CUDA(c, grow(slot->d_results, out_bytes));
    cudaStream_t st = slot->stream;
    XD_CUDA(c, cudaMemcpyAsync(slot->d_in.p, h, in_bytes, cudaMemcpyHostToDevice, st));
    char* d = static_cast<char*>(slot->d_in.p);
    v.codes = reinterpret_cast<const uint8_t*>(d + o_codes);
    v.offsets = reinterpret_cast<const uint64_t*>(d + o_offs);
    v.lengths = reinterpret_cast<const uint32_t*>(d + o_lens);
    v.pairs = reinterpret_cast<const xd_pair*>(d + o_pairs);
    auto* d_res = static_cast<xd_result*>(slot->d_results.p);
    if ((s = run_pipeline(c, slot->s, v, d_res, st)) != XD_OK) return s;
    XD_CUDA(c, cudaMemcpyAsync(slot->h_out.p, d_res, sizeof(xd_result) * size_t(b->n_pairs),
                               cudaMemcpyDeviceToHost, st));
    XD_CUDA(c, cudaMemcpyAsync(static_cast<char*>(slot->h_out.p) + out_bytes - 16, slot->s.err.p, 4,
                               cudaMemcpyDeviceToHost, st));
    XD_CUDA(c, cudaEventRecord(slot->done, st));
    slot->busy = true;
    slot->ticket = c->next_ticket++;
    slot->n_pairs = b->n_pairs;
    slot->bytes = need;
    c->in_flight += need;
    *ticket = slot->ticket;
    return XD_OK;
}

xd_status xd_poll(xd_ctx* c, uint64_t ticket, xd_result* out, int32_t wait_ms) {
    if (!c) return XD_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    Slot* slot = nullptr;
    for (Slot& q : c->slots)
        if (q.busy && q.ticket == ticket) { slot = &q; break; }
    if (!slot) return fail(c, XD_ENOTFOUND, "unknown ticket " + std::to_string(ticket));
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(slot->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "cudaEventQuery");
        if (wait_ms == 0) return XD_PENDING;
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (wait_ms > 0 && ms >= wait_ms) return fail(c, XD_ETIMEDOUT, "batch still running");
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(ms < 5 ? 20 : 200));
        lk.lock();
    }
    size_t out_bytes = sizeof(xd_result) * size_t(slot->n_pairs) + 16;
    uint32_t flags = 0;
    std::memcpy(&flags, static_cast<char*>(slot->h_out.p) + out_bytes - 16, 4);
    if (out && slot->n_pairs) par_memcpy(out, slot->h_out.p, sizeof(xd_result) * size_t(slot->n_pairs));
    slot->busy = false;
    c->in_flight -= std::min(c->in_flight, slot->bytes);
    if (flags) return fail(c, XD_EDEVICE, "device validation flags " + std::to_string(flags));
    return XD_OK;
}

xd_status xd_get_stats(const xd_ctx* c, xd_stats* out) {
    if (!c || !out) return XD_EINVAL;
    std::memset(out, 0, sizeof(*out));
    uint64_t dev[16] = {};
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->stats.p) cudaMemcpy(dev, c->stats.p, 128, cudaMemcpyDeviceToHost);
    out->batches = c->batches;
    out->pairs = c->pairs;
    out->units_tier[0] = dev[0];
    out->units_tier[1] = dev[1];
    out->units_tier[2] = dev[2];
    out->escalations = dev[3];
    out->cells = dev[4] + dev[5] + dev[6];
    out->kernel_launches = c->launches;
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
    out->launches = c->launches - c->launches_at_enable;
    return XD_OK;
}

xd_status xd_probe(xd_ctx* c, int32_t op, double* rate) {
    if (!c || !rate) return XD_EINVAL;
    if (!((op >= 0 && op <= 10) || op == 100)) return fail(c, XD_EINVAL, "unknown probe op");
    std::lock_guard<std::mutex> lk(c->mu);
    XD_CUDA(c, cudaSetDevice(c->device));
    XD_CUDA(c, cudaDeviceSynchronize());
    float ms = 0;
    XD_CUDA(c, probe_rate(op, c->n_sm, rate, &ms));
    return XD_OK;
}

xd_status xd_destroy(xd_ctx* c) {
    if (!c) return XD_EINVAL;
    cudaSetDevice(c->device);
    xd_status rc = XD_OK;
    auto t0 = std::chrono::steady_clock::now();
    for (Slot& s : c->slots) {
        if (!s.done) continue;
        while (cudaEventQuery(s.done) == cudaErrorNotReady) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {
                rc = XD_ETIMEDOUT;
                break;
            }
            std::this_thread::sleep_for(std::chrono::milliseconds(1));
        }
    }
    if (rc == XD_OK) cudaDeviceSynchronize();
    for (Slot& s : c->slots) {
        release(s.s);
        release(s.d_in);
        release(s.d_results);
        if (s.h_in.p) cudaFreeHost(s.h_in.p);
        if (s.h_out.p) cudaFreeHost(s.h_out.p);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
    }
    release(c->dev);
    release(c->stats);
    for (auto& set : c->ev_sets)
        for (cudaEvent_t ev : set) cudaEventDestroy(ev);
    if (c->dev_stream) cudaStreamDestroy(c->dev_stream);
    delete c;
    return rc;
}

}  // extern "C"
