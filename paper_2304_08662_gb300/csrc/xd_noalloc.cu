// Allocation-free entry point: xd_run_device_noalloc.
//
// Some callers cannot allocate device memory at all: code running inside a host callback
// or a CUDA-graph-driven pipeline whose memory is fixed up front, processes that run under
// a strict device-memory budget enforced by another allocator, or runtimes that forbid
// cudaMalloc after start-up.  For them this entry point computes the same results as
// xd_run_device using only the caller's input and output buffers plus one scratch array
// that lives in this file for the lifetime of the library.
//
// The kernel is a variant of the generic tier (one warp per side extension, the three
// anti-diagonals of the paper's sweep in global memory): here one warp takes a whole pair,
// reads the caller's unpacked residue codes directly (no packed store, no work-unit list),
// and keeps its anti-diagonal rows in the static array below.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include <cuda.h>   // driver API types only; its functions are reached through the runtime

#include "xdrop.h"
#include "xd_sweep.cuh"

namespace {

constexpr int64_t kScoreLimitN = xd::kScoreLimit;
constexpr int kWarpsPerBlock = 4;
constexpr int kMaxWarps = 4096;
constexpr uint32_t kFlagInvalid = 0x80000000u;   // result flag: the pair's inputs were invalid

// 64 MiB of scratch, held by every GPU that loads the library until the process exits.
// Each warp uses three rows of (max_side_len + 1) int32 (rounded up to 32 entries).  Every
// row entry a warp reads was written earlier in the same side extension, so nothing in the
// array needs to start at zero; calls that overlap on the GPU (two streams at once) share
// the rows and race.
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchBytes / sizeof(int32_t)];

struct Args {
    const uint8_t* codes;
    uint64_t n_codes;
    const uint64_t* offsets;
    const uint32_t* lengths;
    uint32_t n_seqs;
    const xd_pair* pairs;
    uint32_t n_pairs;
    xd_result* out;
    int32_t alpha, gap, X, zdrop;
    uint32_t delta, max_side_len;
    int32_t max_abs;
    int8_t sim[400];
};

__device__ __forceinline__ uint32_t code_at(const Args& a, uint64_t pos, bool& bad) {
    const uint32_t c = a.codes[pos];
    if (c >= uint32_t(a.alpha)) {
        bad = true;
        return 0;
    }
    return c;
}

// One side: H_side[t] = codes[h0 + dir t], V_side[t] = codes[v0 + dir t], swept exactly as
// the generic tier sweeps it (generic_sweep); codes outside the alphabet set `bad`.
__device__ void side_noalloc(const Args& a, const int32_t* sim, int64_t h0, int64_t v0, int64_t dir,
                             int64_t m, int64_t n, int32_t* A, int32_t* B, int32_t* Cc, int lane,
                             xd_side& res, bool& bad) {
    bool lane_bad = false;
    auto sim_at = [&](int64_t i, int64_t j) {
        const uint32_t x = code_at(a, uint64_t(h0 + dir * (i - 1)), lane_bad);
        const uint32_t y = code_at(a, uint64_t(v0 + dir * (j - 1)), lane_bad);
        return sim[x * a.alpha + y];
    };
    const xd::SweepOut o = xd::generic_sweep(m, n, a.gap, a.X, a.delta, a.zdrop, sim_at, A, B, Cc, lane);
    bad |= __any_sync(0xffffffffu, lane_bad);
    res.score = o.best;
    res.h_ext = uint32_t(o.bi);
    res.v_ext = uint32_t(o.bj);
    res.flags = o.flags;
    res.cells = o.cells;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_noalloc(Args a, int32_t* scratch, uint64_t stride) {
    __shared__ int32_t sim[400];
    for (int t = threadIdx.x; t < a.alpha * a.alpha; t += blockDim.x) sim[t] = a.sim[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
    const uint64_t n_warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    int32_t* rows = scratch + warp * 3 * stride;
    for (uint64_t p = warp; p < a.n_pairs; p += n_warps) {
        const xd_pair e = a.pairs[p];
        xd_result r = {};
        bool bad = e.h_id >= a.n_seqs || e.v_id >= a.n_seqs;
        uint64_t ho = 0, vo = 0, lh = 0, lv = 0;
        if (!bad) {
            ho = a.offsets[e.h_id];
            vo = a.offsets[e.v_id];
            lh = a.lengths[e.h_id];
            lv = a.lengths[e.v_id];
            bad = uint64_t(e.h_seed) + e.seed_len > lh || uint64_t(e.v_seed) + e.seed_len > lv ||
                  ho + lh > a.n_codes || vo + lv > a.n_codes;
        }
        const int64_t rm = bad ? 0 : int64_t(lh - e.h_seed - e.seed_len);
        const int64_t rn = bad ? 0 : int64_t(lv - e.v_seed - e.seed_len);
        const int64_t lm = bad ? 0 : int64_t(e.h_seed), ln = bad ? 0 : int64_t(e.v_seed);
        if (!bad && (rm > a.max_side_len || lm > a.max_side_len || (rm + rn) * a.max_abs >= kScoreLimitN ||
                     (lm + ln) * a.max_abs >= kScoreLimitN))
            bad = true;
        if (bad) {
            if (lane == 0) {
                r.left.flags = r.right.flags = kFlagInvalid;
                a.out[p] = r;
            }
            __syncwarp();
            continue;
        }
        side_noalloc(a, sim, int64_t(ho + e.h_seed + e.seed_len), int64_t(vo + e.v_seed + e.seed_len), 1, rm,
                     rn, rows, rows + stride, rows + 2 * stride, lane, r.right, bad);
        side_noalloc(a, sim, e.h_seed ? int64_t(ho + e.h_seed - 1) : int64_t(ho),
                     e.v_seed ? int64_t(vo + e.v_seed - 1) : int64_t(vo), -1, lm, ln, rows, rows + stride,
                     rows + 2 * stride, lane, r.left, bad);
        int64_t seed = 0;
        for (uint32_t t = lane; t < e.seed_len; t += 32) {
            const uint32_t x = code_at(a, ho + e.h_seed + t, bad), y = code_at(a, vo + e.v_seed + t, bad);
            seed += sim[x * a.alpha + y];
        }
        for (int k = 16; k >= 1; k >>= 1) seed += __shfl_xor_sync(0xffffffffu, seed, k);
        bad = __any_sync(0xffffffffu, bad);
        r.total = int64_t(r.left.score) + int64_t(r.right.score) + seed;
        if (bad) {
            r.left.flags |= kFlagInvalid;
            r.right.flags |= kFlagInvalid;
        }
        if (lane == 0) a.out[p] = r;
        __syncwarp();
    }
}

// Device address of the scratch array, resolved once per CUDA context with that context
// current.  The cache is keyed by the context's unique id (cuCtxGetId, never reused within
// a process), not by the device number: a context made after cudaDeviceReset, or a second
// context on the same device made through the driver API, loads its own copy of the module
// and so has its own address.
constexpr int kCacheSlots = 64;
struct CacheSlot {
    unsigned long long ctx_id;
    int32_t* ptr;
};
std::mutex g_mu;
CacheSlot g_cache[kCacheSlots] = {};
int g_cache_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context; false if it cannot be had.  With no context
// current yet, the runtime call that resolves the symbol makes the device's primary context
// current first.
bool current_context_id(unsigned long long& id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext cur = nullptr;
    if (get_current(&cur) != CUDA_SUCCESS) return false;
    if (!cur) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return false;
        if (get_current(&cur) != CUDA_SUCCESS || !cur) return false;
    }
    return get_id(cur, &id) == CUDA_SUCCESS;
}

}  // namespace

extern "C" xd_status xd_run_device_noalloc(const xd_batch* b, uint32_t max_side_len, xd_result* d_out,
                                           void* stream) {
    if (!b || (b->n_pairs && (!d_out || !b->pairs || !b->seq_offsets || !b->seq_lengths)) ||
        (b->n_codes && !b->seq_codes))
        return XD_EINVAL;
    if (b->X < 0 || (b->alpha != XD_DNA2 && b->alpha != XD_PROT5)) return XD_EINVAL;
    if (b->alpha == XD_PROT5 && !b->scoring.matrix20x20) return XD_EINVAL;
    if (b->scoring.gap > 0 || b->scoring.gap < -(1 << 20)) return XD_EINVAL;
    const uint64_t stride = (uint64_t(max_side_len) + 1 + 31) / 32 * 32;
    const uint64_t per_warp = 3 * stride * sizeof(int32_t);
    if (per_warp > kScratchBytes) return XD_EINVAL;   // a single side does not fit the scratch
    if (b->n_pairs == 0) return XD_OK;
    int32_t* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned long long id = 0;
        if (!current_context_id(id)) return XD_EDEVICE;
        for (const CacheSlot& cs : g_cache)
            if (cs.ptr && cs.ctx_id == id) scratch = cs.ptr;
        if (!scratch) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return XD_EDEVICE;
            scratch = static_cast<int32_t*>(p);
            g_cache[g_cache_next] = CacheSlot{id, scratch};
            g_cache_next = (g_cache_next + 1) % kCacheSlots;
        }
    }
    Args a{};
    a.codes = b->seq_codes;
    a.n_codes = b->n_codes;
    a.offsets = b->seq_offsets;
    a.lengths = b->seq_lengths;
    a.n_seqs = b->n_seqs;
    a.pairs = b->pairs;
    a.n_pairs = b->n_pairs;
    a.out = d_out;
    a.alpha = b->alpha == XD_DNA2 ? 4 : 20;
    a.gap = b->scoring.gap;
    a.X = b->X;
    if (b->z_drop < 0) return XD_EINVAL;
    a.zdrop = b->z_drop;
    a.delta = b->delta_b;
    a.max_side_len = max_side_len;
    int32_t max_abs = a.gap < 0 ? -a.gap : a.gap;
    if (a.alpha == 4) {
        if (b->scoring.match > 127 || b->scoring.match < -127 || b->scoring.mismatch > 127 ||
            b->scoring.mismatch < -127)
            return XD_EINVAL;
        for (int x = 0; x < 4; x++)
            for (int y = 0; y < 4; y++) a.sim[x * 4 + y] = int8_t(x == y ? b->scoring.match : b->scoring.mismatch);
    } else {
        std::memcpy(a.sim, b->scoring.matrix20x20, 400);
    }
    for (int t = 0; t < a.alpha * a.alpha; t++) {
        const int32_t v = a.sim[t] < 0 ? -a.sim[t] : a.sim[t];
        if (v > max_abs) max_abs = v;
    }
    a.max_abs = max_abs > 0 ? max_abs : 1;
    uint64_t n_warps = kScratchBytes / per_warp;
    if (n_warps > kMaxWarps) n_warps = kMaxWarps;
    if (n_warps > b->n_pairs) n_warps = b->n_pairs;
    const uint64_t blocks = (n_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    // blocks * kWarpsPerBlock may exceed n_warps by up to 3 warps; keep every warp inside
    // the scratch by launching only whole blocks that fit
    const uint64_t fit_blocks = (kScratchBytes / per_warp) / kWarpsPerBlock;
    const uint64_t grid = blocks < fit_blocks ? blocks : (fit_blocks ? fit_blocks : 0);
    if (grid == 0) {
        // fewer than one block of warps fits: run single-warp blocks
        const uint64_t w = kScratchBytes / per_warp;
        k_noalloc<<<dim3(unsigned(w < b->n_pairs ? w : b->n_pairs)), dim3(32), 0,
                    static_cast<cudaStream_t>(stream)>>>(a, scratch, stride);
    } else {
        k_noalloc<<<dim3(unsigned(grid)), dim3(kWarpsPerBlock * 32), 0, static_cast<cudaStream_t>(stream)>>>(
            a, scratch, stride);
    }
    return cudaGetLastError() == cudaSuccess ? XD_OK : XD_EDEVICE;
}
