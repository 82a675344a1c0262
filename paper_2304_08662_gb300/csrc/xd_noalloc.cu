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

#include "xdrop.h"

namespace {

constexpr int32_t kNegN = -(1 << 30);
constexpr int32_t kDeadLineN = -(1 << 29);
constexpr int64_t kScoreLimitN = int64_t(1) << 29;
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
    int32_t alpha, gap, X;
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

// One side: H_side[t] = codes[h0 + dir t], V_side[t] = codes[v0 + dir t].  Same sweep as the
// generic tier: band from the previous anti-diagonal, optional delta_b window, recurrence,
// X-Drop against T of completed anti-diagonals, warp reductions of live range and best cell.
__device__ void side_noalloc(const Args& a, const int32_t* sim, int64_t h0, int64_t v0, int64_t dir,
                             int64_t m, int64_t n, int32_t* A, int32_t* B, int32_t* Cc, int lane,
                             xd_side& res, bool& bad) {
    int32_t* P1 = A;
    int32_t* P2 = B;
    int32_t* C = Cc;
    int64_t p1lo = 0, p1hi = 0, p2lo = 1, p2hi = 0;
    if (lane == 0) P1[0] = 0;
    __syncwarp();
    int32_t T = 0, best = 0;
    int64_t bi = 0, bj = 0, L = 0, U = 0, prev_arg = 0;
    uint64_t cells = 1;
    uint32_t flags = 0;
    bool lane_bad = false;
    for (int64_t d = 1; d <= m + n; d++) {
        int64_t lo = L, hi = U + 1;
        if (d - n > lo) lo = d - n;
        if (lo < 0) lo = 0;
        if (hi > m) hi = m;
        if (hi > d) hi = d;
        if (a.delta && hi - lo + 1 > int64_t(a.delta)) {
            flags = 1;
            int64_t start = prev_arg - int64_t(a.delta / 2);
            const int64_t latest = hi - int64_t(a.delta) + 1;
            if (latest < start) start = latest;
            if (start > lo) lo = start;
            hi = lo + int64_t(a.delta) - 1;
        }
        const int32_t thr = max(T - a.X, kDeadLineN);
        int32_t first = INT32_MAX, last = -1, bmax = kNegN, barg = INT32_MAX;
        for (int64_t i = lo + lane; i <= hi; i += 32) {
            const int64_t j = d - i;
            int32_t c = kNegN;
            if (i >= 1 && j >= 1 && i - 1 >= p2lo && i - 1 <= p2hi) {
                const uint32_t x = code_at(a, uint64_t(h0 + dir * (i - 1)), lane_bad);
                const uint32_t y = code_at(a, uint64_t(v0 + dir * (j - 1)), lane_bad);
                c = P2[i - 1] + sim[x * a.alpha + y];
            }
            if (i >= 1 && i - 1 >= p1lo && i - 1 <= p1hi) c = max(c, P1[i - 1] + a.gap);
            if (j >= 1 && i >= p1lo && i <= p1hi) c = max(c, P1[i] + a.gap);
            if (c < thr) c = kNegN;
            C[i] = c;
            if (c != kNegN) {
                if (first == INT32_MAX) first = int32_t(i);
                last = int32_t(i);
                if (c > bmax) {
                    bmax = c;
                    barg = int32_t(i);
                }
            }
        }
        cells += uint64_t(hi - lo + 1);
        first = __reduce_min_sync(0xffffffffu, first);
        last = __reduce_max_sync(0xffffffffu, last);
        const int32_t wmax = __reduce_max_sync(0xffffffffu, bmax);
        barg = __reduce_min_sync(0xffffffffu, bmax == wmax ? barg : INT32_MAX);
        __syncwarp();
        if (first == INT32_MAX) break;
        if (wmax > T) {
            T = wmax;
            best = wmax;
            bi = barg;
            bj = d - barg;
        }
        prev_arg = barg;
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
    bad |= __any_sync(0xffffffffu, lane_bad);
    res.score = best;
    res.h_ext = uint32_t(bi);
    res.v_ext = uint32_t(bj);
    res.flags = flags;
    res.cells = cells;
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

// Device address of the scratch array, resolved once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_scratch_ptr[kMaxDevices] = {};

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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return XD_EDEVICE;
    int32_t* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return XD_EDEVICE;
            g_scratch_ptr[dev] = static_cast<int32_t*>(p);
        }
        scratch = g_scratch_ptr[dev];
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
