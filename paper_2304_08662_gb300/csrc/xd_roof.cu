// Integer / DPX throughput microbenchmarks: the measured denominator of the roofline for
// the alignment kernels, which are bound by plain integer arithmetic (no dense
// contraction, negligible DRAM traffic).
//
// Each probe runs eight independent dependency chains per thread of one instruction kind
// (operands rotate through the chains so nothing folds), or the complete per-cell update
// of the register tiers on in-register anti-diagonals.  Results are in thread-operations
// (or cells) per second for the whole GPU.
#include <cstdint>
#include <cuda_runtime.h>
#include "xd_group.cuh"

namespace xd {

enum ProbeOp {
    kProbeIadd = 0,        // x = x + y
    kProbeImnmx = 1,       // x = max(x, y)
    kProbeViaddmax = 2,    // x = max(x + c, y)            (DPX)
    kProbeVimax3 = 3,      // x = max(x, y, z)             (DPX)
    kProbeLop3 = 4,        // x = (x & y) ^ z
    kProbeImad = 5,        // x = x * y + c
    kProbeSel = 6,         // x = (y > c) ? x : z          (compare + select: 2 instructions)
    kProbePrmt = 7,        // x = byte_perm(x, y)
    kProbeViaddmax16 = 8,  // 16x2: x = max(x + c, y) per half   (DPX)
    kProbeVimax3_16 = 9,   // 16x2: x = max(x, y, z) per half    (DPX)
    kProbeVmax16 = 10,     // 16x2: x = max(x, y) per half
    kProbeCellDna = 100,   // the register tiers' cell update (cells_of), DNA, 32 slots
    kProbeCellProt = 101,  // the same, protein (similarity-table offsets), 32 slots
    kProbeCellDna16 = 102, // the 16-bit packed DNA update (cells16 with its best-cell key)
    kProbeCellProt16 = 103, // the same, protein
};

template <int OP>
__device__ __forceinline__ int32_t probe_op(int32_t x, int32_t y, int32_t z, int32_t c) {
    if (OP == kProbeIadd) return x + y;
    if (OP == kProbeImnmx) return max(x, y);
    if (OP == kProbeViaddmax) return __viaddmax_s32(x, c, y);
    if (OP == kProbeVimax3) return __vimax3_s32(x, y, z);
    if (OP == kProbeLop3) return (x & y) ^ z;
    if (OP == kProbeImad) return x * y + c;
    if (OP == kProbeSel) return (y > c) ? x : z;
    if (OP == kProbePrmt) return int32_t(__byte_perm(uint32_t(x), uint32_t(y), 0x5432));
    if (OP == kProbeViaddmax16) return int32_t(__viaddmax_s16x2(uint32_t(x), uint32_t(c), uint32_t(y)));
    if (OP == kProbeVimax3_16) return int32_t(__vimax3_s16x2(uint32_t(x), uint32_t(y), uint32_t(z)));
    if (OP == kProbeVmax16) return int32_t(__vmaxs2(uint32_t(x), uint32_t(y)));
    return x;
}

template <int OP>
__global__ void __launch_bounds__(256) k_probe(int32_t* out, int iters, int32_t seed) {
    int32_t a[8];
#pragma unroll
    for (int u = 0; u < 8; u++) a[u] = int32_t(threadIdx.x * 2654435761u) ^ (seed + u * 97);
    const int32_t c = seed | 1;
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
#pragma unroll
            for (int u = 0; u < 8; u++) a[u] = probe_op<OP>(a[u], a[(u + 1) & 7], a[(u + 2) & 7], c);
        }
    }
    int32_t acc = 0;
#pragma unroll
    for (int u = 0; u < 8; u++) acc ^= a[u];
    if (acc == seed) out[blockIdx.x] = acc;   // practically never true; keeps the chains live
}

// The register tiers' own cell update (cells_of of the group kernels) on 32 in-register
// slots, alternating odd / even anti-diagonals, every slot inside the band; the residue
// slices rotate so that the similarities vary.
template <int A>
__global__ void __launch_bounds__(128, 2) k_probe_cells(int32_t* out, int iters, int32_t seed) {
    __shared__ __align__(16) int32_t tab[kLutInts];
    Problem P{};
    if (A == 4) {
        P.sim[0] = 1;
        P.sim[1] = -1;
    } else {
        for (int t = 0; t < 400; t++) P.sim[t] = int8_t((t * 7 + 3) % 15 - 7);
    }
    build_table<A>(tab, P);
    int32_t R0[32], R1[32];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        R0[t] = (t * 7 + seed) & 15;
        R1[t] = (t * 3 + seed) & 15;
    }
    Res<32, A> res;
    uint64_t x = 0x9E3779B97F4A7C15ull ^ uint64_t(threadIdx.x) * 0xBF58476D1CE4E5B9ull;
    if constexpr (A == 4) {
        res.hs = x;
        res.vs = x * 0x94D049BB133111EBull;
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++) {
            res.hx[k] = uint32_t((x >> (k & 7)) % 20) * 80u | (uint32_t((x >> (k + 9)) % 20) * 80u << 16);
            res.vx[k] = uint32_t((x >> (k + 3)) % 20) * 4u | (uint32_t((x >> (k + 17)) % 20) * 4u << 16);
        }
    }
    int32_t thr = -100, kmax = 0;
    uint32_t lm = 0, acc = 0;
    for (int k = 0; k < iters; k++) {
        cells_of<32, true, A>(R0, R1, kNegR, kNegR, res, 0xffffffffu, thr, -1, tab, kmax, lm);
        acc ^= lm;
        thr = (kmax >> 6) - 40;
        cells_of<32, false, A>(R1, R0, kNegR, kNegR, res, 0xffffffffu, thr, -1, tab, kmax, lm);
        acc ^= lm;
        thr = (kmax >> 6) - 40;
        if constexpr (A == 4) {
            res.hs = (res.hs << 2) | (res.hs >> 62);
        } else {
            const uint32_t t0 = res.hx[0];
#pragma unroll
            for (int q = 0; q < 15; q++) res.hx[q] = res.hx[q + 1];
            res.hx[15] = t0;
        }
    }
    if (acc == uint32_t(seed) && kmax == seed) out[blockIdx.x] = int32_t(acc);
}

// The packed update of the group kernels (cells16 with its best-cell key; A = kDna16 or
// kProt16) on 32 slots held in 16 registers, alternating odd / even anti-diagonals, every
// slot inside the band (the band mask is a run-time zero, so its instructions stay).
template <int A>
__global__ void __launch_bounds__(128, 2) k_probe_cells16(int32_t* out, int iters, int32_t seed) {
    __shared__ __align__(16) int32_t tab[kLutInts];
    Problem P{};
    if (A == kDna16) {
        P.sim[0] = 1;
        P.sim[1] = -1;
        P.gap = -1;
    } else {
        for (int t = 0; t < 400; t++) P.sim[t] = int8_t((t * 7 + 3) % 15 - 7);
        P.gap = -2;
    }
    build_table<A>(tab, P);
    uint32_t R0[16], R1[16];
#pragma unroll
    for (int t = 0; t < 16; t++) {
        R0[t] = pack2(32 * (200 + ((t * 7 + seed) & 15)), 32 * (200 + ((t * 5 + seed) & 15)));
        R1[t] = pack2(32 * (200 + ((t * 3 + seed) & 15)), 32 * (200 + ((t * 11 + seed) & 15)));
    }
    Res<32, A> res;
    uint64_t x = 0x9E3779B97F4A7C15ull ^ uint64_t(threadIdx.x) * 0xBF58476D1CE4E5B9ull;
    if constexpr (A == kDna16) {
        res.hs = x;
        res.vs = x * 0x94D049BB133111EBull;
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++) {
            res.hx[k] = uint32_t((x >> (k & 7)) % 20) * 80u | (uint32_t((x >> (k + 9)) % 20) * 80u << 16);
            res.vx[k] = uint32_t((x >> (k + 3)) % 20) * 4u | (uint32_t((x >> (k + 17)) % 20) * 4u << 16);
        }
    }
    const uint32_t nbv = uint32_t(seed) >> 30;   // zero, unknown to the compiler
    uint32_t nth2 = (uint32_t(-32 * 190) & 0xffffu) * 0x10001u, acc = 0;
    int32_t k = 0;
    for (int it = 0; it < iters; it++) {
        uint32_t mk, dacc;
        cells16<32, true, A>(R0, R1, kDead2, kDead2, res, nbv, nth2, tab, mk, dacc);
        k = max(lo16(mk), hi16(mk));
        acc ^= dacc;
        nth2 = (uint32_t(32 * 20 - (k & ~31)) & 0xffffu) * 0x10001u;
        cells16<32, false, A>(R1, R0, kDead2, kDead2, res, nbv, nth2, tab, mk, dacc);
        k = max(lo16(mk), hi16(mk));
        acc ^= dacc;
        nth2 = (uint32_t(32 * 20 - (k & ~31)) & 0xffffu) * 0x10001u;
        if constexpr (A == kDna16) {
            res.hs = (res.hs << 2) | (res.hs >> 62);
        } else {
            const uint32_t t0 = res.hx[0];
#pragma unroll
            for (int q = 0; q < 15; q++) res.hx[q] = res.hx[q + 1];
            res.hx[15] = t0;
        }
    }
    if (acc == uint32_t(seed) && k == seed) out[blockIdx.x] = int32_t(acc);
}

template <int OP>
static cudaError_t run_probe(int blocks, int iters, cudaStream_t st, int32_t* out) {
    k_probe<OP><<<blocks, 256, 0, st>>>(out, iters, 12345);
    return cudaGetLastError();
}

// ops (or cells) per second of the whole GPU; blocks = resident-block multiple of the SMs
cudaError_t probe_rate(int op, int n_sm, double* rate, float* ms_out) {
    int32_t* out = nullptr;
    cudaError_t e = cudaMalloc(&out, 4096 * sizeof(int32_t));
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = n_sm * 8;
    const bool cells = op == kProbeCellDna || op == kProbeCellProt || op == kProbeCellDna16 ||
                       op == kProbeCellProt16;
    int iters = cells ? 4000 : 20000;
    double per_thread = 0;
    int threads = 256;
    auto launch = [&]() -> cudaError_t {
        switch (op) {
            case kProbeIadd: return run_probe<kProbeIadd>(blocks, iters, 0, out);
            case kProbeImnmx: return run_probe<kProbeImnmx>(blocks, iters, 0, out);
            case kProbeViaddmax: return run_probe<kProbeViaddmax>(blocks, iters, 0, out);
            case kProbeVimax3: return run_probe<kProbeVimax3>(blocks, iters, 0, out);
            case kProbeLop3: return run_probe<kProbeLop3>(blocks, iters, 0, out);
            case kProbeImad: return run_probe<kProbeImad>(blocks, iters, 0, out);
            case kProbeSel: return run_probe<kProbeSel>(blocks, iters, 0, out);
            case kProbePrmt: return run_probe<kProbePrmt>(blocks, iters, 0, out);
            case kProbeViaddmax16: return run_probe<kProbeViaddmax16>(blocks, iters, 0, out);
            case kProbeVimax3_16: return run_probe<kProbeVimax3_16>(blocks, iters, 0, out);
            case kProbeVmax16: return run_probe<kProbeVmax16>(blocks, iters, 0, out);
            case kProbeCellDna:
                k_probe_cells<4><<<n_sm * 2, 128, 0, 0>>>(out, iters, 12345);
                return cudaGetLastError();
            case kProbeCellProt:
                k_probe_cells<20><<<n_sm * 2, 128, 0, 0>>>(out, iters, 12345);
                return cudaGetLastError();
            case kProbeCellDna16:
                k_probe_cells16<kDna16><<<n_sm * 2, 128, 0, 0>>>(out, iters, 12345);
                return cudaGetLastError();
            case kProbeCellProt16:
                k_probe_cells16<kProt16><<<n_sm * 2, 128, 0, 0>>>(out, iters, 12345);
                return cudaGetLastError();
            default: return cudaErrorInvalidValue;
        }
    };
    if (cells) {
        threads = 128;
        per_thread = double(iters) * 64.0;            // cells
    } else {
        per_thread = double(iters) * 64.0;            // 8 rounds x 8 chains
    }
    const int total_blocks = cells ? n_sm * 2 : blocks;
    e = launch();                                      // warm-up
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    float ms = 0;
    if (e == cudaSuccess) {
        cudaEventRecord(a, 0);
        e = launch();
        cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    *rate = double(total_blocks) * threads * per_thread / (double(ms) * 1e-3);
    if (ms_out) *ms_out = ms;
    return cudaSuccess;
}

}  // namespace xd
