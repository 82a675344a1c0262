/* xdrop.h -- C ABI of the batched X-Drop seed-extension library (CUDA, sm_103a).
 *
 * The library computes, for many independent seed extensions at once, the X-Drop
 * semi-global alignment of the paper (Sec. 2.2 recurrence and X-Drop rule, Sec. 3 and
 * Algorithm 1 for the anti-diagonal sweep, the live band and the memory-restricted
 * window).  Every pair (H, V, H_s, V_s) with a seed of length k (the seed-extension tuple
 * e_c of Sec. 4.4) is split into a left and a right extension (Sec. 4.1.2); each side is
 * aligned from S(0,0) = 0 and the best cell is reported.
 *
 * Exact integer arithmetic throughout.  Results are bit-identical to the plain CPU
 * definition of the method (score, end coordinates, overflow flag, evaluated cells).
 *
 * Conventions
 *   - Every call returns an xd_status; nothing throws across the ABI.
 *   - Host pointers passed to xd_submit_batch are read during the call only: the caller
 *     may free or reuse them as soon as it returns.
 *   - Residue codes are unpacked bytes: 0..3 for DNA (A, C, G, T), 0..19 for protein in
 *     the order A R N D C Q E G H I L K M F P S T W Y V.  Packing (2-bit DNA, 5-bit
 *     protein) happens inside the library.
 *   - Side coordinates: right side H_R[t] = H[h_seed + k + t], V_R[t] = V[v_seed + k + t];
 *     left side H_L[t] = H[h_seed - 1 - t], V_L[t] = V[v_seed - 1 - t] (the index
 *     transform op() of Sec. 3).  h_ext / v_ext are the i / j of the best cell, i.e. the
 *     extension lengths; the aligned span on H is [h_seed - left.h_ext,
 *     h_seed + k + right.h_ext), and likewise on V.
 *   - Readings of the paper where it is silent: X-Drop compares strictly (S < T - X)
 *     against the best score T of the completed anti-diagonals; the next band is
 *     [first live, last live + 1] clipped to the matrix; the end cell is the first
 *     anti-diagonal reaching the best score, lowest i on it; the seed is not part of a
 *     side's score and total = left + right + sum of Sim over the seed.
 */
#ifndef XDROP_H
#define XDROP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xd_ctx xd_ctx;

typedef enum {
    XD_OK = 0,
    XD_PENDING = 1,      /* xd_poll: the batch has not finished yet */
    XD_EINVAL = -1,      /* invalid argument; nothing was queued */
    XD_ENOMEM = -2,      /* admission refused (device memory cap or no free slot); retry later */
    XD_ETIMEDOUT = -3,   /* a bounded wait expired; the work is still in flight */
    XD_EDEVICE = -4,     /* CUDA error or no usable device */
    XD_ENOTFOUND = -5    /* unknown or already retired ticket */
} xd_status;

typedef enum { XD_DNA2 = 0, XD_PROT5 = 1 } xd_alphabet;

/* Context configuration.  device: CUDA ordinal.  store_bytes_cap: device bytes the
 * library may hold for admitted host batches (0 = 64 GiB): their sequences (unpacked and
 * packed), seed tuples, results and per-side state; each launch slot also keeps band rows
 * of 3 x (longest side + 1) scores per resident warp of the generic tier.  max_inflight: launches of host
 * batches in flight at once, each on its own stream (0 = 3).  tune_table: path of a tuning
 * table written by xd_autotune, or NULL for built-in defaults.  batching: 0 or 1 = continuous
 * batching (host batches that wait for a free launch slot and share scoring, X and delta_b
 * are merged into one launch); -1 = one launch per host batch.  max_batch_pairs: cap on the
 * pairs of one merged launch (0 = 2^20; a single larger batch still runs alone); a merged
 * launch also holds at most 24 GiB of residue codes. */
typedef struct {
    int32_t device;
    uint64_t store_bytes_cap;
    int32_t max_inflight;
    const char* tune_table;
    int32_t batching;
    uint32_t max_batch_pairs;
} xd_config;

/* Scoring (Sec. 2.2): DNA uses match (> 0), mismatch and gap scores; protein uses a
 * 20x20 row-major substitution matrix (BLOSUM62 in Sec. 5.3) and the gap score.  gap is
 * the (negative) score added per gap symbol: linear gaps only.  matrix20x20 is a host
 * pointer, read during the call. */
typedef struct {
    int32_t match, mismatch, gap;
    const int8_t* matrix20x20;
} xd_scoring;

/* One seed-extension tuple e_c = (H, V, H_s, V_s) plus the seed length k (Sec. 4.4):
 * indices into the batch's sequence table and seed start positions. */
typedef struct {
    uint32_t h_id, v_id;
    uint32_t h_seed, v_seed, seed_len;
} xd_pair;

/* A batch: sequence table (codes + per-sequence offsets/lengths, the detached sequence
 * set of Sec. 4.1.1) and the list of seed tuples.  For xd_submit_batch every pointer is
 * a host pointer; for xd_run_device, seq_codes, seq_offsets, seq_lengths and pairs are
 * device pointers (scoring.matrix20x20 stays a host pointer).  n_codes is the length of
 * seq_codes in bytes.  X >= 0; X >= 2^30 means no pruning (X = infinity).  delta_b = 0
 * runs the unrestricted method, delta_b >= 1 the memory-restricted window of Sec. 3.
 * z_drop = 0 runs X-Drop alone; z_drop > 0 adds the Z-Drop rule that Sec. 1 names among the
 * X-Drop variants, in minimap2's definition: after each anti-diagonal, with (i', j') the
 * best cell so far and (i, j) the anti-diagonal's best live cell (lowest i on ties), the
 * side stops when S(i', j') - S(i, j) > z_drop + |gap| |(i - i') - (j - j')|; its result is
 * the best cell up to that anti-diagonal and carries flags bit 1. */
typedef struct {
    xd_alphabet alpha;
    uint32_t n_seqs;
    uint64_t n_codes;
    const uint8_t* seq_codes;
    const uint64_t* seq_offsets;
    const uint32_t* seq_lengths;
    uint32_t n_pairs;
    const xd_pair* pairs;
    xd_scoring scoring;
    int32_t X;
    uint32_t delta_b;
    int32_t z_drop;
} xd_batch;

/* Result of one side.  flags bit 0: the memory-restricted window was exceeded at least
 * once (the band was clipped to delta_b cells); bit 1: the Z-Drop rule ended the side. */
typedef struct {
    int32_t score;
    uint32_t h_ext, v_ext;
    uint32_t flags;
    uint64_t cells;      /* DP cells evaluated, S(0,0) included (pruned cells included) */
} xd_side;

typedef struct {
    xd_side left, right;
    int64_t total;       /* left.score + right.score + seed score */
} xd_result;

/* Per-context counters, cumulative since xd_create. */
typedef struct {
    uint64_t batches;            /* batches run (host and device entry points) */
    uint64_t pairs;
    uint64_t cells;              /* sum of xd_side.cells over all sides */
    uint64_t units_tier[3];      /* side extensions finished per stage (see xd_timing) */
    uint64_t escalations;        /* side extensions restarted in a wider tier */
    uint64_t kernel_launches;    /* kernels launched by the library */
    uint64_t host_launches;      /* launches of host batches (one per merged group) */
    uint64_t host_requests;      /* host batches those launches ran */
    uint64_t graph_captures;     /* device-entry pipelines captured as CUDA graphs */
    uint64_t graph_replays;      /* device-entry batches run by replaying a graph */
    uint64_t mixed_launches;     /* host launches that carried several parameter sets */
} xd_stats;

/* Create a context on cfg->device (NULL cfg = defaults).  A context plays the part of the
 * paper's wrapping driver class (Sec. 4.4, Multi-IPU Support): it owns the device, the
 * work queue that submitted batches share, and the streams that overlap transfers with
 * computation.  Allocates nothing large until the first batch.  Errors: XD_EINVAL
 * (out == NULL), XD_EDEVICE (no such device or the device is not compute capability 10.3). */
xd_status xd_create(const xd_config* cfg, xd_ctx** out);

/* Validate and enqueue a host batch (Sec. 4.4 tuples; Sec. 3 method).  Copies every input
 * to pinned staging memory before returning, so the caller may free its buffers at once.
 * On XD_OK *ticket identifies the batch for xd_poll.  A dispatcher thread of the context
 * launches waiting batches whenever one of the max_inflight launch slots is free; with
 * continuous batching, every waiting batch joins that launch (up to max_batch_pairs in
 * all): batches with the same alphabet, scoring, X, delta_b and z_drop as one batch of the
 * hot path, and up to four such parameter sets per launch (DNA and protein, several X), each
 * set's kernels on a stream of its own so that they run side by side on the device.  So
 * batches that arrive while others run share the next launch.  Each batch's results are the
 * same whether it ran alone or merged.  Launches overlap on the device as well (copies and
 * tails of one with the extension kernels of another); the fused persistent extension
 * kernels (large DNA sets) run one after another.  Errors: XD_EINVAL (codes out of the alphabet, a seed outside its sequence, X < 0,
 * a protein batch without matrix, scores that could leave the exact integer range),
 * XD_ENOMEM (admitted but unfinished batches would exceed store_bytes_cap, or 65536 batches
 * are outstanding: nothing was queued; retry after polling), XD_EDEVICE. */
xd_status xd_submit_batch(xd_ctx* ctx, const xd_batch* batch, uint64_t* ticket);

/* Resident sequence store: the detached sequence set of Sec. 4.1.1 kept on the device across
 * batches, one per alphabet.  xd_store_add copies n_seqs sequences (host codes, offsets
 * and lengths as in xd_batch), packs each distinct sequence once, and writes one handle per
 * input sequence to handles[n_seqs]; a sequence equal (same codes) to one already stored
 * gets the existing handle, so shared reads are stored once.  The store counts against
 * store_bytes_cap for the context's lifetime.  Synchronous.  Errors: XD_EINVAL (codes
 * outside the alphabet, sequences past n_codes), XD_ENOMEM (cap), XD_EDEVICE. */
xd_status xd_store_add(xd_ctx* ctx, xd_alphabet alpha, uint32_t n_seqs, uint64_t n_codes,
                       const uint8_t* seq_codes, const uint64_t* seq_offsets, const uint32_t* seq_lengths,
                       uint32_t* handles);

/* Sequences held and device bytes used by the resident store of one alphabet. */
xd_status xd_store_info(const xd_ctx* ctx, xd_alphabet alpha, uint64_t* n_seqs, uint64_t* device_bytes);

/* Seed tuples on the resident store: h_id / v_id are handles from xd_store_add. */
typedef struct {
    xd_alphabet alpha;
    uint32_t n_pairs;
    const xd_pair* pairs;
    xd_scoring scoring;
    int32_t X;
    uint32_t delta_b;
    int32_t z_drop;
} xd_pairs_batch;

/* As xd_submit_batch, but only the seed tuples travel: the sequences are already resident.
 * Poll with xd_poll.  Such batches merge with each other (same scoring, X and delta_b), not
 * with host batches.  Errors as xd_submit_batch; XD_EINVAL also for unknown handles. */
xd_status xd_submit_pairs(xd_ctx* ctx, const xd_pairs_batch* batch, uint64_t* ticket);

/* Completion side of the driver's shared work queue (Sec. 4.4: batches are submitted to a
 * queue and their results collected once the device has run them).
 * Wait up to wait_ms milliseconds (0 = do not wait, < 0 = wait without limit) for the
 * batch of `ticket`; on XD_OK copies n_pairs results to the host array `out` and retires
 * the ticket.  Returns XD_PENDING if not finished and wait_ms == 0, XD_ETIMEDOUT if the
 * wait expired, XD_ENOTFOUND for an unknown ticket, XD_EDEVICE if the launch that ran the
 * batch failed (the ticket is retired).  Thread-safe: several threads may poll at once. */
xd_status xd_poll(xd_ctx* ctx, uint64_t ticket, xd_result* out, int32_t wait_ms);

/* Run the whole hot path on device-resident inputs, asynchronously on `stream`
 * (a cudaStream_t, NULL = the legacy default stream): pack, build work units, order them
 * by cost, extend all sides, write n_pairs results to the device array d_out.  Scratch
 * comes from the context and is grown on demand (call xd_reserve first to keep
 * allocations out of a timed region).  Input validation happens on the device; read it
 * with xd_device_status after the stream has finished.  Not reentrant per context.
 * A call whose arguments (device pointers, sizes, scoring, X, delta_b, stream) repeat the
 * previous call's exactly is captured as a CUDA graph and later such calls replay it (the
 * buffers' contents may change between calls; on a non-default stream, when timing is
 * off).  The call may itself be captured into the caller's graph.
 * Errors: XD_EINVAL (null pointers, X < 0, protein without matrix), XD_ENOMEM, XD_EDEVICE. */
xd_status xd_run_device(xd_ctx* ctx, const xd_batch* dev_batch, xd_result* d_out, void* stream);

/* Several device batches in one pass of the hot path: as xd_run_device, but the n_batches
 * batches (device pointers as for xd_run_device) share one set of launches -- one packed
 * store, one cost-ordered list of all their side extensions, one persistent extension grid
 * -- so the long serial chains of one batch overlap the bulk work of the others instead of
 * leaving the GPU idle at the end of each batch (the load-balancing goal of Sec. 4.2 and the
 * shared work queue of Sec. 4.4, across batches).  The batches must share alphabet, scoring,
 * X and delta_b.  d_out receives the results of every pair in batch order: batch k's pairs
 * start at the sum of the earlier batches' n_pairs.  Each batch's results are identical to
 * running it alone.  Never captured as a graph by the library (the call may still be
 * captured into the caller's graph).  Not reentrant per context; shares the scratch of
 * xd_run_device (size it with xd_reserve for the sum of the batches).  Errors: XD_EINVAL
 * (null pointers, differing parameters, X < 0, protein without matrix, 2^31 or more pairs in
 * all), XD_ENOMEM, XD_EDEVICE; device-side validation as for xd_run_device. */
xd_status xd_run_device_many(xd_ctx* ctx, uint32_t n_batches, const xd_batch* batches, xd_result* d_out,
                             void* stream);

/* Pre-size the scratch used by xd_run_device for batches up to the given sizes. */
xd_status xd_reserve(xd_ctx* ctx, uint64_t n_codes, uint32_t n_seqs, uint32_t n_pairs,
                     uint32_t max_seq_len);

/* Synchronise the context's device work and report the device-side validation word of
 * the last xd_run_device batch: 0 = valid; bit 0 code outside the alphabet, bit 1 a bad
 * tuple (sequence id outside the table, seed outside its sequence, or a sequence whose
 * offset + length passes n_codes; such pairs get empty sides and no seed score), bit 2
 * score range exceeded, bit 3 a bounded device wait gave up. */
xd_status xd_device_status(xd_ctx* ctx, uint32_t* flags);

xd_status xd_get_stats(const xd_ctx* ctx, xd_stats* out);

/* Timing of the device pipeline, summed over every batch run since timing was enabled,
 * recorded with CUDA events on the stream the kernels are launched on.  Stage times are
 * in milliseconds.  The side extensions run in three stages: tier 0 = the first register
 * launch (the fused persistent grid of the first three register levels, or the first
 * level alone), tier 1 = the later register levels and the band tier (one warp per side
 * with a shared-memory ring), tier 2 = the generic tier (any band width, rows in global
 * memory).  tier_units / tier_cells are the side extensions each stage finished and their
 * DP cells; discarded_cells were evaluated by a level before a side was escalated without
 * an escalation record. */
typedef struct {
    uint64_t batches;            /* batches summed below */
    float pack_ms, units_ms, order_ms;
    float tier_ms[3];
    float totals_ms;
    float total_ms;
    uint64_t tier_units[3];
    uint64_t tier_cells[3];
    uint64_t escalations;
    uint64_t discarded_cells;
    uint64_t launches;           /* kernels the library launched */
    uint64_t window_shifts;      /* register-window re-centrings */
    uint64_t register_band_cells;   /* cells inside the band evaluated by the register levels */
    uint64_t register_slot_cells;   /* window slots those levels evaluated (anti-diagonals x window) */
} xd_timing;

/* enable != 0 synchronises the context, clears the timing sums and records stage events
 * for every following batch (up to 4096 batches); enable == 0 stops recording. */
xd_status xd_set_timing(xd_ctx* ctx, int32_t enable);

/* Synchronises the context's device work and returns the sums since timing was enabled.
 * XD_ENOTFOUND if no batch was recorded. */
xd_status xd_get_timing(xd_ctx* ctx, xd_timing* out);

/* Per-side timeline of xd_run_device batches (tracing; off by default).  With enable != 0
 * every following xd_run_device batch of the context records, for each side extension
 * (unit u: pair u / 2, right side for even u, left side for odd u) and each level that
 * worked on it, one xd_trace_rec at index u * 8 + level: level 0 - 4 the register levels
 * (0 - 3: the roles of the fused persistent grid), 5 the band tier, 6 the generic tier,
 * 7 the persistent grid's long-side role; records of levels that never saw the side stay
 * zero.  Each batch overwrites the previous one's records.  Tracing adds a clock read and a
 * 24-byte store per side and level, turns off graph capture, and allocates 192 bytes per
 * side extension of device memory (grown on demand, kept until xd_destroy). */
typedef struct {
    uint64_t start_ns;      /* globaltimer when the level took the side */
    uint32_t dur_ns;        /* until the level finished or escalated it */
    uint32_t diags;         /* anti-diagonals the level computed (register levels) */
    uint16_t window;        /* window slots of the level */
    uint16_t smid;          /* SM that ran it */
    uint8_t lanes;          /* lanes per side (band tier: warps) */
    uint8_t level;
    uint16_t outcome;       /* 1 the side finished here, 2 it was escalated */
} xd_trace_rec;

xd_status xd_set_trace(xd_ctx* ctx, int32_t enable);

/* Synchronises the last traced batch's stream and copies up to capacity bytes of its
 * records (8 xd_trace_rec per side extension) to the host buffer out; *n_units (may be
 * NULL) receives the number of side extensions.  XD_ENOTFOUND if no batch was traced. */
xd_status xd_get_trace(xd_ctx* ctx, void* out, uint64_t capacity, uint64_t* n_units);

/* Throughput microbenchmarks on the context's device: the measured integer/DPX
 * denominators of the alignment kernels' roofline (the method is bound by plain integer
 * arithmetic, Sec. 2.2 recurrence and X-Drop test).  op selects one instruction kind run
 * as eight independent dependency chains per thread:
 *   0 add, 1 max, 2 DPX add-max, 3 DPX 3-way max, 4 3-input logic, 5 multiply-add,
 *   6 compare + select (two instructions), 7 byte permute, 8 DPX add-max on 16x2,
 *   9 DPX 3-way max on 16x2, 10 max on 16x2,
 * or op 100 / 101: the register tiers' own cell update on 32 in-register slots for DNA /
 * protein scoring (every slot in the band, no band bookkeeping); op 102 / 103: the DNA /
 * protein update with 16-bit packed scores (two cells per register) including its dead
 * mask and best-cell key.
 * *rate receives operations (ops 100-103: cells) per second for the whole GPU.  Synchronous;
 * runs for a few tens of milliseconds.  Errors: XD_EINVAL (unknown op), XD_EDEVICE. */
xd_status xd_probe(xd_ctx* ctx, int32_t op, double* rate);

/* Autotuner of the batching scheme (Sec. 4.2 Batching: per-batch cost estimation and
 * distribution of the comparisons over the compute units; here the choice of launch
 * configuration for a class of batches).  Runs the host batch `sample` (pointers as for
 * xd_submit_batch) under candidate configurations -- the register-level chain (lanes per
 * side extension and window of every level, i.e. threads per alignment and band tile
 * width), the queue chunk of single-lane levels (1 - 64), the band tier's warps per side
 * (1 - 32, i.e. 32 - 1024 threads per alignment of the widest bands), the long-side head of
 * the persistent grid and its role mix -- three runs each on a stream of its own, and keeps the
 * fastest for the sample's bucket: alphabet x X (<= 15, <= 30, more) x longest side
 * (<= 2,048, <= 20,000, more) x size (< 8,192, < 65,536, < 1,048,576, more side extensions
 * in one launch) x memory-restricted window (unrestricted, delta_b <= 512, <= 2,048, more;
 * Sec. 3.3).  Every
 * candidate must reproduce the first candidate's results bit for bit, else the call fails
 * with XD_EDEVICE and keeps nothing.  The winner applies to later batches of the context;
 * if path is not NULL or empty it is also merged into the text table at path (created if
 * missing), which xd_config.tune_table loads.  *best_ms (may be NULL) receives the winner's
 * pipeline time in milliseconds.  Synchronous; allocates and frees its own device buffers.
 * Errors: XD_EINVAL (invalid or empty sample, unreadable or unwritable table), XD_ENOMEM,
 * XD_EDEVICE. */
xd_status xd_autotune(xd_ctx* ctx, const xd_batch* sample, const char* path, float* best_ms);

/* Allocation-free variant of xd_run_device (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory, such as code running in a host callback, a
 * pipeline whose device memory is fixed up front, or a process whose memory is managed by
 * another allocator under a strict budget).  It needs no context and calls no allocating
 * routine: the caller passes device inputs (dev_batch as for xd_run_device) and the device
 * output array d_out[n_pairs]; the anti-diagonal rows live in a 64 MiB array inside the
 * library that every GPU loading the library keeps until the process exits.  Results are
 * identical to xd_run_device.  It runs one warp per pair with the generic sweep, so it is
 * much slower than xd_run_device.
 *   max_side_len: an upper bound on every side's H length (h_seed and
 *   length(H) - h_seed - seed_len); XD_EINVAL if three rows of max_side_len + 1 scores do
 *   not fit the 64 MiB array.  Pairs with invalid inputs (bad ids, seeds outside their
 *   sequence, codes outside the alphabet, a side longer than max_side_len) get flags bit 31
 *   set on both sides instead of a result.
 * The first call in each CUDA context looks up the array's device address with that context
 * current (the calling thread's current context, or the current device's primary context
 * when none is current); make that first call before any stream capture.  A context made
 * later (for instance after cudaDeviceReset) gets its own look-up on its first call.  The array is shared by all calls: calls that overlap on the GPU (for instance
 * on two streams at once) race and give wrong results.  Asynchronous on `stream`.
 * Errors: XD_EINVAL, XD_EDEVICE. */
xd_status xd_run_device_noalloc(const xd_batch* dev_batch, uint32_t max_side_len, xd_result* d_out,
                                void* stream);

/* Tear down the driver of Sec. 4.4: stop the dispatcher, wait (at most 60 s) for launches in
 * flight, fail batches that never launched, then free every resource of the context.
 * XD_ETIMEDOUT if the wait expired; the context is freed either way and must not be used
 * again.  XD_EINVAL for ctx == NULL. */
xd_status xd_destroy(xd_ctx* ctx);

/* Last error message of the context (never NULL; "" when none), the host-side error report
 * of the Sec. 4.4 driver.  The string belongs to the library and stays valid until the
 * next call on the same context.  ctx may be NULL for errors of xd_create. */
const char* xd_last_error(const xd_ctx* ctx);

/* Library version string. */
const char* xd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XDROP_H */
