/* X-Drop seed-extension oracle: plain, slow, single-threaded C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU-baseline
 * leg may load this code.  It shares no code, header, table or helper with the CUDA
 * library; it reads the same residue codes and seed tuples and nothing else.
 *
 * What it computes (paper, Sec. 2.2 and Sec. 3, Algorithm 1):
 *   - Score matrix S over prefixes of the side strings H (length m, index i) and
 *     V (length n, index j): S(0,0) = 0, cells outside the matrix are -inf (Sec. 2.2),
 *     S(i,j) = max{ S(i-1,j-1) + Sim(H[i-1], V[j-1]),  S(i,j-1) + gap,  S(i-1,j) + gap }
 *     (the recurrence of Sec. 2.2, read as a maximum; gap is a negative score added).
 *   - Anti-diagonal sweep d = i + j = 1, 2, ... starting from S(0,0) (Zhang's traversal,
 *     Sec. 2.2); each cell needs only the two previous anti-diagonals.
 *   - X-Drop rule: with T the best score over the completed anti-diagonals, a cell with
 *     S(i,j) < T - X is set to -inf (Sec. 2.2; Algorithm 1 keeps T' while sweeping and
 *     copies it into T only after the anti-diagonal is done).
 *   - Live band: the next anti-diagonal covers i from the first live index L to the last
 *     live index U plus one, clipped to the matrix (Algorithm 1, the L/U update).
 *   - Termination: stop when an anti-diagonal has no live cell, or at d = m + n.
 *   - Memory-restricted variant with window delta_b (Sec. 3, Algorithm 1): when the band
 *     of an anti-diagonal is wider than delta_b cells, only delta_b cells are kept, the
 *     window being realigned to the position of the previous anti-diagonal's best cell;
 *     the result then carries the overflow flag.
 *   - Left/right extension: each seed splits a pair into a right extension read forward
 *     from the seed end and a left extension read backward from the seed start, through
 *     an index transform op(.) rather than reversed copies (Sec. 3, the op(.) paragraph).
 *   - Z-Drop, optional (z > 0): the paper names the Z-Drop variant among the X-Drop
 *     variants genomic pipelines use (Sec. 1) and cites minimap2 for it; its definition is
 *     minimap2's (Li 2018): with (i', j') the best cell so far and (i, j) the best cell of
 *     the anti-diagonal just completed, the extension stops when
 *     S(i', j') - S(i, j) > Z + e |(i - i') - (j - j')|, e the gap-extension penalty (here
 *     the linear gap's |gap|).  It is applied after each anti-diagonal on top of the X-Drop
 *     pruning; the result is the best cell up to and including that anti-diagonal, flag bit 1.
 *
 * Readings where the paper is silent or garbled (each one is listed in the design notes):
 *   R1 cell (i,j) with i,j >= 1 pairs H[i-1] with V[j-1]; i indexes H.
 *   R2 the X-Drop comparison is strict (<) and uses T of completed anti-diagonals.
 *   R3 next band: lo = max(L, d-n, 0), hi = min(U+1, m, d) in prefix coordinates.
 *   R4 end cell tie-break: the first anti-diagonal that reaches the final best score,
 *      lowest i on it (strictly-greater update in increasing i).
 *   R5 per-side score excludes the seed; pair total = left + right + seed score.
 *   R6 restricted overflow: centre on b = lowest-index maximum live cell of the previous
 *      anti-diagonal: lo' = max(lo, min(b - floor(delta/2), hi - delta + 1)),
 *      hi' = lo' + delta - 1; flag bit 0.
 *   R7 the cell count includes every cell evaluated (pruned ones too) plus S(0,0).
 *   R8 Z-Drop: (i, j) is the anti-diagonal's best live cell, lowest i on ties; (i', j') is
 *      the best cell after that anti-diagonal's update of T (so an anti-diagonal that sets
 *      a new best never triggers it); the comparison is strict.
 *
 * Scores are int64; -inf is represented by an explicit "not live" state, never by an
 * arithmetic sentinel.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t score;      /* best score of the side (seed excluded) */
    uint32_t h_ext;     /* i of the best cell: extension length on H */
    uint32_t v_ext;     /* j of the best cell: extension length on V */
    uint32_t flags;     /* bit 0: restricted window was exceeded */
    uint64_t cells;     /* cells evaluated, S(0,0) included */
} orc_side;

/* One anti-diagonal: values for i in [lo, hi]; live[i] says whether S > -inf. */
typedef struct {
    int64_t* val;
    uint8_t* live;
    int64_t lo, hi;     /* computed range; empty when lo > hi */
} orc_diag;

static int diag_live(const orc_diag* a, int64_t i) {
    return i >= a->lo && i <= a->hi && a->live[i];
}

/* Side strings through op(.): H_side[t] = h[t * h_step], V_side[t] = v[t * v_step]. */
typedef struct {
    const uint8_t* h; int64_t h_step; int64_t m;
    const uint8_t* v; int64_t v_step; int64_t n;
} orc_strings;

static uint8_t side_h(const orc_strings* s, int64_t t) { return s->h[t * s->h_step]; }
static uint8_t side_v(const orc_strings* s, int64_t t) { return s->v[t * s->v_step]; }

/* Extend one side.  sim is a dense alpha x alpha table.  z > 0: Z-Drop with Z = z. */
int orc_extend_z(const uint8_t* h, int64_t h_step, int64_t m,
                 const uint8_t* v, int64_t v_step, int64_t n,
                 const int32_t* sim, int alpha, int32_t gap, int32_t X, uint32_t delta,
                 int32_t z, orc_side* out)
{
    orc_strings s = { h, h_step, m, v, v_step, n };
    orc_diag buf[3];
    for (int k = 0; k < 3; k++) {
        buf[k].val = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
        buf[k].live = (uint8_t*)calloc((size_t)m + 1, 1);
        if (!buf[k].val || !buf[k].live) return -1;
        buf[k].lo = 1; buf[k].hi = 0;
    }
    orc_diag* P2 = &buf[0];     /* anti-diagonal d-2 */
    orc_diag* P1 = &buf[1];     /* anti-diagonal d-1 */
    orc_diag* C = &buf[2];      /* anti-diagonal d   */

    /* initialisation: S(0,0) = 0, T = 0, band [0, 0] */
    P1->lo = 0; P1->hi = 0; P1->val[0] = 0; P1->live[0] = 1;
    int64_t T = 0, best = 0, best_i = 0, best_j = 0;
    int64_t L = 0, U = 0;
    uint64_t cells = 1;
    uint32_t flags = 0;

    for (int64_t d = 1; d <= m + n; d++) {
        int64_t lo = L, hi = U + 1;
        if (d - n > lo) lo = d - n;
        if (lo < 0) lo = 0;
        if (m < hi) hi = m;
        if (d < hi) hi = d;

        if (delta > 0 && hi - lo + 1 > (int64_t)delta) {
            /* memory-restricted window: realign to the previous anti-diagonal's best cell */
            flags |= 1u;
            int64_t b = -1, bv = 0;
            for (int64_t i = P1->lo; i <= P1->hi; i++)
                if (P1->live[i] && (b < 0 || P1->val[i] > bv)) { b = i; bv = P1->val[i]; }
            int64_t centred = b - (int64_t)(delta / 2);
            int64_t latest = hi - (int64_t)delta + 1;
            int64_t start = centred < latest ? centred : latest;
            if (start > lo) lo = start;
            hi = lo + (int64_t)delta - 1;
        }

        int64_t T_new = T;          /* T' of Algorithm 1 */
        int64_t first = -1, last = -1;
        C->lo = lo; C->hi = hi;
        for (int64_t i = lo; i <= hi; i++) {
            int64_t j = d - i;
            int has = 0;
            int64_t c = 0;
            if (i >= 1 && j >= 1 && diag_live(P2, i - 1)) {           /* S(i-1, j-1) + Sim */
                int64_t t = P2->val[i - 1] + sim[side_h(&s, i - 1) * alpha + side_v(&s, j - 1)];
                if (!has || t > c) { c = t; has = 1; }
            }
            if (i >= 1 && diag_live(P1, i - 1)) {                     /* S(i-1, j) + gap */
                int64_t t = P1->val[i - 1] + gap;
                if (!has || t > c) { c = t; has = 1; }
            }
            if (j >= 1 && diag_live(P1, i)) {                         /* S(i, j-1) + gap */
                int64_t t = P1->val[i] + gap;
                if (!has || t > c) { c = t; has = 1; }
            }
            cells++;
            int live = has && !(c < T - (int64_t)X);                  /* X-Drop condition */
            C->live[i] = (uint8_t)live;
            C->val[i] = live ? c : 0;
            if (live) {
                if (first < 0) first = i;
                last = i;
                if (c > T_new) { T_new = c; best = c; best_i = i; best_j = j; }
            }
        }
        if (first < 0) break;                                         /* no live cell */
        L = first; U = last;
        T = T_new;
        if (z > 0) {
            /* Z-Drop: this anti-diagonal's best live cell against the best cell so far */
            int64_t zi = -1, zv = 0;
            for (int64_t i = lo; i <= hi; i++)
                if (C->live[i] && (zi < 0 || C->val[i] > zv)) { zi = i; zv = C->val[i]; }
            int64_t shift = (zi - best_i) - ((d - zi) - best_j);
            if (shift < 0) shift = -shift;
            if (best - zv > (int64_t)z + (-(int64_t)gap) * shift) { flags |= 2u; break; }
        }
        orc_diag* old = P2; P2 = P1; P1 = C; C = old;
    }

    out->score = (int32_t)best;
    out->h_ext = (uint32_t)best_i;
    out->v_ext = (uint32_t)best_j;
    out->flags = flags;
    out->cells = cells;
    for (int k = 0; k < 3; k++) { free(buf[k].val); free(buf[k].live); }
    return 0;
}

int orc_extend(const uint8_t* h, int64_t h_step, int64_t m,
               const uint8_t* v, int64_t v_step, int64_t n,
               const int32_t* sim, int alpha, int32_t gap, int32_t X, uint32_t delta,
               orc_side* out)
{
    return orc_extend_z(h, h_step, m, v, v_step, n, sim, alpha, gap, X, delta, 0, out);
}

/* Similarity table: DNA (alpha 4) from match/mismatch, protein (alpha 20) from the
 * 20x20 substitution matrix given row-major (Sec. 2.2 scoring; BLOSUM62 in Sec. 5.3). */
static void build_sim(int alpha, int32_t match, int32_t mismatch, const int8_t* matrix, int32_t* sim)
{
    for (int a = 0; a < alpha; a++)
        for (int b = 0; b < alpha; b++)
            sim[a * alpha + b] = alpha == 20 ? (int32_t)matrix[a * 20 + b] : (a == b ? match : mismatch);
}

/* A batch of seed extensions e_c = (H, V, H_s, V_s) plus the seed length (Sec. 4.4).
 * pairs holds 5 uint32 per pair: h_id, v_id, h_seed, v_seed, seed_len.  Pairs
 * [first, first + count) are processed; results are written at the same indices.
 * Right side: H_R[t] = H[h_seed + k + t], V_R[t] = V[v_seed + k + t].
 * Left side:  H_L[t] = H[h_seed - 1 - t], V_L[t] = V[v_seed - 1 - t].
 * total = left.score + right.score + sum of Sim over the seed. */
int orc_batch_z(int alpha, const uint8_t* codes, const uint64_t* offsets, const uint32_t* lengths,
                const uint32_t* pairs, uint64_t first, uint64_t count,
                int32_t match, int32_t mismatch, int32_t gap, const int8_t* matrix,
                int32_t X, uint32_t delta, int32_t z,
                orc_side* left, orc_side* right, int64_t* total)
{
    if (alpha != 4 && alpha != 20) return -1;
    if (alpha == 20 && !matrix) return -1;
    int32_t sim[400];
    build_sim(alpha, match, mismatch, matrix, sim);
    for (uint64_t p = first; p < first + count; p++) {
        const uint32_t* e = pairs + 5 * p;
        const uint8_t* H = codes + offsets[e[0]];
        const uint8_t* V = codes + offsets[e[1]];
        int64_t lh = lengths[e[0]], lv = lengths[e[1]];
        int64_t hs = e[2], vs = e[3], k = e[4];
        if (hs + k > lh || vs + k > lv) return -2;
        int rc = orc_extend_z(H + hs + k, 1, lh - hs - k, V + vs + k, 1, lv - vs - k,
                              sim, alpha, gap, X, delta, z, &right[p]);
        if (rc) return rc;
        rc = orc_extend_z(hs > 0 ? H + hs - 1 : H, -1, hs, vs > 0 ? V + vs - 1 : V, -1, vs,
                          sim, alpha, gap, X, delta, z, &left[p]);
        if (rc) return rc;
        int64_t seed_score = 0;
        for (int64_t t = 0; t < k; t++) seed_score += sim[H[hs + t] * alpha + V[vs + t]];
        total[p] = (int64_t)left[p].score + (int64_t)right[p].score + seed_score;
    }
    return 0;
}

int orc_batch(int alpha, const uint8_t* codes, const uint64_t* offsets, const uint32_t* lengths,
              const uint32_t* pairs, uint64_t first, uint64_t count,
              int32_t match, int32_t mismatch, int32_t gap, const int8_t* matrix,
              int32_t X, uint32_t delta,
              orc_side* left, orc_side* right, int64_t* total)
{
    return orc_batch_z(alpha, codes, offsets, lengths, pairs, first, count, match, mismatch, gap, matrix,
                       X, delta, 0, left, right, total);
}
