/* Synthetic sequence-pair construction for the seeded workloads (input generation only).
 *
 * Every pair owns an independent random stream seeded from (seed, pair index) with
 * SplitMix64 and advanced with xoshiro256**, so the output does not depend on how pairs
 * are split across threads.  Three pair kinds:
 *   0  related:   H random, V = mutate(H)
 *   1  dovetail:  H random, V = mutate(suffix of H of length ov) + random tail
 *   2  unrelated: H and V random, one shared k-mer planted at uniform positions
 * Mutation per source position: deletion (p_del), insertion before it (p_ins),
 * substitution (p_sub), else kept.  DNA indels have length 1, protein indels a geometric
 * length with mean 2.  The seed is a uniform k-mer inside the mutated region whose
 * positions all survived unchanged; if none did, one is planted by forcing a k-mer to
 * survive.  When a second seed is asked for, it is drawn last (so the sequences do not
 * change) uniformly among the clean k-mers that do not overlap the first; without one, the
 * first seed is repeated.  gen_pairs() is called twice: with out == NULL it only reports
 * lengths.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t next_u64(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static double next_f64(rng_t* r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static uint32_t next_below(rng_t* r, uint32_t n) { return (uint32_t)(next_f64(r) * n) % n; }
static void rng_seed(rng_t* r, uint64_t seed, uint64_t idx) {
    uint64_t x = seed * 0x632BE59BD9B4E019ULL ^ (idx + 0x1234567ULL) * 0x9E3779B97F4A7C15ULL;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}

typedef struct {
    int alphabet;                 /* 0 DNA, 1 protein */
    int k;
    uint64_t seed;
    const double* bg_cdf;         /* [20] protein residue CDF */
    const double* sub_cdf;        /* [20*20] protein P(b|a) CDF rows */
    /* per pair */
    const uint8_t* kind;
    const uint32_t* lh, *lv, *ov;
    const double* p_sub, *p_ins, *p_del;
    /* outputs */
    uint32_t* out_lv;             /* [n] length of V */
    uint32_t* h_seed, *v_seed;
    uint32_t* h_seed2, *v_seed2;  /* second seed per pair, or NULL */
    uint8_t* out;                 /* NULL on the sizing pass */
    const uint64_t* h_off, *v_off;
    uint64_t begin, end;
} job_t;

static uint8_t draw_residue(rng_t* r, const job_t* j) {
    if (j->alphabet == 0) return (uint8_t)(next_u64(r) >> 62);
    double u = next_f64(r);
    int a = 0;
    while (a < 19 && u >= j->bg_cdf[a]) a++;
    return (uint8_t)a;
}
static uint8_t draw_sub(rng_t* r, const job_t* j, uint8_t a) {
    if (j->alphabet == 0) return (uint8_t)((a + 1 + next_below(r, 3)) & 3);
    double u = next_f64(r);
    int b = 0;
    const double* c = j->sub_cdf + 20 * a;
    while (b < 19 && u >= c[b]) b++;
    if (b == a) b = (a + 1) % 20;   /* CDF row has zero mass on a; guard rounding */
    return (uint8_t)b;
}
static uint32_t indel_len(rng_t* r, const job_t* j) {
    if (j->alphabet == 0) return 1;
    uint32_t g = 1;
    while (g < 64 && next_f64(r) < 0.5) g++;
    return g;
}

enum { OP_KEEP = 0, OP_SUB = 1, OP_DEL = 2 };

/* Scratch per thread: ops/ins/subst value per source position. */
typedef struct { uint8_t* op; uint32_t* ins; uint8_t* val; uint32_t* tgt; uint64_t cap; } scratch_t;

static void ensure(scratch_t* s, uint64_t n) {
    if (n <= s->cap) return;
    free(s->op); free(s->ins); free(s->val); free(s->tgt);
    s->cap = n + 1024;
    s->op = malloc(s->cap); s->ins = malloc(4 * s->cap); s->val = malloc(s->cap);
    s->tgt = malloc(4 * s->cap);
}

static void do_pair(const job_t* j, uint64_t p, scratch_t* sc) {
    rng_t r;
    rng_seed(&r, j->seed, p);
    const uint32_t lh = j->lh[p], k = (uint32_t)j->k;
    uint8_t* H = j->out ? j->out + j->h_off[p] : NULL;
    uint8_t* V = j->out ? j->out + j->v_off[p] : NULL;
    /* H is drawn first in every kind */
    ensure(sc, lh);
    uint8_t* hres = malloc(lh ? lh : 1);
    for (uint32_t t = 0; t < lh; t++) hres[t] = draw_residue(&r, j);
    if (H) memcpy(H, hres, lh);

    if (j->kind[p] == 2) {
        uint32_t lv = j->lv[p];
        uint32_t hs = next_below(&r, lh - k + 1), vs = next_below(&r, lv - k + 1);
        j->out_lv[p] = lv;
        j->h_seed[p] = hs; j->v_seed[p] = vs;
        if (j->h_seed2) { j->h_seed2[p] = hs; j->v_seed2[p] = vs; }
        for (uint32_t t = 0; t < lv; t++) {
            uint8_t c = draw_residue(&r, j);
            if (V) V[t] = c;
        }
        if (V) memcpy(V + vs, hres + hs, k);
        free(hres);
        return;
    }
    /* kinds 0 and 1: mutate source region [src0, lh) of H */
    uint32_t src0 = j->kind[p] == 1 ? lh - j->ov[p] : 0;
    uint32_t ls = lh - src0;
    const uint8_t* src = hres + src0;
    double pd = j->p_del[p], pi = j->p_ins[p], ps = j->p_sub[p];
    uint8_t* op = sc->op; uint32_t* ins = sc->ins; uint8_t* val = sc->val; uint32_t* tgt = sc->tgt;
    for (uint32_t t = 0; t < ls; t++) { op[t] = OP_KEEP; ins[t] = 0; val[t] = src[t]; }
    for (uint32_t t = 0; t < ls; t++) {
        double u = next_f64(&r);
        if (u < pd) {
            uint32_t g = indel_len(&r, j);
            for (uint32_t q = t; q < ls && q < t + g; q++) op[q] = OP_DEL;
        } else if (u < pd + pi) {
            ins[t] = indel_len(&r, j);
        } else if (u < pd + pi + ps) {
            if (op[t] != OP_DEL) { op[t] = OP_SUB; val[t] = draw_sub(&r, j, src[t]); }
        }
    }
    /* seed: uniform among clean k-mers, else plant one */
    uint64_t n_clean = 0;
    uint32_t run = 0;
    for (uint32_t t = 0; t < ls; t++) {
        int clean = op[t] == OP_KEEP && ins[t] == 0;
        run = clean ? run + 1 : 0;
        if (run >= k) n_clean++;
    }
    uint32_t seed_src;
    double u = next_f64(&r);
    if (n_clean > 0) {
        uint64_t pick = (uint64_t)(u * (double)n_clean);
        if (pick >= n_clean) pick = n_clean - 1;
        run = 0;
        seed_src = 0;
        for (uint32_t t = 0; t < ls; t++) {
            int clean = op[t] == OP_KEEP && ins[t] == 0;
            run = clean ? run + 1 : 0;
            if (run >= k) { if (pick == 0) { seed_src = t + 1 - k; break; } pick--; }
        }
    } else {
        seed_src = (uint32_t)(u * (double)(ls - k + 1));
        if (seed_src > ls - k) seed_src = ls - k;
        for (uint32_t q = seed_src; q < seed_src + k; q++) { op[q] = OP_KEEP; ins[q] = 0; val[q] = src[q]; }
    }
    /* emit mutated region */
    uint32_t o = 0, seed_tgt = 0;
    for (uint32_t t = 0; t < ls; t++) {
        for (uint32_t q = 0; q < ins[t]; q++) { uint8_t c = draw_residue(&r, j); if (V) V[o] = c; o++; }
        if (t == seed_src) seed_tgt = o;
        tgt[t] = o;
        if (op[t] != OP_DEL) { if (V) V[o] = val[t]; o++; }
    }
    if (j->kind[p] == 1) {           /* dovetail: random tail up to the target length */
        uint32_t lv = j->lv[p];
        for (; o < lv; o++) { uint8_t c = draw_residue(&r, j); if (V) V[o] = c; }
    }
    j->out_lv[p] = o;
    j->h_seed[p] = src0 + seed_src;
    j->v_seed[p] = seed_tgt;
    if (j->h_seed2) {
        /* second seed: a clean k-mer that does not overlap the first, drawn last */
        uint64_t n2 = 0;
        run = 0;
        for (uint32_t t = 0; t < ls; t++) {
            int clean = op[t] == OP_KEEP && ins[t] == 0;
            run = clean ? run + 1 : 0;
            if (run >= k) {
                uint32_t st = t + 1 - k;
                if (st + k <= seed_src || st >= seed_src + k) n2++;
            }
        }
        uint32_t s2 = seed_src;
        double u2 = next_f64(&r);
        if (n2 > 0) {
            uint64_t pick = (uint64_t)(u2 * (double)n2);
            if (pick >= n2) pick = n2 - 1;
            run = 0;
            for (uint32_t t = 0; t < ls; t++) {
                int clean = op[t] == OP_KEEP && ins[t] == 0;
                run = clean ? run + 1 : 0;
                if (run >= k) {
                    uint32_t st = t + 1 - k;
                    if (st + k <= seed_src || st >= seed_src + k) {
                        if (pick == 0) { s2 = st; break; }
                        pick--;
                    }
                }
            }
        }
        j->h_seed2[p] = src0 + s2;
        j->v_seed2[p] = s2 == seed_src ? seed_tgt : tgt[s2];
    }
    free(hres);
}

static void* worker(void* arg) {
    job_t* j = (job_t*)arg;
    scratch_t sc = {0};
    for (uint64_t p = j->begin; p < j->end; p++) do_pair(j, p, &sc);
    free(sc.op); free(sc.ins); free(sc.val); free(sc.tgt);
    return NULL;
}

int gen_pairs(int alphabet, int k, uint64_t seed, const double* bg_cdf, const double* sub_cdf,
              uint64_t n, const uint8_t* kind, const uint32_t* lh, const uint32_t* lv,
              const uint32_t* ov, const double* p_sub, const double* p_ins, const double* p_del,
              uint32_t* out_lv, uint32_t* h_seed, uint32_t* v_seed, uint32_t* h_seed2, uint32_t* v_seed2,
              uint8_t* out, const uint64_t* h_off, const uint64_t* v_off, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < n_threads; t++) {
        job_t* j = &jobs[t];
        j->alphabet = alphabet; j->k = k; j->seed = seed; j->bg_cdf = bg_cdf; j->sub_cdf = sub_cdf;
        j->kind = kind; j->lh = lh; j->lv = lv; j->ov = ov;
        j->p_sub = p_sub; j->p_ins = p_ins; j->p_del = p_del;
        j->out_lv = out_lv; j->h_seed = h_seed; j->v_seed = v_seed;
        j->h_seed2 = h_seed2; j->v_seed2 = v_seed2;
        j->out = out; j->h_off = h_off; j->v_off = v_off;
        j->begin = n * (uint64_t)t / n_threads;
        j->end = n * (uint64_t)(t + 1) / n_threads;
        pthread_create(&th[t], NULL, worker, j);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    return 0;
}
