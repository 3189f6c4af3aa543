/*
 * Plain CPU oracle of Scrooge's windowed GenASM alignment.
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA path, never to stand
 * in for it: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code with the CUDA library.
 *
 * What it computes, step by step in the paper's order and notation:
 *   - pattern masks PM[X] (Section 2.2.1): bit j of PM[X] is 0 iff pattern[j] == X;
 *   - GenASM-DC, Algorithm 1: the whole (n+1) x (k+1) table R of m-bit
 *     vectors, every row d = 0..k (no early termination), keeping the three
 *     GenASM edge vectors I, D and M of every entry as GenASM-TB expects
 *     (Section 2.2.2: S is D shifted, so only I, D, M are kept);
 *   - the edit distance: the smallest d whose entry R[0][d] has a 0 in its
 *     first (most significant) bit, Algorithm 1's last step;
 *   - GenASM-TB (Section 2.2.2): follow 0s of the stored edges from that entry
 *     toward the north-east corner, naming each crossed edge as an edit;
 *   - the windowing heuristic (Section 2.2.3): align W-character windows,
 *     keep the traceback only through the first W-O characters, continue with
 *     the rest of both strings.
 *
 * Readings where the paper is silent:
 *   - bit order: bit j = 0 is the most significant bit; "<< 1" moves bit j+1
 *     into bit j and shifts a 0 into bit m-1;
 *   - "distance" is the edit distance with a free end in the text: by
 *     Theorem 1 with the initial column R[n][d] = 1..1 << d, bit j of R[i][d]
 *     is 0 iff some prefix of text[i:n) is within d edits of pattern[j:m);
 *   - the traceback of a window stops as soon as it has consumed W-O text
 *     characters, or W-O pattern characters, or the whole pattern window;
 *     the next window starts where it stopped (text and pattern cursors move
 *     by the characters consumed);
 *   - when several edges hold a 0, the traceback takes M, then S, then I,
 *     then D;
 *   - a shift by d >= m of the all-ones vector gives all zeros;
 *   - the reported edit count is the number of X, I and D operations of the
 *     stitched CIGAR; a window with no d <= k fails the whole pair (-1).
 *
 * Bitvectors are arrays of two 64-bit words, bit j in word j / 64 at position
 * 63 - j % 64, so windows up to W = 128 fit. Bits j >= m are kept 0.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXW 128
#define ORC_NWORD 2

/* CIGAR operation codes (SAM): '=' match, 'X' substitution, 'I' consumes
 * only the pattern (read), 'D' consumes only the text (reference). */
#define ORC_OP_I 1
#define ORC_OP_D 2
#define ORC_OP_EQ 7
#define ORC_OP_X 8

typedef struct {
    uint64_t w[ORC_NWORD];
} bv;

static int bv_bit(const bv *v, int j) {
    if (j < 0 || j >= ORC_MAXW) return 0; /* bit m (and beyond) is the shifted-in 0 */
    return (int)((v->w[j >> 6] >> (63 - (j & 63))) & 1u);
}

static void bv_setbit(bv *v, int j) { v->w[j >> 6] |= (uint64_t)1 << (63 - (j & 63)); }

static bv bv_zero(void) {
    bv r;
    memset(&r, 0, sizeof r);
    return r;
}

/* "<< 1": bit j takes bit j+1, bit 127 takes 0. */
static bv bv_shl1(bv a) {
    bv r;
    r.w[0] = (a.w[0] << 1) | (a.w[1] >> 63);
    r.w[1] = a.w[1] << 1;
    return r;
}

static bv bv_and(bv a, bv b) {
    bv r;
    for (int k = 0; k < ORC_NWORD; ++k) r.w[k] = a.w[k] & b.w[k];
    return r;
}

static bv bv_or(bv a, bv b) {
    bv r;
    for (int k = 0; k < ORC_NWORD; ++k) r.w[k] = a.w[k] | b.w[k];
    return r;
}

/* The m-bit all-ones vector shifted left by d: bits j < m - d are 1. */
static bv bv_ones_shl(int m, int d) {
    bv r = bv_zero();
    for (int j = 0; j < m - d; ++j) bv_setbit(&r, j);
    return r;
}

/* One window's GenASM-DC table with the GenASM traceback edges. */
typedef struct {
    int n, m, k;
    bv pm[4];
    bv *R;  /* (n+1) x (k+1): R[i*(k+1)+d] */
    bv *EI; /* insertion edge  I = R[i][d-1] << 1        (d >= 1, i <= n) */
    bv *ED; /* deletion edge   D = R[i+1][d-1]           (d >= 1, i < n)  */
    bv *EM; /* match edge      M = (R[i+1][d] << 1) | PM (i < n)          */
} orc_table;

#define AT(tab, i, d) ((size_t)(i) * (size_t)((tab)->k + 1) + (size_t)(d))

/* Pattern masks, Section 2.2.1: bit j of PM[X] is 0 iff pattern[j] == X. */
static void build_pattern_masks(const uint8_t *pattern, int m, bv pm[4]) {
    for (int x = 0; x < 4; ++x) {
        pm[x] = bv_zero();
        for (int j = 0; j < m; ++j)
            if (pattern[j] != x) bv_setbit(&pm[x], j);
    }
}

/* Algorithm 1 over text[0:n), pattern[0:m), rows d = 0..k, all of them. */
static void genasm_dc(const uint8_t *text, int n, const uint8_t *pattern, int m, int k, orc_table *t) {
    t->n = n;
    t->m = m;
    t->k = k;
    build_pattern_masks(pattern, m, t->pm);
    /* right column: R[n][d] = 1..1 << d for all 0 <= d <= k */
    for (int d = 0; d <= k; ++d) t->R[AT(t, n, d)] = bv_ones_shl(m, d);
    /* the insertion edges of the right column, used when the text is exhausted */
    for (int d = 1; d <= k; ++d) t->EI[AT(t, n, d)] = bv_shl1(t->R[AT(t, n, d - 1)]);
    for (int i = n - 1; i >= 0; --i) {
        bv cur = t->pm[text[i]];
        /* top row: exact match */
        bv M0 = bv_or(bv_shl1(t->R[AT(t, i + 1, 0)]), cur);
        t->EM[AT(t, i, 0)] = M0;
        t->R[AT(t, i, 0)] = M0;
        for (int d = 1; d <= k; ++d) {
            bv I = bv_shl1(t->R[AT(t, i, d - 1)]);
            bv D = t->R[AT(t, i + 1, d - 1)];
            bv S = bv_shl1(t->R[AT(t, i + 1, d - 1)]);
            bv M = bv_or(bv_shl1(t->R[AT(t, i + 1, d)]), cur);
            t->EI[AT(t, i, d)] = I;
            t->ED[AT(t, i, d)] = D;
            t->EM[AT(t, i, d)] = M;
            t->R[AT(t, i, d)] = bv_and(bv_and(I, D), bv_and(S, M));
        }
    }
}

/* Smallest d with a 0 in the first bit of R[0][d]; -1 if none up to k. */
static int edit_distance_row(const orc_table *t) {
    for (int d = 0; d <= t->k; ++d)
        if (bv_bit(&t->R[AT(t, 0, d)], 0) == 0) return d;
    return -1;
}

typedef struct {
    uint32_t *ops; /* run-length CIGAR, (len << 4) | op */
    int64_t cap, len;
    int overflow;
    int64_t edits;
} orc_cigar;

static void cigar_push(orc_cigar *c, int op) {
    if (op != ORC_OP_EQ) c->edits += 1;
    if (c->len > 0 && (int)(c->ops[c->len - 1] & 15u) == op) {
        c->ops[c->len - 1] += 16u;
        return;
    }
    if (c->len >= c->cap) {
        c->overflow = 1;
        return;
    }
    c->ops[c->len++] = (1u << 4) | (uint32_t)op;
}

/*
 * GenASM-TB over one window (Section 2.2.2). Starts at (i, j, d) = (0, 0,
 * d_opt) and crosses one edge per step, preferring M, S, I, D in that order:
 *   M: bit j of M[i][d] is 0      -> '=' (i+1, j+1, d)
 *   S: bit j of (D[i][d] << 1) 0  -> 'X' (i+1, j+1, d-1)
 *   I: bit j of I[i][d] is 0      -> 'I' (i,   j+1, d-1)
 *   D: bit j of D[i][d] is 0      -> 'D' (i+1, j,   d-1)
 * and stops once j == m, or i == limit, or j == limit (limit = W - O).
 * Returns the characters consumed in *ci (text) and *cj (pattern).
 */
static int genasm_tb(const orc_table *t, int d_opt, int limit, orc_cigar *out, int *ci, int *cj) {
    int i = 0, j = 0, d = d_opt;
    while (j < t->m && i < limit && j < limit) {
        if (i < t->n && bv_bit(&t->EM[AT(t, i, d)], j) == 0) {
            cigar_push(out, ORC_OP_EQ);
            i += 1;
            j += 1;
        } else if (d > 0 && i < t->n && bv_bit(&t->ED[AT(t, i, d)], j + 1) == 0) {
            cigar_push(out, ORC_OP_X);
            i += 1;
            j += 1;
            d -= 1;
        } else if (d > 0 && bv_bit(&t->EI[AT(t, i, d)], j) == 0) {
            cigar_push(out, ORC_OP_I);
            j += 1;
            d -= 1;
        } else if (d > 0 && i < t->n && bv_bit(&t->ED[AT(t, i, d)], j) == 0) {
            cigar_push(out, ORC_OP_D);
            i += 1;
            d -= 1;
        } else {
            return -1; /* no 0 edge: impossible by Theorem 1 */
        }
    }
    *ci = i;
    *cj = j;
    return 0;
}

typedef struct {
    orc_table tab;
} orc_work;

static int work_init(orc_work *w, int k) {
    size_t cells = (size_t)(ORC_MAXW + 1) * (size_t)(k + 1);
    w->tab.R = (bv *)calloc(cells, sizeof(bv));
    w->tab.EI = (bv *)calloc(cells, sizeof(bv));
    w->tab.ED = (bv *)calloc(cells, sizeof(bv));
    w->tab.EM = (bv *)calloc(cells, sizeof(bv));
    return (w->tab.R && w->tab.EI && w->tab.ED && w->tab.EM) ? 0 : -1;
}

static void work_free(orc_work *w) {
    free(w->tab.R);
    free(w->tab.EI);
    free(w->tab.ED);
    free(w->tab.EM);
}

static int min_int(int64_t a, int64_t b) { return (int)(a < b ? a : b); }

/*
 * The windowing heuristic (Section 2.2.3) over one pair. Returns 0 on
 * success, 1 if some window has no edit distance within k (the pair fails:
 * edit count -1, empty CIGAR), -2 on CIGAR overflow, -1 on an internal error.
 */
static int align_pair(orc_work *w, const uint8_t *text, int64_t n, const uint8_t *pattern, int64_t m,
                      int W, int O, int k, orc_cigar *cig, int64_t *text_consumed, int64_t *n_windows,
                      int32_t *dopt_log, int32_t *wedit_log, int64_t dopt_cap) {
    int64_t ti = 0, pj = 0, win = 0;
    while (pj < m) {
        int nw = min_int(W, n - ti);
        int mw = min_int(W, m - pj);
        genasm_dc(text + ti, nw, pattern + pj, mw, k, &w->tab);
        int d_opt = edit_distance_row(&w->tab);
        if (dopt_log && win < dopt_cap) dopt_log[win] = d_opt;
        win += 1;
        if (d_opt < 0) {
            cig->len = 0;
            cig->edits = 0;
            *text_consumed = 0;
            *n_windows = win;
            return 1;
        }
        int ci = 0, cj = 0;
        const int64_t edits_before = cig->edits;
        if (genasm_tb(&w->tab, d_opt, W - O, cig, &ci, &cj) != 0) return -1;
        /* edits of the kept traceback: the rows it descended below d_opt */
        if (wedit_log && win - 1 < dopt_cap) wedit_log[win - 1] = (int32_t)(cig->edits - edits_before);
        ti += ci;
        pj += cj;
    }
    *text_consumed = ti;
    *n_windows = win;
    return cig->overflow ? -2 : 0;
}

/* ---------------------------------------------------------------- exports */

/* Full Algorithm 1 table of one window as bytes: bits[(i*(k+1)+d)*m + j]. */
int orc_window_table(const uint8_t *text, int n, const uint8_t *pattern, int m, int k, uint8_t *bits,
                     int *d_opt) {
    if (n < 0 || m < 0 || n > ORC_MAXW || m > ORC_MAXW || k < 0) return -1;
    orc_work w;
    if (work_init(&w, k) != 0) return -1;
    genasm_dc(text, n, pattern, m, k, &w.tab);
    for (int i = 0; i <= n; ++i)
        for (int d = 0; d <= k; ++d)
            for (int j = 0; j < m; ++j)
                bits[((size_t)i * (size_t)(k + 1) + (size_t)d) * (size_t)m + (size_t)j] =
                    (uint8_t)bv_bit(&w.tab.R[AT(&w.tab, i, d)], j);
    *d_opt = edit_distance_row(&w.tab);
    work_free(&w);
    return 0;
}

/* Pattern masks of one pattern window as bytes: pm[x*m + j]. */
int orc_pattern_masks(const uint8_t *pattern, int m, uint8_t *pm) {
    if (m < 0 || m > ORC_MAXW) return -1;
    bv v[4];
    build_pattern_masks(pattern, m, v);
    for (int x = 0; x < 4; ++x)
        for (int j = 0; j < m; ++j) pm[x * m + j] = (uint8_t)bv_bit(&v[x], j);
    return 0;
}

static int check_args(int W, int O, int k) {
    if (W < 1 || W > ORC_MAXW) return -1;
    if (O < 0 || O >= W) return -1;
    if (k < 0 || k > W) return -1;
    return 0;
}

/* One pair; cigar must hold cigar_cap runs. Returns the align_pair status.
 * Optional per-window logs (dopt_cap entries each, may be NULL): dopt_log the
 * window's edit distance, wedit_log the edits its kept traceback took. */
int orc_align_pair(const uint8_t *text, int64_t n, const uint8_t *pattern, int64_t m, int W, int O, int k,
                   int32_t *edit_count, int64_t *text_consumed, uint32_t *cigar, int64_t cigar_cap,
                   int64_t *cigar_len, int32_t *dopt_log, int32_t *wedit_log, int64_t dopt_cap,
                   int64_t *n_windows) {
    if (check_args(W, O, k) != 0 || n < 0 || m < 0) return -1;
    orc_work w;
    if (work_init(&w, k) != 0) return -1;
    orc_cigar c = {cigar, cigar_cap, 0, 0, 0};
    int64_t tc = 0, nwin = 0;
    int st = align_pair(&w, text, n, pattern, m, W, O, k, &c, &tc, &nwin, dopt_log, wedit_log, dopt_cap);
    work_free(&w);
    /* a CIGAR overflow still aligned the pair: only the run count reports it */
    *edit_count = (st == 0 || st == -2) ? (int32_t)c.edits : -1;
    *text_consumed = (st == 0 || st == -2) ? tc : 0;
    *cigar_len = st == 0 ? c.len : (st == -2 ? -1 : 0);
    if (n_windows) *n_windows = nwin;
    return st;
}

typedef struct {
    const uint8_t *texts;
    const int64_t *text_off;
    const uint8_t *patterns;
    const int64_t *pattern_off;
    int W, O, k;
    int32_t *edit_counts;
    int32_t *text_consumed;
    uint32_t *cigar;
    const int64_t *cigar_off;
    int32_t *cigar_lens;
    int64_t n_pairs;
    int64_t next;
    int err;
    pthread_mutex_t lock;
} orc_batch;

static void *batch_worker(void *arg) {
    orc_batch *b = (orc_batch *)arg;
    orc_work w;
    if (work_init(&w, b->k) != 0) {
        pthread_mutex_lock(&b->lock);
        b->err = -1;
        pthread_mutex_unlock(&b->lock);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&b->lock);
        int64_t p = b->next++;
        pthread_mutex_unlock(&b->lock);
        if (p >= b->n_pairs) break;
        int64_t n = b->text_off[p + 1] - b->text_off[p];
        int64_t m = b->pattern_off[p + 1] - b->pattern_off[p];
        orc_cigar c = {b->cigar + b->cigar_off[p], b->cigar_off[p + 1] - b->cigar_off[p], 0, 0, 0};
        int64_t tc = 0, nwin = 0;
        int st = align_pair(&w, b->texts + b->text_off[p], n, b->patterns + b->pattern_off[p], m, b->W, b->O,
                            b->k, &c, &tc, &nwin, NULL, NULL, 0);
        if (st == -1) {
            pthread_mutex_lock(&b->lock);
            b->err = -1;
            pthread_mutex_unlock(&b->lock);
        }
        b->edit_counts[p] = (st == 0 || st == -2) ? (int32_t)c.edits : -1;
        b->text_consumed[p] = (st == 0 || st == -2) ? (int32_t)tc : 0;
        b->cigar_lens[p] = st == 0 ? (int32_t)c.len : (st == -2 ? -1 : 0);
    }
    work_free(&w);
    return NULL;
}

/*
 * A batch of pairs over `threads` POSIX threads pulling pairs from a shared
 * counter. Sequences are codes 0..3, one per byte; pair p is
 * texts[text_off[p]:text_off[p+1]) and patterns[pattern_off[p]:...).
 * Pair p may write CIGAR runs to cigar[cigar_off[p]:cigar_off[p+1]);
 * cigar_lens[p] is the run count, or -1 on overflow.
 */
int orc_align_batch(const uint8_t *texts, const int64_t *text_off, const uint8_t *patterns,
                    const int64_t *pattern_off, int64_t n_pairs, int W, int O, int k, int threads,
                    int32_t *edit_counts, int32_t *text_consumed, uint32_t *cigar, const int64_t *cigar_off,
                    int32_t *cigar_lens) {
    if (check_args(W, O, k) != 0 || n_pairs < 0) return -1;
    if (threads < 1) threads = 1;
    orc_batch b;
    memset(&b, 0, sizeof b);
    b.texts = texts;
    b.text_off = text_off;
    b.patterns = patterns;
    b.pattern_off = pattern_off;
    b.W = W;
    b.O = O;
    b.k = k;
    b.edit_counts = edit_counts;
    b.text_consumed = text_consumed;
    b.cigar = cigar;
    b.cigar_off = cigar_off;
    b.cigar_lens = cigar_lens;
    b.n_pairs = n_pairs;
    pthread_mutex_init(&b.lock, NULL);
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!tid) return -1;
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&tid[t], NULL, batch_worker, &b) == 0) started++;
        else break;
    if (started == 0) batch_worker(&b);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    free(tid);
    pthread_mutex_destroy(&b.lock);
    return b.err;
}
