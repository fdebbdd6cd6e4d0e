/*
 * hs_oracle.c -- plain, slow CPU oracle for the heuristic pair-wise
 * alignment of Nag & Karforma, "A Space-Efficient Approach towards Distantly
 * Homologous Protein Similarity Searches" (arXiv 1508.06561), in its
 * database-search form (Sec. III.B.3), plus the exact dynamic programmes
 * used to pin it.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  The GPU library shares no
 * code, table or header with it: this file has its own alphabet table, its
 * own matrix parser and its own Philox generator.
 *
 * The heuristic's own choices (how long each piece is, which shift wins,
 * what a step lays out) are pinned by an independent step trace in the
 * tests: draws sliced from numpy's Philox, the piece sizes in Python
 * integers, the best shift by a numpy sliding-window argmax; it predicts
 * every alignment column and the cell count, and copies of this file with
 * plausible mistakes planted fail it.  The rest is pinned by what the
 * mathematics fixes -- Philox known answers, SCORE closed forms, the exact
 * DP optimum as an upper bound, rescoring of the emitted rows, special cases
 * with closed forms.
 *
 * Structure follows Fig. 1 of the paper:
 *   or_align_sequences   -- AlignSequences: best of `rounds` randomised runs
 *   align_round          -- Align: chop both sequences into sub-sequences
 *   best_subsequence     -- getBestSubsequenceAlignment: slide small vs large
 *   virtual_score        -- getVirtualAlignmentScore: score of one shift
 *   or_score_rows        -- SCORE: score of a finished gapped alignment
 *
 * Readings taken where the paper is silent (the numbering matches the
 * design notes; every one is also restated next to the code that uses it):
 *   A1  virtual score = ungapped sum of M over the overlap at shift k.
 *   A2  SCORE: residue/residue column scores M; gap characters before the
 *       first or after the last residue/residue column cost PGP each; every
 *       maximal gap run of one row inside that core costs GOP+(n-1)*GEP.
 *   A3  affine convention GOP + (n-1)*GEP.
 *   A4  lf = max(MinFactor, LFactor*U1), sf = max(MinFactor, SFactor*U2).
 *   A6  Q16 fixed point, floors; ls >= 1; 1 <= ss <= min(Srem, ls).
 *   A8  sub-sequences are prefixes of what is left of each sequence.
 *   A9  a step consumes the first k*+ss letters of large.
 *   A10 ties: lowest shift, first round.
 *   A12 random(): Philox4x64-10 draws, 16 bits each (see draw16 below).
 *   A13 large = target when |T| >= |Q|.
 * Full-slide mode (the pair-wise form of Fig. 1, without Sec. III.B.3 b):
 *   F1  shifts k = -(ss-1) .. ls-1 (overlap >= 1), V(k) over the overlap only,
 *       lowest k on ties;
 *   F2  1 <= ss <= Srem (no ls bound: a piece may overhang the window);
 *   F3  a step lays out: the letters of whichever piece starts first against
 *       gaps in the other row, the overlap, then small's letters past the
 *       window's end against gaps in large's row; large gives up its letters
 *       through the end of the overlap, small its ss letters;
 *   F4  SCORE is taken over the finished rows (so gap runs may merge across
 *       steps, and leading/trailing runs in either row are periphery).
 * Scores use the matrix as M[query letter][target letter]; the matrix must
 * be symmetric for the library, but the oracle keeps the orientation explicit.
 *
 * Parity pins live in tests/: Philox against numpy's Philox and the
 * published known-answer vectors; SCORE against closed forms; the
 * periphery DP against exhaustive enumeration and against Smith-Waterman
 * (PGP = 0); the heuristic against the DP optimum, the rescore of its own
 * rows, the self-alignment closed form, and step by step (piece sizes,
 * shifts, the rows of both modes, cell counts) against the independent
 * trace of tests/test_oracle_steps.py, a hand-worked first step included.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_NSYM 24
#define OR_GAP 0xFFu
#define OR_MODE_DB 0
#define OR_MODE_FULL 1

/* ------------------------------------------------------------------ */
/* Alphabet: the 24 symbols of BLOSUM62 (Sec. III.A) in NCBI order.      */
/* ------------------------------------------------------------------ */
static const char OR_LETTERS[OR_NSYM + 1] = "ARNDCQEGHILKMFPSTWYVBZX*";
#define OR_CODE_X 22

int or_letter_code(int c)
{
    if (c >= 'a' && c <= 'z') c -= 'a' - 'A';
    for (int i = 0; i < OR_NSYM; i++)
        if (OR_LETTERS[i] == c) return i;
    return OR_CODE_X;                  /* unknown letters read as X */
}

int or_encode(const char *ascii, int64_t n, uint8_t *codes)
{
    for (int64_t i = 0; i < n; i++) codes[i] = (uint8_t)or_letter_code((unsigned char)ascii[i]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Matrix parser: NCBI text layout.  A header line lists the column      */
/* letters; each following line is "<letter> v v v ...".  '#' lines are */
/* comments.  Returns 0, or -1 on a malformed or incomplete table.       */
/* ------------------------------------------------------------------ */
int or_parse_matrix(const char *text, int8_t *out)
{
    int cols[64];
    int ncols = 0, have_header = 0, seen[OR_NSYM] = {0};
    const char *p = text;
    while (*p) {
        const char *eol = p;
        while (*eol && *eol != '\n') eol++;
        const char *s = p;
        while (s < eol && (*s == ' ' || *s == '\t' || *s == '\r')) s++;
        if (s < eol && *s != '#') {
            if (!have_header) {
                for (const char *c = s; c < eol; c++) {
                    if (*c == ' ' || *c == '\t' || *c == '\r') continue;
                    if (ncols >= 64) return -1;
                    cols[ncols++] = or_letter_code((unsigned char)*c);
                }
                have_header = 1;
            } else {
                int row = or_letter_code((unsigned char)*s);
                const char *c = s + 1;
                for (int j = 0; j < ncols; j++) {
                    char *end;
                    while (c < eol && (*c == ' ' || *c == '\t')) c++;
                    if (c >= eol) return -1;
                    long v = strtol(c, &end, 10);
                    if (end == c || v < -128 || v > 127) return -1;
                    out[row * OR_NSYM + cols[j]] = (int8_t)v;
                    c = end;
                }
                seen[row] = 1;
            }
        }
        p = *eol ? eol + 1 : eol;
    }
    if (ncols != OR_NSYM) return -1;
    for (int i = 0; i < OR_NSYM; i++)
        if (!seen[i]) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by   */
/* fixed odd constants, swaps and xors the halves with the key; the key  */
/* is bumped by Weyl constants between rounds.                           */
/* ------------------------------------------------------------------ */
void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * random() of Fig. 1 (reading A12).  The pair with database index d, in
 * round r, owns the stream of 16-bit draws  D_0, D_1, D_2, ...  where draw i
 * is 16-bit field (i mod 4), most significant first, of word ((i mod 16)/4)
 * of block  Philox4x64-10(counter = (d, r, i/16, 0), key = (seed, 0)).
 * A draw D stands for the real number D / 65536 in [0, 1).
 * D_0 and D_1 feed lf and sf of the round; D_(2+t) feeds step t.
 */
static uint32_t draw16(uint64_t seed, uint64_t d, uint64_t r, uint64_t i)
{
    uint64_t ctr[4] = {d, r, i / 16, 0}, key[2] = {seed, 0}, blk[4];
    or_philox4x64_10(ctr, key, blk);
    uint64_t w = blk[(i % 16) / 4];
    return (uint32_t)((w >> (48 - 16 * (i % 4))) & 0xFFFFu);
}

uint32_t or_draw16(uint64_t seed, uint64_t d, uint64_t r, uint64_t i) { return draw16(seed, d, r, i); }

/* ------------------------------------------------------------------ */
/* Parameters (Sec. III.B.1; defaults of Sec. IV).                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t pgp, gop, gep, rounds;
    uint32_t lfactor_q16, sfactor_q16, minfactor_q16;   /* 65536 == 1.0 */
    int32_t mode;                                      /* OR_MODE_DB */
} or_params;

/* ------------------------------------------------------------------ */
/* SCORE(rowQ, rowT) of a finished alignment (reading A2/A3).            */
/* Rows hold letter codes, OR_GAP for '-'.  Returns 0 and the score, or  */
/* -1 when a column has gaps in both rows.                               */
/* ------------------------------------------------------------------ */
int or_score_rows(const uint8_t *rq, const uint8_t *rt, int64_t ncols, const int8_t *M,
                  int32_t pgp, int32_t gop, int32_t gep, int64_t *score_out)
{
    int64_t first = -1, last = -1;
    for (int64_t c = 0; c < ncols; c++) {
        if (rq[c] == OR_GAP && rt[c] == OR_GAP) return -1;
        if (rq[c] != OR_GAP && rt[c] != OR_GAP) {
            if (first < 0) first = c;
            last = c;
        }
    }
    int64_t s = 0;
    if (first < 0) {                      /* no residue pair: all periphery */
        *score_out = -(int64_t)pgp * ncols;
        return 0;
    }
    s -= (int64_t)pgp * first;            /* leading periphery gaps */
    s -= (int64_t)pgp * (ncols - 1 - last); /* trailing periphery gaps */
    int64_t c = first;
    while (c <= last) {
        if (rq[c] != OR_GAP && rt[c] != OR_GAP) {
            s += M[rq[c] * OR_NSYM + rt[c]];
            c++;
            continue;
        }
        /* a maximal run of gaps in one row */
        int gap_in_q = (rq[c] == OR_GAP);
        int64_t n = 0;
        while (c <= last && ((gap_in_q && rq[c] == OR_GAP) || (!gap_in_q && rt[c] == OR_GAP))) {
            n++;
            c++;
        }
        s -= (int64_t)gop + (n - 1) * (int64_t)gep;
    }
    *score_out = s;
    return 0;
}

/* ------------------------------------------------------------------ */
/* getVirtualAlignmentScore(large, small, k) (reading A1): the ungapped  */
/* score of small laid against large with small[0] under large[k],       */
/* summed over the columns where both have a letter.  `q_is_large` keeps */
/* the matrix orientation M[query][target].                               */
/* ------------------------------------------------------------------ */
static int64_t virtual_score(const uint8_t *large, int64_t nl, const uint8_t *small, int64_t ns,
                             int64_t k, const int8_t *M, int q_is_large, int64_t *cells)
{
    int64_t s = 0;
    for (int64_t j = 0; j < ns; j++) {
        int64_t i = k + j;
        if (i < 0 || i >= nl) continue;
        int a = large[i], b = small[j];
        s += q_is_large ? M[a * OR_NSYM + b] : M[b * OR_NSYM + a];
        (*cells)++;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* getBestSubsequenceAlignment(large, small) (Fig. 1).  The paper slides  */
/* i over [start, end] with k = i - |small| + 1; database mode            */
/* (Sec. III.B.3 b) sets start = |small|-1 and end = |large|-1, so k runs  */
/* over 0..|large|-|small| and small lies wholly inside large.  The best  */
/* score is kept with a strict '>', so the lowest k wins ties (A10).      */
/* ------------------------------------------------------------------ */
static int64_t best_subsequence(const uint8_t *large, int64_t nl, const uint8_t *small, int64_t ns,
                                int mode, const int8_t *M, int q_is_large, int64_t *best_k,
                                int64_t *cells)
{
    int64_t n = ns + nl - 1;
    int64_t start = 0, end = n - 1;
    if (mode == OR_MODE_DB) { start = ns - 1; end = nl - 1; }
    int64_t best = INT64_MIN;
    *best_k = 0;
    for (int64_t i = start; i <= end; i++) {
        int64_t k = i - ns + 1;
        int64_t score = virtual_score(large, nl, small, ns, k, M, q_is_large, cells);
        if (score > best) { best = score; *best_k = k; }
    }
    return best;
}

/* One full-slide step (F1), for the same check with partial overlaps. */
int64_t or_best_shift_full(const uint8_t *large, int64_t nl, const uint8_t *small, int64_t ns,
                           const int8_t *M, int64_t *best_k)
{
    int64_t cells = 0;
    return best_subsequence(large, nl, small, ns, OR_MODE_FULL, M, 1, best_k, &cells);
}

/* Exported single-step scan, so tests can check it against an
 * independent numpy sliding-window computation. */
int64_t or_best_shift(const uint8_t *large, int64_t nl, const uint8_t *small, int64_t ns,
                      const int8_t *M, int64_t *best_k)
{
    int64_t cells = 0;
    return best_subsequence(large, nl, small, ns, OR_MODE_DB, M, 1, best_k, &cells);
}

/* ------------------------------------------------------------------ */
/* Align(large, small, LF, SF) (Fig. 1, Sec. III.B.2), database mode.     */
/* Builds the two rows, then scores them with SCORE, as the paper does.   */
/* Rows are written as (large row, small row) into rl/rs.                 */
/* ------------------------------------------------------------------ */
static int64_t align_round(const uint8_t *large, int64_t nl, const uint8_t *small, int64_t ns,
                           uint32_t lf, uint32_t sf, const or_params *p, const int8_t *M,
                           int q_is_large, uint64_t seed, uint64_t d, uint64_t r,
                           uint8_t *rl, uint8_t *rs, int64_t *ncols_out, int64_t *cells)
{
    int64_t Lp = 0, Sp = 0, t = 0, nc = 0;
    while (Lp < nl && Sp < ns) {              /* until either sequence is used up (Fig. 1) */
        int64_t Lrem = nl - Lp, Srem = ns - Sp;
        /* ls = length(large) * LF, ss = length(small) * SF * random()  (A6) */
        int64_t ls = (int64_t)(((uint64_t)Lrem * lf) >> 16);
        if (ls < 1) ls = 1;
        uint64_t u = draw16(seed, d, r, 2 + (uint64_t)t);
        int64_t ss = (int64_t)(((uint64_t)Srem * sf * u) >> 32);
        int64_t cap = p->mode == OR_MODE_DB ? (Srem < ls ? Srem : ls) : Srem;   /* A6/A7; F2 */
        if (ss > cap) ss = cap;
        if (ss < 1) ss = 1;
        int64_t kstar;
        best_subsequence(large + Lp, ls, small + Sp, ss, p->mode, M, q_is_large, &kstar, cells);
        if (p->mode != OR_MODE_DB) {
            /* F3: the step's columns for any shift, overhangs included */
            const int64_t j0 = kstar < 0 ? -kstar : 0;                /* first overlapping small letter */
            const int64_t j1 = (ls - kstar < ss) ? ls - kstar : ss;   /* one past the last */
            for (int64_t j = 0; j < j0; j++) { rl[nc] = OR_GAP; rs[nc] = small[Sp + j]; nc++; }
            for (int64_t i = 0; i < kstar; i++) { rl[nc] = large[Lp + i]; rs[nc] = OR_GAP; nc++; }
            for (int64_t j = j0; j < j1; j++) { rl[nc] = large[Lp + kstar + j]; rs[nc] = small[Sp + j]; nc++; }
            for (int64_t j = j1; j < ss; j++) { rl[nc] = OR_GAP; rs[nc] = small[Sp + j]; nc++; }
            Lp += kstar + j1;
            Sp += ss;
            t++;
            continue;
        }
        /* A9: large gives up its first k*+ss letters; the first k* stand
         * against gaps in small's row, the next ss against small's piece. */
        for (int64_t i = 0; i < kstar; i++) { rl[nc] = large[Lp + i]; rs[nc] = OR_GAP; nc++; }
        for (int64_t j = 0; j < ss; j++) { rl[nc] = large[Lp + kstar + j]; rs[nc] = small[Sp + j]; nc++; }
        Lp += kstar + ss;
        Sp += ss;                             /* small gives up its first ss letters (A9) */
        t++;
    }
    /* the leftover letters of either sequence go against gaps (Fig. 1) */
    while (Lp < nl) { rl[nc] = large[Lp++]; rs[nc] = OR_GAP; nc++; }
    while (Sp < ns) { rl[nc] = OR_GAP; rs[nc] = small[Sp++]; nc++; }
    *ncols_out = nc;
    int64_t score;
    if (q_is_large) or_score_rows(rl, rs, nc, M, p->pgp, p->gop, p->gep, &score);
    else            or_score_rows(rs, rl, nc, M, p->pgp, p->gop, p->gep, &score);
    return score;
}

/*
 * AlignSequences (Fig. 1) for one (query, target) pair.
 *   rq/rt (optional, capacity |Q|+|T|) receive the winning alignment as
 *   (query row, target row); *ncols its length; *round_out the winning round.
 *   *cells counts virtual-score cells (one per letter pair summed) over all
 *   rounds.  Returns the best score (strict '>' keeps the first best round).
 */
int64_t or_align_pair(const uint8_t *q, int64_t qlen, const uint8_t *t, int64_t tlen,
                      const int8_t *M, const or_params *p, uint64_t seed, uint64_t dbidx,
                      uint8_t *rq, uint8_t *rt, int64_t *ncols, int32_t *round_out,
                      int64_t *cells)
{
    int q_is_large = !(tlen >= qlen);          /* A13: the target is large on ties */
    const uint8_t *large = q_is_large ? q : t, *small = q_is_large ? t : q;
    int64_t nl = q_is_large ? qlen : tlen, ns = q_is_large ? tlen : qlen;
    int64_t cap = qlen + tlen + 1;
    uint8_t *rl = (uint8_t *)malloc((size_t)cap), *rs = (uint8_t *)malloc((size_t)cap);
    uint8_t *bl = (uint8_t *)malloc((size_t)cap), *bs = (uint8_t *)malloc((size_t)cap);
    int64_t best = INT64_MIN, bestn = 0, c = 0;
    int32_t bestr = -1;
    for (int32_t r = 0; r < p->rounds; r++) {
        /* lf = MAX(minFactor, random()), sf likewise, scaled by LFactor and
         * SFactor (reading A4). */
        uint64_t u1 = draw16(seed, dbidx, (uint64_t)r, 0), u2 = draw16(seed, dbidx, (uint64_t)r, 1);
        uint32_t lf = (uint32_t)(((uint64_t)p->lfactor_q16 * u1) >> 16);
        uint32_t sf = (uint32_t)(((uint64_t)p->sfactor_q16 * u2) >> 16);
        if (lf < p->minfactor_q16) lf = p->minfactor_q16;
        if (sf < p->minfactor_q16) sf = p->minfactor_q16;
        int64_t n;
        int64_t score = align_round(large, nl, small, ns, lf, sf, p, M, q_is_large, seed, dbidx,
                                    (uint64_t)r, rl, rs, &n, &c);
        if (score > best) {
            best = score; bestr = r; bestn = n;
            memcpy(bl, rl, (size_t)n); memcpy(bs, rs, (size_t)n);
        }
    }
    if (rq && rt) {
        memcpy(rq, q_is_large ? bl : bs, (size_t)bestn);
        memcpy(rt, q_is_large ? bs : bl, (size_t)bestn);
    }
    if (ncols) *ncols = bestn;
    if (round_out) *round_out = bestr;
    if (cells) *cells = c;
    free(rl); free(rs); free(bl); free(bs);
    return best;
}

/* ------------------------------------------------------------------ */
/* Database search (Sec. III.B.3): the query against every target.       */
/* Targets are  codes[offsets[i] .. offsets[i+1])  with database index    */
/* idx[i] (idx == NULL: i itself).  Threads share a plain atomic counter. */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint8_t *codes; const int64_t *offsets; const int64_t *idx; int64_t n;
    const uint8_t *q; int64_t qlen; const int8_t *M; const or_params *p; uint64_t seed;
    int64_t *scores; int64_t *cells; int64_t next;
} or_job;

static void *search_worker(void *arg)
{
    or_job *J = (or_job *)arg;
    for (;;) {
        int64_t i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (i >= J->n) break;
        int64_t d = J->idx ? J->idx[i] : i;
        int64_t c = 0;
        J->scores[i] = or_align_pair(J->q, J->qlen, J->codes + J->offsets[d],
                                     J->offsets[d + 1] - J->offsets[d], J->M, J->p, J->seed,
                                     (uint64_t)d, NULL, NULL, NULL, NULL, &c);
        if (J->cells) J->cells[i] = c;
    }
    return NULL;
}

/* scores_out[i] (and cells_out[i], if given) for target idx[i]; offsets
 * index the whole database.  Returns the number of threads used. */
int32_t or_search_scores(const uint8_t *codes, const int64_t *offsets, const int64_t *idx, int64_t n,
                         const uint8_t *q, int64_t qlen, const int8_t *M, const or_params *p,
                         uint64_t seed, int32_t nthreads, int64_t *scores_out, int64_t *cells_out)
{
    or_job J = {codes, offsets, idx, n, q, qlen, M, p, seed, scores_out, cells_out, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int32_t started = 0;
    for (int32_t i = 1; i < nthreads; i++)
        if (pthread_create(&th[started], NULL, search_worker, &J) == 0) started++;
    search_worker(&J);
    for (int32_t i = 0; i < started; i++) pthread_join(th[i], NULL);
    return started + 1;
}

/* Ranking (Sec. IV's threshold reporting, read as top-k): order by score
 * descending, then database index ascending (A10).  Plain selection of
 * the k best by repeated scans -- O(n k), fine for an oracle. */
int32_t or_topk(const int64_t *scores, int64_t n, int32_t k, int64_t *idx_out)
{
    int32_t m = 0;
    if (k > n) k = (int32_t)n;
    unsigned char *taken = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (; m < k; m++) {
        int64_t b = -1;
        for (int64_t i = 0; i < n; i++) {
            if (taken[i]) continue;
            if (b < 0 || scores[i] > scores[b]) b = i;   /* first index wins ties */
        }
        taken[b] = 1;
        idx_out[m] = b;
    }
    free(taken);
    return m;
}

/* ------------------------------------------------------------------ */
/* Exact optimum under the same scoring (A2/A3): a Gotoh-style DP over    */
/* alignments of x and y whose leading and trailing gap columns cost PGP  */
/* and whose interior gap runs cost GOP+(n-1)GEP.                         */
/*   H[i][j]: best prefix alignment ending in the column (x[i-1], y[j-1]) */
/*   E[i][j]: ... ending in (x[i-1], -) after at least one letter pair    */
/*   F[i][j]: ... ending in (-, y[j-1]) after at least one letter pair    */
/* The first letter pair may be preceded by any i-1 + j-1 periphery gaps. */
/* M is indexed M[x letter][y letter].                                    */
/* ------------------------------------------------------------------ */
#define NEG_INF (INT64_MIN / 4)
static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t max3(int64_t a, int64_t b, int64_t c) { return max2(a, max2(b, c)); }

int64_t or_periphery_opt(const uint8_t *x, int64_t nx, const uint8_t *y, int64_t ny,
                         const int8_t *M, int32_t pgp, int32_t gop, int32_t gep)
{
    int64_t W = ny + 1;
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * (size_t)((nx + 1) * W));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)((nx + 1) * W));
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)((nx + 1) * W));
    for (int64_t i = 0; i <= nx; i++)
        for (int64_t j = 0; j <= ny; j++) {
            int64_t o = i * W + j;
            H[o] = E[o] = F[o] = NEG_INF;
            if (i > 0 && j > 0) {
                int64_t lead = -(int64_t)pgp * ((i - 1) + (j - 1));
                int64_t prev = max2(lead, max3(H[o - W - 1], E[o - W - 1], F[o - W - 1]));
                H[o] = prev + M[x[i - 1] * OR_NSYM + y[j - 1]];
            }
            if (i > 0)
                E[o] = max3(H[o - W] - gop, E[o - W] - gep, F[o - W] - gop);
            if (j > 0)
                F[o] = max3(H[o - 1] - gop, F[o - 1] - gep, E[o - 1] - gop);
        }
    int64_t best = -(int64_t)pgp * (nx + ny);        /* no letter pair at all */
    for (int64_t i = 1; i <= nx; i++)
        for (int64_t j = 1; j <= ny; j++)
            best = max2(best, H[i * W + j] - (int64_t)pgp * ((nx - i) + (ny - j)));
    free(H); free(E); free(F);
    return best;
}

/* Textbook Smith-Waterman with affine gaps (Gotoh 1982 recurrences):
 * local optimum, empty alignment scoring 0. */
int64_t or_smith_waterman(const uint8_t *x, int64_t nx, const uint8_t *y, int64_t ny,
                          const int8_t *M, int32_t gop, int32_t gep)
{
    int64_t W = ny + 1, best = 0;
    int64_t *H = (int64_t *)calloc((size_t)((nx + 1) * W), sizeof(int64_t));
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)((nx + 1) * W));
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)((nx + 1) * W));
    for (int64_t o = 0; o < (nx + 1) * W; o++) E[o] = F[o] = NEG_INF;
    for (int64_t i = 1; i <= nx; i++)
        for (int64_t j = 1; j <= ny; j++) {
            int64_t o = i * W + j;
            E[o] = max2(H[o - W] - gop, E[o - W] - gep);
            F[o] = max2(H[o - 1] - gop, F[o - 1] - gep);
            H[o] = max2(0, max3(H[o - W - 1] + M[x[i - 1] * OR_NSYM + y[j - 1]], E[o], F[o]));
            best = max2(best, H[o]);
        }
    free(H); free(E); free(F);
    return best;
}
