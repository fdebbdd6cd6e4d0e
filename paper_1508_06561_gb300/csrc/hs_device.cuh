// hs_device.cuh -- device building blocks of the heuristic alignment
// (Fig. 1 of Nag & Karforma, arXiv 1508.06561, in database mode, Sec. III.B.3).
//
// One warp runs one (query, target) pair.  The pair's state -- positions in
// both sequences, step, running score, the round's size factors, one cached
// random block -- is a handful of warp-uniform registers (the O(1) auxiliary
// space of Sec. III.B.4).  Inside a step the 32 lanes split the shifts of
// getBestSubsequenceAlignment: each lane owns 4 adjacent shifts packed into
// the 4 byte lanes of one 32-bit register, so one 32-bit load of the query
// profile and one integer add score 4 cells.
#pragma once
#include <climits>
#include <cstdint>

#include "hs_internal.h"

namespace hs {

// ---------------------------------------------------------------------------
// random(): Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The pair with
// database index d in round r owns 16-bit draws D_0, D_1, ...; draw i is the
// 16-bit field i%4 (most significant first) of word (i%16)/4 of the block for
// counter (d, r, i/16, 0) under key (seed, 0).  D_0 and D_1 size the round
// (lf, sf), D_(2+t) sizes step t; D / 65536 is the uniform number in [0, 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4])
{
    constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ull, kMul1 = 0xCA5A826395121157ull;
    constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull, kWeyl1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round) { k0 += kWeyl0; k1 += kWeyl1; }
        const uint64_t hi0 = __umul64hi(kMul0, c0), lo0 = kMul0 * c0;
        const uint64_t hi1 = __umul64hi(kMul1, c2), lo1 = kMul1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

struct DrawStream {
    uint64_t seed, d, r;
    int64_t blk;
    uint64_t w0, w1, w2, w3;
    __device__ __forceinline__ void init(uint64_t s, uint64_t dd, uint64_t rr)
    {
        seed = s; d = dd; r = rr; blk = -1;
    }
    __device__ __forceinline__ uint32_t get(uint64_t i)
    {
        const int64_t b = (int64_t)(i >> 4);
        if (b != blk) {
            uint64_t o[4];
            philox4x64_10(d, r, (uint64_t)b, 0, seed, 0, o);
            w0 = o[0]; w1 = o[1]; w2 = o[2]; w3 = o[3];
            blk = b;
        }
        const unsigned wi = (unsigned)(i >> 2) & 3u;
        const uint64_t w = wi == 0 ? w0 : wi == 1 ? w1 : wi == 2 ? w2 : w3;
        return (uint32_t)(w >> (48 - 16 * (unsigned)(i & 3))) & 0xFFFFu;
    }
};

// ---------------------------------------------------------------------------
// Query profile.  For role `rev` (the query is the small sequence) the
// profile holds, for every target letter a, the biased scores M[Q[.]][a] with
// the query reversed; for role `fwd` (the query is the large sequence) in
// query order.  Stored column s = c + 4 (4 zero columns of padding in front).
// Four copies r = 0..3, copy r shifted by r bytes, so any 4 consecutive
// columns are one aligned 32-bit word: columns [s, s+4) of letter a are word
//   prof[((s & 3) * 24 + a) * S + (s >> 2)].
// S (words per row) is odd, so the 24 rows of one column fall in 24 distinct
// shared-memory banks: lanes reading different letters never conflict.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t profile_word_value(const uint8_t *q, int qlen, bool rev,
                                                       const int8_t *m, int bias, int r, int a, int w)
{
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int c = 4 * w + r + b - 4;
        uint32_t v = 0;
        if (c >= 0 && c < qlen) {
            const int qc = q[rev ? qlen - 1 - c : c];
            v = (uint32_t)(m[qc * kNSym + a] + bias) & 0xFFu;
        }
        word |= v << (8 * b);
    }
    return word;
}

// ---------------------------------------------------------------------------
// One getBestSubsequenceAlignment call in database mode (Sec. III.B.3 b):
// shifts k = 0 .. ls-ss; V(k) = sum over the ss letters of the small piece of
// M against the large piece shifted by k (the virtual score, no gaps).
// Returns, uniform over the warp, the best V and the lowest k attaining it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void spread_bytes(uint32_t acc, uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t &a3)
{
    a0 += acc & 0xFFu;
    a1 += (acc >> 8) & 0xFFu;
    a2 += (acc >> 16) & 0xFFu;
    a3 += acc >> 24;
}

__device__ __forceinline__ void lane_best1(uint32_t acc, int k, int nshift, int32_t off, int32_t &bv, int32_t &bk)
{
    const int32_t v = (int32_t)acc - off;
    if (k < nshift && v > bv) { bv = v; bk = k; }
}

// shifts ascend within a lane, so a strict '>' keeps the lowest k
__device__ __forceinline__ void lane_best(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, int k0,
                                          int nshift, int32_t off, int32_t &bv, int32_t &bk)
{
    lane_best1(a0, k0, nshift, off, bv, bk);
    lane_best1(a1, k0 + 1, nshift, off, bv, bk);
    lane_best1(a2, k0 + 2, nshift, off, bv, bk);
    lane_best1(a3, k0 + 3, nshift, off, bv, bk);
}

__device__ __forceinline__ void warp_argmax(int32_t bv, int32_t bk, int32_t &vmax, int32_t &kstar)
{
    vmax = __reduce_max_sync(0xFFFFFFFFu, bv);
    kstar = __reduce_min_sync(0xFFFFFFFFu, bv == vmax ? bk : INT_MAX);
}

// Query is the large sequence: large piece = Q[Lp, Lp+ls), small piece =
// tsmall[0, ss) (target letters).  Cells are grouped by small letter j: the
// row is the target letter tsmall[j], shared by all lanes, and lane's 4
// shifts read 4 consecutive query columns Lp+k0+j .. +3.
__device__ __forceinline__ void scan_fwd(const uint32_t *prof, int S, const uint8_t *tsmall, int Lp,
                                         int ls, int ss, int bias, int flush, int lane,
                                         int32_t &vmax, int32_t &kstar)
{
    const int nshift = ls - ss + 1;
    int32_t bv = INT_MIN, bk = INT_MAX;
    for (int base = 0; base < nshift; base += 128) {
        const int k0 = base + 4 * lane;
        const bool active = k0 < nshift;
        const int s0 = active ? Lp + k0 + 4 : 4;
        uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int j0 = 0; j0 < ss; j0 += flush) {
            const int jend = min(ss, j0 + flush);
            uint32_t acc = 0;
            for (int j = j0; j < jend; j++) {
                const int a = tsmall[j];
                const int s = s0 + j;
                acc += prof[((s & 3) * kNSym + a) * S + (s >> 2)];
            }
            spread_bytes(acc, a0, a1, a2, a3);
        }
        if (active) lane_best(a0, a1, a2, a3, k0, nshift, bias * ss, bv, bk);
    }
    warp_argmax(bv, bk, vmax, kstar);
}

// Query is the small sequence: large piece = tlarge[0, ls) (target letters),
// small piece = Q[Sp, Sp+ss).  Cells are grouped by large position p relative
// to the lane's first shift: the row is the target letter tlarge[k0+p] and
// the 4 shifts k0+w read reversed-query columns qlen-1-(Sp+p-w), i.e. 4
// consecutive stored columns.  Byte w holds a real cell only while
// 0 <= p-w < ss, so the first and last 3 positions are masked.
__device__ __forceinline__ void scan_rev(const uint32_t *prof, int S, const uint8_t *tlarge, int qlen,
                                         int Sp, int ls, int ss, int bias, int flush, int lane,
                                         int32_t &vmax, int32_t &kstar)
{
    const int nshift = ls - ss + 1;
    const int sbase = qlen + 3 - Sp;        // stored column of (p = 0, w = 0)
    int32_t bv = INT_MIN, bk = INT_MAX;
    for (int base = 0; base < nshift; base += 128) {
        const int k0 = base + 4 * lane;
        const bool active = k0 < nshift;
        const uint8_t *tk = tlarge + (active ? k0 : 0);
        uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0, acc = 0;
        int since = 0;
        for (int p = 0; p <= ss + 2; p++) {
            const int a = tk[p];
            const int s = sbase - p;
            uint32_t word = prof[((s & 3) * kNSym + a) * S + (s >> 2)];
            if (p < 3 || p >= ss) {
                const uint32_t lo = p >= 3 ? 0xFFFFFFFFu : (0xFFFFFFFFu >> (8 * (3 - p)));
                const int h = p - ss + 1;
                const uint32_t hi = h <= 0 ? 0xFFFFFFFFu : (h >= 4 ? 0u : (0xFFFFFFFFu << (8 * h)));
                word &= lo & hi;
            }
            acc += word;
            if (++since == flush) {
                spread_bytes(acc, a0, a1, a2, a3);
                acc = 0;
                since = 0;
            }
        }
        spread_bytes(acc, a0, a1, a2, a3);
        if (active) lane_best(a0, a1, a2, a3, k0, nshift, bias * ss, bv, bk);
    }
    warp_argmax(bv, bk, vmax, kstar);
}

// ---------------------------------------------------------------------------
// Run-length writer for the alignment ops (lane 0 only).
// ---------------------------------------------------------------------------
struct OpWriter {
    uint32_t *out;
    int64_t cap, n, cur_len;
    uint32_t cur_op;
    __device__ __forceinline__ void init(uint32_t *o, int64_t c) { out = o; cap = c; n = 0; cur_len = 0; cur_op = 0; }
    __device__ __forceinline__ void flush()
    {
        if (cur_len > 0) {
            if (n < cap) out[n] = ((uint32_t)cur_len << 2) | cur_op;
            n++;
            cur_len = 0;
        }
    }
    __device__ __forceinline__ void push(uint32_t op, int64_t len)
    {
        if (len <= 0) return;
        if (cur_len > 0 && op == cur_op) { cur_len += len; return; }
        flush();
        cur_op = op;
        cur_len = len;
    }
};

struct Span { int32_t qb, qe, tb, te; };

// ---------------------------------------------------------------------------
// Align (Fig. 1) for one round, database mode, with the score kept
// incrementally instead of by SCORE over finished rows: every step ends in
// ss letter pairs, so its k* gap letters (in the small sequence's row) form
// one run -- periphery (PGP each) on the first step, GOP+(k*-1)GEP after --
// and the letters left when the loop ends are trailing periphery.
// Cells are counted as (ls-ss+1)*ss per step.
// ---------------------------------------------------------------------------
struct PairCtx {
    const uint32_t *prof;     // profile of this pair's role
    int S;
    const uint8_t *t;         // target letters
    int32_t tlen, qlen;
    bool qsmall;              // |T| >= |Q|: the query is the small sequence
};

template <bool EMIT>
__device__ __forceinline__ int32_t align_round(const PairCtx &c, const KParams &kp, uint64_t d, int r,
                                               int lane, int64_t &cells, OpWriter *ow, Span *span)
{
    const int32_t nl = c.qsmall ? c.tlen : c.qlen, ns = c.qsmall ? c.qlen : c.tlen;
    DrawStream ds;
    ds.init(kp.seed, d, (uint64_t)r);
    // lf = MAX(minFactor, LFactor*random()), sf likewise (Fig. 1, Sec. III.B.1)
    uint32_t lf = (uint32_t)(((uint64_t)kp.lf_q16 * ds.get(0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)kp.sf_q16 * ds.get(1)) >> 16);
    lf = max(lf, kp.minf_q16);
    sf = max(sf, kp.minf_q16);
    int32_t Lp = 0, Sp = 0, score = 0;
    int64_t t = 0;
    const uint32_t gap_op = c.qsmall ? HS_OP_D : HS_OP_I;    // letters of large against gaps
    const uint32_t tail_small_op = c.qsmall ? HS_OP_I : HS_OP_D;
    while (Lp < nl && Sp < ns) {
        const int32_t Lrem = nl - Lp, Srem = ns - Sp;
        int32_t ls = (int32_t)(((uint64_t)Lrem * lf) >> 16);
        ls = max(ls, 1);
        const uint64_t u = ds.get(2 + (uint64_t)t);
        int64_t ssw = (int64_t)(((uint64_t)Srem * sf * u) >> 32);
        const int32_t ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)min(Srem, ls)));
        int32_t vmax, kstar;
        if (c.qsmall)
            scan_rev(c.prof, c.S, c.t + Lp, c.qlen, Sp, ls, ss, kp.bias, kp.flush, lane, vmax, kstar);
        else
            scan_fwd(c.prof, c.S, c.t + Sp, Lp, ls, ss, kp.bias, kp.flush, lane, vmax, kstar);
        cells += (int64_t)(ls - ss + 1) * ss;
        int32_t gap = 0;
        if (kstar > 0) gap = (t == 0) ? kp.pgp * kstar : kp.gop + (kstar - 1) * kp.gep;
        score += vmax - gap;
        if (EMIT && lane == 0) {
            ow->push(gap_op, kstar);
            ow->push(HS_OP_M, ss);
            const int32_t qb = c.qsmall ? Sp : Lp + kstar, tb = c.qsmall ? Lp + kstar : Sp;
            if (span->qb < 0) { span->qb = qb; span->tb = tb; }
            span->qe = qb + ss;
            span->te = tb + ss;
        }
        Lp += kstar + ss;
        Sp += ss;
        t++;
    }
    score -= kp.pgp * ((nl - Lp) + (ns - Sp));
    if (EMIT && lane == 0) {
        ow->push(gap_op, nl - Lp);
        ow->push(tail_small_op, ns - Sp);
        ow->flush();
    }
    return score;
}

// AlignSequences (Fig. 1): best of `rounds` (strict '>', first best wins).
__device__ __forceinline__ int32_t align_pair(const PairCtx &c, const KParams &kp, uint64_t d, int lane,
                                              int64_t &cells, int *best_round)
{
    int32_t best = INT_MIN;
    int br = 0;
    for (int r = 0; r < kp.rounds; r++) {
        const int32_t s = align_round<false>(c, kp, d, r, lane, cells, nullptr, nullptr);
        if (s > best) { best = s; br = r; }
    }
    if (best_round) *best_round = br;
    return best;
}

}  // namespace hs
