// Host check of the scan's per-lane arithmetic (compiled with g++ against
// the stub cuda_runtime.h next to this file).  Random queries, targets,
// matrices and step windows; every 4-shift chunk sum, split into random
// segments, and every lane-local step must equal a naive sum of matrix
// entries, and every profile/target read must stay inside its buffer: the
// buffers end at PROT_NONE guard pages, so a stray read faults.
// Also checked: the full-slide mode's chunks (every shift of a step, the
// overhanging ones included, with windows where ss exceeds ls); the
// flattened scan's per-chunk keys (their maximum over a
// step's chunks gives the step's best shift), the same keys through a flat
// step's packed descriptor, and the owners from the pass start masks.
// Both accumulator forms are checked: 32-bit sums always, 16-bit pair sums
// whenever range * (qlen + 3) <= 65535 (the condition the library uses).
// usage: lane_emu SEED [MIN MAX]   (matrix entries drawn from [MIN, MAX])
#include <sys/mman.h>
#include <unistd.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <random>
#include "hs_device.cuh"
using namespace hs;
// buffer with PROT_NONE guard pages on both sides; data placed flush against the tail guard
template <class T> T *guarded(size_t n, T **base_out) {
    size_t pg = sysconf(_SC_PAGESIZE);
    size_t bytes = n * sizeof(T);
    size_t body = (bytes + pg - 1) / pg * pg;
    char *m = (char *)mmap(nullptr, body + 2 * pg, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    mprotect(m, pg, PROT_NONE);
    mprotect(m + pg + body, pg, PROT_NONE);
    T *p = (T *)(m + pg + body - bytes);      // end of data touches the guard
    *base_out = p;
    return p;
}
// one 4-shift chunk summed over nseg iteration segments into one accumulator;
// returns the number of shifts checked, or -1 - x for a mismatch at shift k0 + x
template <bool P16>
long check_chunk(const uint32_t *prof, int R, int qlen, const uint8_t *t, int Lp, int Sp, int ss, bool qsmall,
                 int k0, int nseg, int nshift, int flush, int bias, const std::vector<int> &V) {
    int niter = qsmall ? ss + 3 : ss;
    Acc<P16> A;
    A.zero();
    for (int sg = 0; sg < nseg; sg++) {
        int it0 = sg * niter / nseg, it1 = (sg + 1) * niter / nseg;
        if (qsmall) rev_segment<P16>(prof, R, t + Lp + k0, qlen + 3 - Sp, ss, it0, it1, sg == 0, sg == nseg - 1, flush, A);
        else fwd_chunk<P16>(prof, R, t + Sp, Lp + k0 + 4, it0, it1, flush, A);
    }
    long n = 0;
    for (int x = 0; x < 4 && k0 + x < nshift; x++, n++)
        if ((int)A.get(x) - bias * ss != V[k0 + x]) return -1 - x;
    return n;
}
// full-slide mode (readings F1-F3): chunk k0 of a step's shifts -(ss-1) ..
// ls-1, its iterations split into 2^lgj segments summed into one
// accumulator; same return convention as check_chunk
template <bool P16>
long check_full_chunk(const uint32_t *prof, int R, int qlen, const Plan &g, int k0, int lgj, int flush, int bias,
                      const std::vector<int> &Vf) {
    Acc<P16> A;
    A.zero();
    for (int gj = 0; gj < (1 << lgj); gj++) full_chunk<P16>(prof, R, qlen, g, k0, gj, lgj, flush, A);
    long n = 0;
    for (int x = 0; x < 4 && k0 + x < g.ls; x++, n++)
        if ((int)A.get(x) - bias * full_overlap(g.ls, g.ss, k0 + x) != Vf[k0 + x + g.ss - 1]) return -1 - x;
    return n;
}
template <bool P16>
bool check_lane_scan(const uint32_t *prof, int R, int qlen, const Plan &g, int bias, int flush, int bestv, int bestk) {
    int32_t vm, ks;
    lane_scan_t<P16>(prof, R, qlen, g, bias, flush, vm, ks);
    return vm == bestv && ks == bestk;
}
int main(int argc, char **argv) {
    std::mt19937_64 rng(argc > 1 ? atoi(argv[1]) : 1);
    int8_t M[576];
    int mlo = argc > 2 ? atoi(argv[2]) : -4, mhi = argc > 3 ? atoi(argv[3]) : 11;
    for (int a = 0; a < 24; a++) for (int b = 0; b <= a; b++) { int v = mlo + (int)(rng() % (mhi - mlo + 1)); M[a*24+b] = M[b*24+a] = (int8_t)v; }
    int lo = 127, hi = -128; for (int i = 0; i < 576; i++) { lo = std::min<int>(lo, M[i]); hi = std::max<int>(hi, M[i]); }
    int bias = -lo, flush = hi == lo ? 255 : std::max(1, 255 / (hi - lo));
    long checks = 0, full_checks = 0;
    for (int trial = 0; trial < 3000; trial++) {
        int qlen = 1 + rng() % 300;
        int tlen = 1 + rng() % 600;
        std::vector<uint8_t> q(qlen);
        for (auto &c : q) c = rng() % 24;
        // database: the target, then 64 pad bytes (as the library allocates)
        uint8_t *tb; uint8_t *t = guarded<uint8_t>(tlen + kCodesPad, &tb);
        for (int i = 0; i < tlen; i++) t[i] = rng() % 24;
        memset(t + tlen, 0, kCodesPad);
        int R = profile_stride(qlen);
        // 16-bit pair sums whenever the library would pick them
        const bool p16 = (long)(hi - lo) * (qlen + 3) <= 65535;
        for (int rev = 0; rev < 2; rev++) {
            uint32_t *pb; uint32_t *prof = guarded<uint32_t>((size_t)profile_words(qlen), &pb);
            for (int a = 0; a < 24; a++) for (int s = 0; s < R; s++) prof[a * R + s] = profile_word_value(q.data(), qlen, rev, M, bias, a, s);
            bool qsmall = rev;   // rev profile <-> query small
            int nl = qsmall ? tlen : qlen, ns = qsmall ? qlen : tlen;
            const uint8_t *L = qsmall ? t : q.data(), *S = qsmall ? q.data() : t;
            // random step windows
            for (int w = 0; w < 20; w++) {
                int Lp = rng() % nl, Sp = rng() % ns;
                int Lrem = nl - Lp, Srem = ns - Sp;
                int ls = 1 + rng() % Lrem;
                int ss = 1 + rng() % std::min(Srem, ls);
                Plan g = {t, Lp, Sp, ls, ss, qsmall ? 1 : 0, 0, 0, 0};
                int nshift = ls - ss + 1;
                // naive
                int bestv = INT32_MIN, bestk = 0;
                std::vector<int> V(nshift);
                for (int k = 0; k < nshift; k++) { int v = 0; for (int j = 0; j < ss; j++) { int a = L[Lp+k+j], b = S[Sp+j]; v += qsmall ? M[b*24+a] : M[a*24+b]; } V[k] = v; if (v > bestv) { bestv = v; bestk = k; } }
                // lane scan (whole step) and per-chunk segments with random splits
                if (nshift <= 64) {
                    if (!check_lane_scan<false>(prof, R, qlen, g, bias, flush, bestv, bestk) ||
                        (p16 && !check_lane_scan<true>(prof, R, qlen, g, bias, flush, bestv, bestk))) {
                        printf("lane_scan mismatch trial %d\n", trial); return 1;
                    }
                }
                if (p16 && nshift <= 65536) {
                    uint32_t key = 0;
                    for (int k0 = 0; k0 < nshift; k0 += 4) key = std::max(key, unit_key(prof, R, qlen, g, k0, nshift, flush));
                    if ((int)(key >> 16) - bias * ss != bestv || (int)(0xFFFFu - (key & 0xFFFFu)) != bestk) {
                        printf("unit_key mismatch trial %d\n", trial); return 1;
                    }
                    // the same through a flat step's descriptor
                    const uint4 dsc = flat_desc(g, qlen);
                    for (int k0 = 0; k0 < nshift; k0 += 4)
                        if (desc_key(prof, prof, R, dsc, k0, flush) != unit_key(prof, R, qlen, g, k0, nshift, flush)) {
                            printf("desc_key mismatch trial %d\n", trial); return 1;
                        }
                }
                // full-slide windows: ss up to Srem, so it may exceed ls (F2)
                {
                    const int fss = 1 + rng() % Srem;
                    Plan f = {t, Lp, Sp, ls, fss, qsmall ? 1 : 0, 0, 0, 0};
                    std::vector<int> Vf(ls + fss - 1);
                    for (int k = -(fss - 1); k < ls; k++) {
                        int v = 0;
                        for (int j = std::max(0, -k); j < std::min(fss, ls - k); j++) {
                            int a = L[Lp + k + j], b = S[Sp + j];
                            v += qsmall ? M[b * 24 + a] : M[a * 24 + b];
                        }
                        Vf[k + fss - 1] = v;
                    }
                    for (int k0 = -(fss - 1); k0 < ls; k0 += 4) {
                        const int lgj = (int)(rng() % 4);
                        long c = check_full_chunk<false>(prof, R, qlen, f, k0, lgj, flush, bias, Vf);
                        if (c >= 0 && p16) c = check_full_chunk<true>(prof, R, qlen, f, k0, lgj, flush, bias, Vf);
                        if (c < 0) { printf("full chunk mismatch trial %d k %ld\n", trial, k0 - 1 - c); return 1; }
                        checks += c;
                        full_checks += c;
                    }
                }
                int niter = qsmall ? ss + 3 : ss;
                for (int k0 = 0; k0 < nshift; k0 += 4) {
                    int nseg = 1 + rng() % 4;
                    int minseg = qsmall ? 6 : 4;
                    if (niter < nseg * minseg) nseg = 1;
                    long c = check_chunk<false>(prof, R, qlen, t, Lp, Sp, ss, qsmall, k0, nseg, nshift, flush, bias, V);
                    if (c >= 0 && p16) c = check_chunk<true>(prof, R, qlen, t, Lp, Sp, ss, qsmall, k0, nseg, nshift, flush, bias, V);
                    if (c < 0) { printf("chunk mismatch trial %d k %ld\n", trial, k0 - 1 - c); return 1; }
                    checks += c;
                }
            }
        }
    }
    // owner search of the flattened list: random unit counts (many zero)
    for (int trial = 0; trial < 20000; trial++) {
        // ranks: flat steps first (1..63 units each), then steps with none
        int32_t firsts[32], units[32];
        int u0 = 0, owner[32 * 64];
        const int nflat = (int)(rng() % 33);
        for (int j = 0; j < 32; j++) {
            const int n = j < nflat ? 1 + (int)(rng() % 63) : 0;
            firsts[j] = u0;
            units[j] = n;
            for (int x = 0; x < n; x++) owner[u0 + x] = j;
            u0 += n;
        }
        int carry = -1, carry_u0 = 0;
        for (int base = 0; base < u0; base += 32) {
            unsigned starts = 0;
            for (int r = 0; r < 32; r++) starts |= start_bit(firsts[r], units[r], base);
            int last = -1, last_u0 = 0;
            for (int lane = 0; lane < 32; lane++) {
                const int o = pass_owner(carry, starts, lane);
                const int f = pass_first_unit(carry_u0, starts, base, lane);
                if (base + lane < u0 && (o != owner[base + lane] || f != firsts[o])) {
                    printf("owner mismatch trial %d unit %d\n", trial, base + lane); return 1;
                }
                // the fold's one-owner test: no step begins after lane 0
                if ((starts >> 1) == 0u && base + lane < u0 && owner[base + lane] != owner[base]) {
                    printf("one-owner test wrong trial %d unit %d\n", trial, base + lane); return 1;
                }
                last = o;
                last_u0 = f;
            }
            carry = last;
            carry_u0 = last_u0;
        }
    }
    printf("emu ok: %ld shift sums checked (%ld of them full-slide)\n", checks, full_checks);
    return 0;
}
