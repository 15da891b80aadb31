/*
 * CPU oracle: the sqrt(c)-walk Monte Carlo single-source SimRank estimator,
 * written step by step in plain C (C11 + OpenMP over targets).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by the
 * CPU baseline of the benchmark; never by the library.  It shares no source
 * file, header or table generator with the CUDA path.
 *
 * Steps, in the paper's order (Section 4, Algorithms 1 and 2):
 *   a2  walk generation (Alg. 1, lines 4-7; Section 4.1(a)): from every node,
 *       N_l walks of fixed length l for l = 0..L, in stratum order (walk r has
 *       length l when P[l] <= r < P[l+1]).  A step moves to a uniformly chosen
 *       in-neighbour (the out-neighbour on the reversed graph, Section 2.2).
 *       A walk that reaches a node without in-neighbours stops there.
 *   a3  shuffling (Section 4.1(b), Section 5.2): the source's walks are
 *       relabelled by one uniform permutation sigma (Fisher-Yates); pair j
 *       joins source walk sigma[j] with walk j of the target.
 *   a4  meeting detection (Section 4.2, Lemma 2, Algorithm 2): the pair meets
 *       when both walks visit the same node at the same step i >= 1; each
 *       pair counts once (Section 5.5) and adds the Lemma 7 weight of its two
 *       lengths, quantised to 2^-32 units and passed in by the caller.
 *
 * Random numbers: two generators of Salmon, Moraes, Dror, Shaw ("Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), restated from that paper's
 * definitions.  Philox4x32-10: ten rounds of two 32x32->64 multiplies by
 * 0xD2511F53 and 0xCD9E8D57, the two key words bumped by the Weyl constants
 * 0x9E3779B9 and 0xBB67AE85 between rounds.  Philox2x32-10: ten rounds of one
 * multiply by 0xD256D193, (x0, x1) -> (hi ^ k ^ x1, lo), the 32-bit key
 * bumped by 0x9E3779B9 between rounds.
 *   Fisher-Yates draw t (Philox4x32-10, key (seed mod 2^32, seed >> 32)):
 *           counter (t >> 1, 0xFFFFFFFF, 0xFFFFFFFF, s), words 2*(t&1) (high)
 *           and 2*(t&1)+1 (low) form R; k_t = floor(R * (t+1) / 2^64).
 *   walks (Philox2x32-10): the walk key of word q is
 *           kappa(seed, q) = h32(q ^ (mix64(seed) mod 2^32))
 *           (h32 and mix64 below; q = s: the source's walks, and its target
 *           walks by default).  Step i >= 1 of walk replica r from node v
 *           takes word (i-1)&1 of the block with counter
 *           (((i-1) >> 1) * 2^24 + r, v), w.  The in-neighbour index below
 *           d is Lemire's bounded draw (D. Lemire, "Fast random integer
 *           generation in an interval", ACM TOMACS 2019): floor(w d / 2^32)
 *           when (w d mod 2^32) >= (2^32 mod d), which gives every index
 *           exactly floor(2^32 / d) of the 2^32 words; otherwise (probability
 *           below d / 2^32) floor(R d / 2^64) with R = (y0 * 2^32 + y1) from
 *           the block of counter (c0 + 2^31, v) for an odd step and
 *           (c0, v + 2^31) for an even one (r < 2^24, i <= 255 and v < 2^31,
 *           so these never name a step's own block).  The index is uniform
 *           up to d / 2^64.
 *
 * Optional shared target walks (Algorithm 1 draws every node's walks once,
 * whatever the query): target walks then take the key kappa(seed,
 * 0xFFFFFFFE), so the walks of v are the same for every source and a batch of
 * sources can share them; source walks keep kappa(seed, s) (s < 2^31 and
 * kappa is injective in q, so the two keys differ).
 *
 * Optional literal shuffle of the targets' walks (every node's walks are
 * shuffled in Section 5.2; the default shuffles only the source's): target u
 * pairs walk pi_u(j) with source walk sigma[j], where pi_u is a keyed
 * permutation of 0..N_tot-1 (the identity when N_tot = 1): an unbalanced
 * 4-round Feistel network on b bits, b the smallest integer with
 * 2^b >= N_tot.  The value splits into A (the high floor(b/2) bits) and B
 * (the low ceil(b/2) bits); a round maps (A, B) to (B, A ^ (F_r(B) mod
 * 2^|A|)), so the two widths swap each round and are back after four.  The
 * round function of target u is F_r(B) = h32(B ^ K_r(u)), with h32 the
 * 32-bit finalizer "lowbias32" of C. Wellons ("Prospecting for hash
 * functions", 2018):
 *     x ^= x >> 16; x *= 0x7FEB352D; x ^= x >> 15; x *= 0x846CA68B; x ^= x >> 16
 * and the 32-bit round key K_r(u) = low half of mix64(k_r ^ u), where mix64
 * is the output function of SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014):
 *     z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
 *     z *= 0x94D049BB133111EB; z ^= z >> 31
 * and k_r = mix64(seed + (4 s + r + 1) 0x9E3779B97F4A7C15), the
 * (4s + r + 1)-th output of SplitMix64 seeded with seed.  The network is
 * applied to its own output until the value falls below N_tot (cycle
 * walking; fewer than two passes on average since 2^b < 2 N_tot).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u
#define PHILOX2_M 0xD256D193u

void srko_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                        uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void srko_philox2x32_10(const uint32_t ctr[2], uint32_t key, uint32_t out[2]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], k = key;
    for (int round = 0; round < 10; ++round) {
        uint64_t p = (uint64_t)PHILOX2_M * x0;
        uint32_t hi = (uint32_t)(p >> 32), lo = (uint32_t)p;
        x0 = hi ^ k ^ x1;
        x1 = lo;
        k += PHILOX_W0;
    }
    out[0] = x0; out[1] = x1;
}

/* floor(r * d / 2^64): a uniform index in [0, d) from a 64-bit draw. */
uint32_t srko_index(uint64_t r, uint32_t d) {
    return (uint32_t)(((unsigned __int128)r * d) >> 64);
}

static uint64_t draw64(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       uint64_t seed, int half) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    srko_philox4x32_10(ctr, key, w);
    return ((uint64_t)w[2 * half] << 32) | w[2 * half + 1];
}

/* Key word of the shared target walks, as a signed 32-bit value. */
#define SRKO_SHARED_KEY ((int32_t)-2)

static uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

static uint32_t h32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

/* kappa(seed, q): the Philox2x32-10 key of the walks of key word q. */
uint32_t srko_walk_key(uint64_t seed, uint32_t q) {
    return h32(q ^ (uint32_t)mix64(seed));
}

/* Lemire's bounded draw of an index in [0, d) from the 32-bit word w, with
 * the 64-bit draw r standing in when w is rejected. */
uint32_t srko_bounded(uint32_t w, uint32_t d, uint64_t r) {
    uint64_t m = (uint64_t)w * d;
    uint32_t low = (uint32_t)m;
    uint32_t threshold = (uint32_t)(((uint64_t)1 << 32) % d);
    if (low >= threshold) return (uint32_t)(m >> 32);
    return srko_index(r, d);
}

/* The in-neighbour index below d of step i of walk replica r from v. */
uint32_t srko_step_index(uint32_t key, int i, uint32_t r, uint32_t v, uint32_t d) {
    uint32_t c0 = ((uint32_t)(i - 1) >> 1) * 16777216u + r;
    uint32_t ctr[2] = {c0, v}, w[2];
    srko_philox2x32_10(ctr, key, w);
    int odd = ((i - 1) & 1) == 0;
    uint32_t alt[2] = {odd ? c0 + 2147483648u : c0, odd ? v : v + 2147483648u}, y[2];
    srko_philox2x32_10(alt, key, y);
    return srko_bounded(w[(i - 1) & 1], d, ((uint64_t)y[0] << 32) | y[1]);
}

/* One walk of nominal length `len` from v, replica r, key word q (the query
 * source, or SRKO_SHARED_KEY).  Writes the node at step i to pos[i-1];
 * returns the number of steps taken (smaller than len only when a node
 * without in-neighbours was reached). */
int srko_walk(const int32_t *row_ptr, const int32_t *col, int32_t v,
              int32_t r, int32_t q, uint64_t seed, int len, int32_t *pos) {
    uint32_t key = srko_walk_key(seed, (uint32_t)q);
    int32_t x = v;
    for (int i = 1; i <= len; ++i) {
        int32_t beg = row_ptr[x], deg = row_ptr[x + 1] - row_ptr[x];
        if (deg == 0) return i - 1;
        x = col[beg + srko_step_index(key, i, (uint32_t)r, (uint32_t)v, (uint32_t)deg)];
        pos[i - 1] = x;
    }
    return len;
}

/* pi_u(j): the keyed permutation of the literal target shuffle (see above). */
int32_t srko_feistel(int32_t u, int32_t s, uint64_t seed, int32_t N, int32_t j) {
    if (N <= 1) return 0;
    int b = 1;
    while (((int64_t)1 << b) < (int64_t)N) ++b;
    const int hi_bits = b / 2, lo_bits = b - hi_bits;
    uint32_t K[4];
    for (int r = 0; r < 4; ++r) {
        const uint64_t k = mix64(seed + (4 * (uint64_t)(uint32_t)s + (uint64_t)r + 1) *
                                            0x9E3779B97F4A7C15ull);
        K[r] = (uint32_t)mix64(k ^ (uint64_t)(uint32_t)u);
    }
    uint32_t v = (uint32_t)j;
    do {
        int na = hi_bits, nb = lo_bits;
        uint32_t A = v >> lo_bits, B = v & (((uint32_t)1 << lo_bits) - 1u);
        for (int r = 0; r < 4; ++r) {
            const uint32_t f = h32(B ^ K[r]);
            const uint32_t C = A ^ (f & (((uint32_t)1 << na) - 1u));
            A = B;
            B = C;
            const int t = na;
            na = nb;
            nb = t;
        }
        v = (A << nb) | B;
    } while (v >= (uint32_t)N);
    return (int32_t)v;
}

static int stratum_of(const int32_t *P, int L, int32_t r) {
    int lo = 0, hi = L;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (P[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* All N_tot = P[L+1] walks of node v in stratum order (step a2).  pos is
 * N_tot x max(L,1), -1 beyond a walk's end; eff[r] = steps walk r took. */
void srko_walks(const int32_t *row_ptr, const int32_t *col, int32_t v,
                int32_t s, uint64_t seed, int L, const int32_t *P,
                int32_t *pos, int32_t *eff) {
    int stride = L > 0 ? L : 1;
    int32_t N_tot = P[L + 1];
    for (int32_t r = 0; r < N_tot; ++r) {
        int len = stratum_of(P, L, r);
        int32_t *row = pos + (int64_t)r * stride;
        for (int i = 0; i < stride; ++i) row[i] = -1;
        eff[r] = srko_walk(row_ptr, col, v, r, s, seed, len, row);
    }
}

/* Step a3: sigma = one Fisher-Yates permutation of 0..N_tot-1 keyed by
 * (seed, s): for t = N_tot-1 down to 1, swap sigma[t] with sigma[k_t],
 * k_t uniform in [0, t]. */
void srko_fisher_yates(int32_t s, uint64_t seed, int32_t N_tot,
                       int32_t *sigma) {
    for (int32_t t = 0; t < N_tot; ++t) sigma[t] = t;
    for (int32_t t = N_tot - 1; t >= 1; --t) {
        uint64_t R = draw64((uint32_t)t >> 1, 0xFFFFFFFFu, 0xFFFFFFFFu,
                            (uint32_t)s, seed, t & 1);
        int32_t k = (int32_t)srko_index(R, (uint32_t)t + 1u);
        int32_t tmp = sigma[t];
        sigma[t] = sigma[k];
        sigma[k] = tmp;
    }
}

/*
 * Steps a2-a4 for query source s and the targets listed in `targets`
 * (literal != 0: target walks are paired through pi_u, see above; shared != 0:
 * target walks take the shared key, see above)
 * (n_targets entries; any node ids, s included).  wq is the (L+1)x(L+1)
 * quantised weight table, row l1 (source length), column l2 (target length).
 * Outputs per listed target: meet count, weight sum (2^-32 units) and the
 * number of target-walk steps a walker that stops at the first meeting, at a
 * node without in-neighbours or after min(l2, steps the source walk took)
 * steps would take.  Returns 0, or -1 when memory runs out.
 */
int srko_sampler(const int32_t *row_ptr, const int32_t *col, int32_t n,
                 int32_t s, uint64_t seed, int L, const int32_t *P,
                 const uint64_t *wq, const int32_t *targets,
                 int64_t n_targets, uint32_t *count, uint64_t *wsum,
                 uint64_t *steps, uint64_t *source_steps, int threads,
                 int literal, int shared) {
    (void)n;
    int stride = L > 0 ? L : 1;
    int32_t N_tot = P[L + 1];
    int32_t *spos = (int32_t *)malloc(sizeof(int32_t) * (size_t)N_tot * stride);
    int32_t *seff = (int32_t *)malloc(sizeof(int32_t) * (size_t)N_tot);
    int32_t *sigma = (int32_t *)malloc(sizeof(int32_t) * (size_t)N_tot);
    if (!spos || !seff || !sigma) {
        free(spos); free(seff); free(sigma);
        return -1;
    }
    /* a2: the source's walks */
    srko_walks(row_ptr, col, s, s, seed, L, P, spos, seff);
    if (source_steps) {
        uint64_t tot = 0;
        for (int32_t r = 0; r < N_tot; ++r) tot += (uint64_t)seff[r];
        *source_steps = tot;
    }
    /* a3: pairing by one uniform shuffle of the source's walks */
    srko_fisher_yates(s, seed, N_tot, sigma);

    int failed = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
    {
        int32_t *tpos = (int32_t *)malloc(sizeof(int32_t) * (size_t)stride);
        if (!tpos) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int64_t t = 0; t < n_targets; ++t) {
            int32_t u = targets[t];
            uint32_t cnt = 0;
            uint64_t ws = 0, st = 0;
            if (tpos && u != s) {
                for (int32_t j = 0; j < N_tot; ++j) {
                    /* a4: pair j = (source walk sigma[j], target walk j) */
                    /* target walk paired with source walk sigma[j] */
                    int32_t tw = literal ? srko_feistel(u, s, seed, N_tot, j) : j;
                    int l2 = stratum_of(P, L, tw);
                    int32_t w = sigma[j];
                    int l1 = stratum_of(P, L, w);
                    int teff = srko_walk(row_ptr, col, u, tw, shared ? SRKO_SHARED_KEY : s,
                                         seed, l2, tpos);
                    int m = teff < seff[w] ? teff : seff[w];
                    const int32_t *sp = spos + (int64_t)w * stride;
                    int met = 0;
                    for (int i = 1; i <= m; ++i) {
                        if (tpos[i - 1] == sp[i - 1]) { met = i; break; }
                    }
                    if (met) {
                        cnt += 1;
                        ws += wq[(int64_t)l1 * (L + 1) + l2];
                        st += (uint64_t)met;
                    } else {
                        st += (uint64_t)m;
                    }
                }
            }
            count[t] = cnt;
            wsum[t] = ws;
            steps[t] = st;
        }
        free(tpos);
    }
    free(spos); free(seff); free(sigma);
    return failed ? -1 : 0;
}
