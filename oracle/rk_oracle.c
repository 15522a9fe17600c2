/*
 * Oracle for multi-pattern Rabin-Karp matching.  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the bench's CPU-baseline / reference legs
 * load it; the product (the CUDA library and its binding) never does.
 *
 * What is computed (the problem of Section 1: find every occurrence of every
 * pattern in a text; per-offset windows of Section 3.1):
 *
 *     M = { (p, x) : 0 <= p < k, 0 <= x <= n - len_p,
 *                    T[x .. x + len_p) == P_p byte for byte }
 *
 * reported in ascending (p, x) order.  Readings of the paper used here:
 *   - the last window x = n - len_p is included (the GPU listing's bound
 *     "x <= n - m"; the sequential listing's "x < n - m" drops it);
 *   - bytes are unsigned and compared exactly;
 *   - each pattern index is reported on its own, duplicates included;
 *   - a pattern longer than the text has no window.
 *
 * Two independent implementations, sharing no code:
 *   oracle_bruteforce   the definition: compare every window with every
 *                       pattern (the brute-force matcher named in Section 2);
 *   oracle_rabin_karp   Section 3.1's method generalised to a pattern set:
 *                       hash every pattern once, hash every window of each
 *                       pattern length, and compare bytes only where the
 *                       hashes agree.
 * and the Rabin hash itself, in the paper's Horner form (h = h*B + c, Section
 * 3.1, where the paper takes B = 2 and no modulus) reduced mod p = 2^61 - 1:
 *   oracle_hash                h(s) = sum_i s[i] * B^(len-1-i)  mod p
 *   oracle_window_hashes       h of every window, by the rolling update
 *                              h' = (h - T[x] * B^(L-1)) * B + T[x+L]  mod p
 *
 * ORACLE_MUTANT (compile-time, tests only) plants one known mistake so the
 * tests can show their pins catch it; 0 = the real oracle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_P ((uint64_t)0x1FFFFFFFFFFFFFFFull) /* 2^61 - 1 */

/* (a * b) mod p through a full 128-bit product. */
uint64_t oracle_mulmod(uint64_t a, uint64_t b) {
    unsigned __int128 prod = (unsigned __int128)(a % ORACLE_P) * (unsigned __int128)(b % ORACLE_P);
#if ORACLE_MUTANT == 8
    /* mutant: one Mersenne fold, no final conditional subtract */
    return (uint64_t)(prod & ORACLE_P) + (uint64_t)(prod >> 61);
#else
    return (uint64_t)(prod % ORACLE_P);
#endif
}

static uint64_t addmod(uint64_t a, uint64_t b) { /* a, b < p */
    uint64_t s = a + b;
    return s >= ORACLE_P ? s - ORACLE_P : s;
}

static uint64_t submod(uint64_t a, uint64_t b) { /* a, b < p */
    return a >= b ? a - b : a + ORACLE_P - b;
}

/* B^e mod p by repeated squaring. */
uint64_t oracle_powmod(uint64_t base, uint64_t e) {
    uint64_t r = 1 % ORACLE_P, b = base % ORACLE_P;
    while (e) {
        if (e & 1) r = oracle_mulmod(r, b);
        b = oracle_mulmod(b, b);
        e >>= 1;
    }
    return r;
}

/* Rabin hash of s[0..len): Horner's rule h = h*B + s[i], reduced mod p. */
uint64_t oracle_hash(const uint8_t *s, uint64_t len, uint64_t base) {
    uint64_t h = 0;
    for (uint64_t i = 0; i < len; ++i) {
#if ORACLE_MUTANT == 5
        uint8_t c = s[len - 1 - i]; /* mutant: operand order reversed */
#else
        uint8_t c = s[i];
#endif
        h = addmod(oracle_mulmod(h, base), (uint64_t)c);
    }
    return h;
}

/* Hash of every window T[x..x+L), x = 0..n-L, by the rolling update.
 * out must hold n-L+1 values.  Returns the number written (0 if L > n or L = 0). */
uint64_t oracle_window_hashes(const uint8_t *T, uint64_t n, uint64_t L, uint64_t base,
                              uint64_t *out) {
    if (L == 0 || L > n) return 0;
#if ORACLE_MUTANT == 3
    uint64_t top = oracle_powmod(base, L); /* mutant: wrong exponent */
#else
    uint64_t top = oracle_powmod(base, L - 1); /* weight of the outgoing byte */
#endif
    uint64_t h = oracle_hash(T, L, base);
    uint64_t nw = n - L + 1;
    out[0] = h;
    for (uint64_t x = 0; x + 1 < nw; ++x) {
        h = submod(h, oracle_mulmod((uint64_t)T[x], top));
        h = addmod(oracle_mulmod(h, base), (uint64_t)T[x + L]);
        out[x + 1] = h;
    }
    return nw;
}

/* ---------------------------------------------------------------- brute force */

/* Writes up to cap matches (pattern id, offset) in ascending (p, x) order and
 * returns the total number of matches.  Patterns are concatenated in P with
 * lengths lens[0..k). */
int64_t oracle_bruteforce(const uint8_t *T, uint64_t n, const uint8_t *P, const uint32_t *lens,
                          uint32_t k, uint32_t *out_pid, uint64_t *out_off, uint64_t cap) {
    uint64_t count = 0, poff = 0;
    for (uint32_t p = 0; p < k; ++p) {
        uint64_t m = lens[p];
        const uint8_t *pat = P + poff;
        poff += m;
        if (m == 0 || m > n) continue;
#if ORACLE_MUTANT == 1
        uint64_t last = n - m; /* mutant: the sequential listing's bound drops x = n-m */
        for (uint64_t x = 0; x < last; ++x) {
#else
        for (uint64_t x = 0; x + m <= n; ++x) {
#endif
            uint64_t i = 0;
#if ORACLE_MUTANT == 4
            uint64_t cmp_len = m - 1; /* mutant: last byte never compared */
#else
            uint64_t cmp_len = m;
#endif
            while (i < cmp_len && T[x + i] == pat[i]) ++i;
            if (i == cmp_len) {
                if (count < cap) {
                    out_pid[count] = p;
                    out_off[count] = x;
                }
                ++count;
            }
        }
    }
    return (int64_t)count;
}

/* ---------------------------------------------------------------- Rabin-Karp */

typedef struct {
    uint64_t h;
    uint32_t pid;
} hp_pair;

typedef struct {
    uint32_t pid;
    uint64_t off;
} match_rec;

static int cmp_hp(const void *a, const void *b) {
    const hp_pair *x = (const hp_pair *)a, *y = (const hp_pair *)b;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    return x->pid < y->pid ? -1 : (x->pid > y->pid);
}

static int cmp_match(const void *a, const void *b) {
    const match_rec *x = (const match_rec *)a, *y = (const match_rec *)b;
    if (x->pid != y->pid) return x->pid < y->pid ? -1 : 1;
    return x->off < y->off ? -1 : (x->off > y->off);
}

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y);
}

/* first index i in [0, cnt) with tab[i].h >= h */
static uint64_t lower_bound(const hp_pair *tab, uint64_t cnt, uint64_t h) {
    uint64_t lo = 0, hi = cnt;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (tab[mid].h < h) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Same contract as oracle_bruteforce; base is the Rabin base B (2 <= B < p).
 * Returns -1 if memory runs out. */
int64_t oracle_rabin_karp(const uint8_t *T, uint64_t n, const uint8_t *P, const uint32_t *lens,
                          uint32_t k, uint64_t base, uint32_t *out_pid, uint64_t *out_off,
                          uint64_t cap) {
    if (k == 0) return 0;
    uint64_t *poff = (uint64_t *)malloc(sizeof(uint64_t) * k);
    uint32_t *dl = (uint32_t *)malloc(sizeof(uint32_t) * k);
    hp_pair *tab = (hp_pair *)malloc(sizeof(hp_pair) * k);
    uint64_t mcap = 1024, mcount = 0;
    match_rec *ms = (match_rec *)malloc(sizeof(match_rec) * mcap);
    if (!poff || !dl || !tab || !ms) {
        free(poff); free(dl); free(tab); free(ms);
        return -1;
    }
    uint64_t acc = 0;
    for (uint32_t p = 0; p < k; ++p) {
        poff[p] = acc;
        acc += lens[p];
        dl[p] = lens[p];
    }
    /* distinct pattern lengths */
    qsort(dl, k, sizeof(uint32_t), cmp_u32);
    uint32_t nd = 0;
    for (uint32_t i = 0; i < k; ++i)
        if (i == 0 || dl[i] != dl[i - 1]) dl[nd++] = dl[i];

    for (uint32_t g = 0; g < nd; ++g) {
        uint64_t L = dl[g];
        if (L == 0 || L > n) continue;
        /* pattern hashes hx for this length, sorted for lookup */
        uint64_t cnt = 0;
        for (uint32_t p = 0; p < k; ++p)
            if (lens[p] == L) {
                tab[cnt].h = oracle_hash(P + poff[p], L, base);
                tab[cnt].pid = p;
                ++cnt;
            }
        qsort(tab, cnt, sizeof(hp_pair), cmp_hp);
        /* window hashes hy by the rolling update */
#if ORACLE_MUTANT == 3
        uint64_t top = oracle_powmod(base, L);
#else
        uint64_t top = oracle_powmod(base, L - 1);
#endif
        uint64_t hy = oracle_hash(T, L, base);
#if ORACLE_MUTANT == 1
        uint64_t nwin = n - L; /* mutant: drops the last window */
#else
        uint64_t nwin = n - L + 1;
#endif
        for (uint64_t x = 0; x < nwin; ++x) {
            if (x > 0) {
                hy = submod(hy, oracle_mulmod((uint64_t)T[x - 1], top));
#if ORACLE_MUTANT == 7
                hy = addmod(oracle_mulmod(hy, base), (uint64_t)T[x - 2 + L]); /* mutant: incoming byte one early */
#else
                hy = addmod(oracle_mulmod(hy, base), (uint64_t)T[x - 1 + L]);
#endif
            }
            for (uint64_t i = lower_bound(tab, cnt, hy); i < cnt && tab[i].h == hy; ++i) {
                uint32_t p = tab[i].pid;
#if ORACLE_MUTANT == 2
                int equal = 1; /* mutant: hash equality taken as a match */
#else
                int equal = memcmp(P + poff[p], T + x, L) == 0;
#endif
                if (!equal) continue;
                if (mcount == mcap) {
                    mcap *= 2;
                    match_rec *nm = (match_rec *)realloc(ms, sizeof(match_rec) * mcap);
                    if (!nm) {
                        free(poff); free(dl); free(tab); free(ms);
                        return -1;
                    }
                    ms = nm;
                }
                ms[mcount].pid = p;
                ms[mcount].off = x;
                ++mcount;
#if ORACLE_MUTANT == 6
                break; /* mutant: one pattern id per hash value (duplicates collapsed) */
#endif
            }
        }
    }
    qsort(ms, mcount, sizeof(match_rec), cmp_match);
    for (uint64_t i = 0; i < mcount && i < cap; ++i) {
        out_pid[i] = ms[i].pid;
        out_off[i] = ms[i].off;
    }
    free(poff); free(dl); free(tab); free(ms);
    return (int64_t)mcount;
}

int oracle_mutant_id(void) { return ORACLE_MUTANT; }
