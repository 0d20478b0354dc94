/*
 * Seeded synthetic-input support: the Jordan-Wigner image of a real, spin-free
 * electronic Hamiltonian.
 *
 * Input side of the iQCC path only (Sec. "Theoretical Framework", Eq. 1 -> Eq. 2;
 * App. A, Eq. 8 -> Eq. 9).  Neither the dressing nor the energy/gradient
 * arithmetic lives here; this file only turns integrals into a list of real
 * Pauli strings that both the CUDA library and the oracle consume.
 *
 *   H = sum_{pq,s} h_pq a+_{ps} a_{qs}
 *     + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
 *
 * (App. A's physicist form g_ijkl a+_i a+_j a_l a_k with g_ijkl = (ik|jl).)
 * Spin orbital P = 2p + s (alpha/beta interleaved), qubit j = spin orbital j,
 * |1> = occupied.  With these conventions
 *
 *   a+_P = Z_{<P} X_P (I + Z_P)/2 ,   a_P = Z_{<P} X_P (I - Z_P)/2 ,
 *
 * so every ladder operator is a real combination of "X^x Z^z" words (per
 * qubit: X^{x_j} Z^{z_j}).  Products of such words only pick up signs,
 * (X^a Z^b)(X^c Z^d) = (-1)^{popc(b & c)} X^{a^c} Z^{b^d}, and the final
 * word is converted to a Hermitian Pauli string with X^x Z^z = (-i)^{#Y} P(x,z),
 * #Y = popc(x & z).  Odd-#Y parts cancel between an operator and its
 * Hermitian conjugate (both are generated from the same index multiset), so
 * only even-#Y strings are kept.
 *
 * Enumeration: index multisets {a<=b(<=c<=d)} of spin orbitals; for each, all
 * distinct orderings are expanded into a 16-entry local accumulator (one entry
 * per z-pattern on the multiset's distinct sites), which is then flushed into
 * the output (see flush()).  The output order is fixed by the loop order
 * (deterministic, not sorted).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define MAXW 4

typedef struct {
    uint64_t k[2 * MAXW]; /* x[0..W-1], z[0..W-1] */
    double c;
    int used;
} slot_t;

typedef struct {
    int W;
    size_t cap; /* power of two */
    size_t n;
    slot_t* s;
} table_t;

static uint64_t mix64(uint64_t h) {
    h ^= h >> 33; h *= 0xff51afd7ed558ccdULL;
    h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ULL;
    h ^= h >> 33;
    return h;
}

static uint64_t key_hash(const uint64_t* k, int W) {
    uint64_t h = 0x9e3779b97f4a7c15ULL;
    for (int i = 0; i < 2 * W; ++i) h = mix64(h ^ (k[i] + 0x632be59bd9b4e019ULL * (uint64_t)(i + 1)));
    return h;
}

static int table_init(table_t* t, int W, size_t cap) {
    t->W = W; t->cap = cap; t->n = 0;
    t->s = (slot_t*)calloc(cap, sizeof(slot_t));
    return t->s ? 0 : -1;
}

static int table_add(table_t* t, const uint64_t* k, double c);

static int table_grow(table_t* t) {
    table_t nt;
    if (table_init(&nt, t->W, t->cap * 2)) return -1;
    for (size_t i = 0; i < t->cap; ++i)
        if (t->s[i].used && table_add(&nt, t->s[i].k, t->s[i].c)) { free(nt.s); return -1; }
    free(t->s);
    *t = nt;
    return 0;
}

static int table_add(table_t* t, const uint64_t* k, double c) {
    if (2 * (t->n + 1) > t->cap && table_grow(t)) return -1;
    int L = 2 * t->W;
    size_t i = key_hash(k, t->W) & (t->cap - 1);
    for (;;) {
        slot_t* s = &t->s[i];
        if (!s->used) {
            s->used = 1; memcpy(s->k, k, sizeof(uint64_t) * L); s->c = c; t->n++;
            return 0;
        }
        if (memcmp(s->k, k, sizeof(uint64_t) * L) == 0) { s->c += c; return 0; }
        i = (i + 1) & (t->cap - 1);
    }
}

static inline void setbit(uint64_t* w, int j) { w[j >> 6] ^= (1ULL << (j & 63)); }
static inline int getbit(const uint64_t* w, int j) { return (int)((w[j >> 6] >> (j & 63)) & 1ULL); }

/* XOR of the "Z below P" masks for P = 0..n-1, as words. */
static void below_mask(uint64_t* m, int P, int W) {
    memset(m, 0, sizeof(uint64_t) * W);
    for (int j = 0; j < P; ++j) setbit(m, j);
}

/*
 * One ordered operator product O_1 ... O_L (L = 2 or 4), creators first then
 * annihilators, on spin orbitals idx[0..L-1], with scalar weight v, expanded
 * over its 2^L (I +- Z) choices and added to acc[16] (indexed by the z-pattern
 * on the multiset's distinct sites u[0..nu-1]).
 */
static void expand_product(const int* idx, int L, int ncre, double v,
                           const int* u, int nu, double* acc) {
    /* Reordering sign: moving word k left past words j < k costs bit idx[k] of
       z_j, with z_j = below(idx[j]) ^ b_j e_{idx[j]}.  The b-independent part is
       the inversion count s0; the b-dependent part is b_j for every later k on
       the same site.  Annihilators add b_k from their (I - Z).  So the sign of
       pattern b is (-1)^(s0 + popc(b & E)). */
    int s0 = 0, E = 0, site[4];
    for (int k = 0; k < L; ++k) {
        for (int j = 0; j < k; ++j) s0 ^= (idx[k] < idx[j]);
        int e = (k >= ncre);
        for (int l = k + 1; l < L; ++l) e ^= (idx[l] == idx[k]);
        if (e) E |= (1 << k);
        site[k] = 0;
        for (int t = 0; t < nu; ++t) if (u[t] == idx[k]) { site[k] = t; break; }
    }
    double w = v / (double)(1 << L);
    for (int b = 0; b < (1 << L); ++b) {
        int pat = 0;
        for (int k = 0; k < L; ++k) if ((b >> k) & 1) pat ^= (1 << site[k]);
        int sgn = s0 ^ (__builtin_popcount((unsigned)(b & E)) & 1);
        acc[pat] += sgn ? -w : w;
    }
}

/* Growable output array of rows (2W key words + coefficient bits). */
typedef struct { uint64_t* r; size_t n, cap; int L; } rows_t;

static int rows_push(rows_t* o, const uint64_t* key, double c, int W) {
    if (o->n == o->cap) {
        size_t nc = o->cap ? 2 * o->cap : 1 << 16;
        uint64_t* p = (uint64_t*)realloc(o->r, sizeof(uint64_t) * o->L * nc);
        if (!p) return -1;
        o->r = p; o->cap = nc;
    }
    memcpy(o->r + o->n * o->L, key, sizeof(uint64_t) * 2 * W);
    memcpy(o->r + o->n * o->L + 2 * W, &c, sizeof(double));
    o->n++;
    return 0;
}

/* Flush a multiset's local accumulator.  A multiset of four distinct sites has
   a 4-bit flip mask that no other multiset produces, and its 16 patterns have
   distinct z, so its strings go straight to the output; all other strings are
   summed in the table. */
static int flush(table_t* t, rows_t* o, const int* idx, int L, const int* u, int nu,
                 const double* acc, int W) {
    uint64_t x[MAXW], zb[MAXW], m[MAXW];
    memset(x, 0, sizeof x); memset(zb, 0, sizeof zb);
    for (int k = 0; k < L; ++k) {
        setbit(x, idx[k]);
        below_mask(m, idx[k], W);
        for (int w = 0; w < W; ++w) zb[w] ^= m[w];
    }
    for (int pat = 0; pat < (1 << nu); ++pat) {
        if (acc[pat] == 0.0) continue;
        uint64_t key[2 * MAXW];
        memset(key, 0, sizeof key);
        for (int w = 0; w < W; ++w) { key[w] = x[w]; key[W + w] = zb[w]; }
        for (int s = 0; s < nu; ++s) if ((pat >> s) & 1) setbit(key + W, u[s]);
        int ny = 0;
        for (int w = 0; w < W; ++w) ny += __builtin_popcountll(key[w] & key[W + w]);
        if (ny & 1) continue; /* imaginary part: cancels against the Hermitian conjugate */
        double c = ((ny / 2) & 1) ? -acc[pat] : acc[pat];
        if (nu == 4 && L == 4) { if (rows_push(o, key, c, W)) return -1; }
        else if (table_add(t, key, c)) return -1;
    }
    return 0;
}

/* Distinct permutations of a sorted small array (lexicographic next permutation). */
static int next_perm(int* a, int L) {
    int i = L - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = L - 1;
    while (a[j] <= a[i]) --j;
    int tmp = a[i]; a[i] = a[j]; a[j] = tmp;
    for (int l = i + 1, r = L - 1; l < r; ++l, --r) { tmp = a[l]; a[l] = a[r]; a[r] = tmp; }
    return 1;
}

static int distinct_sites(const int* ms, int L, int* u) {
    int nu = 0;
    for (int k = 0; k < L; ++k) if (nu == 0 || u[nu - 1] != ms[k]) u[nu++] = ms[k];
    return nu;
}

/*
 * Build the JW Hamiltonian.  h: [norb][norb], eri: [norb]^4 chemist order
 * (pq|rs) at ((p*norb+q)*norb+r)*norb+s.  Strings with |c| < rel_drop*max|c|
 * are dropped.  On success *out_rows is a malloc'd array of M rows of
 * (2W words + 1 double as bits), unique keys in generator order; returns M,
 * or -1 on error.
 */
long long hamgen_jw(int norb, const double* h, const double* eri, double rel_drop,
                    uint64_t** out_rows) {
    int n = 2 * norb;
    int W = (n + 63) / 64;
    if (n < 2 || W > MAXW) return -1;
    table_t t;
    if (table_init(&t, W, 1 << 16)) return -1;
    rows_t o = {NULL, 0, 0, 2 * W + 1};

    /* one-body part: multisets {a <= b} */
    for (int a = 0; a < n; ++a)
        for (int b = a; b < n; ++b) {
            int ms[2] = {a, b}, u[4], nu = distinct_sites(ms, 2, u);
            double acc[16] = {0};
            int perm[2] = {a, b};
            do {
                int P = perm[0], Q = perm[1];
                if ((P & 1) != (Q & 1)) continue;
                double v = h[(P >> 1) * norb + (Q >> 1)];
                if (v == 0.0) continue;
                expand_product(perm, 2, 1, v, u, nu, acc);
            } while (next_perm(perm, 2));
            if (flush(&t, &o, ms, 2, u, nu, acc, W)) goto fail;
        }

    /* two-body part: multisets {a <= b <= c <= d}; ordering (i1,i2,i3,i4) means
       a+_{i1} a+_{i2} a_{i3} a_{i4} with weight 1/2 (p1 p4 | p2 p3). */
    for (int a = 0; a < n; ++a)
        for (int b = a; b < n; ++b)
            for (int c = b; c < n; ++c)
                for (int d = c; d < n; ++d) {
                    int ms[4] = {a, b, c, d}, u[4], nu = distinct_sites(ms, 4, u);
                    double acc[16] = {0};
                    int any = 0;
                    int perm[4] = {a, b, c, d};
                    do {
                        int i1 = perm[0], i2 = perm[1], i3 = perm[2], i4 = perm[3];
                        if (i1 == i2 || i3 == i4) continue;
                        if ((i1 & 1) != (i4 & 1) || (i2 & 1) != (i3 & 1)) continue;
                        int p = i1 >> 1, q = i4 >> 1, r = i2 >> 1, s = i3 >> 1;
                        double v = 0.5 * eri[((size_t)(p * norb + q) * norb + r) * norb + s];
                        if (v == 0.0) continue;
                        expand_product(perm, 4, 2, v, u, nu, acc);
                        any = 1;
                    } while (next_perm(perm, 4));
                    if (any && flush(&t, &o, ms, 4, u, nu, acc, W)) goto fail;
                }

    /* move the table's strings to the output, then drop tiny and zero strings */
    for (size_t i = 0; i < t.cap; ++i)
        if (t.s[i].used && rows_push(&o, t.s[i].k, t.s[i].c, W)) goto fail;
    free(t.s); t.s = NULL;
    {
        int L = o.L;
        double cmax = 0.0, c;
        for (size_t i = 0; i < o.n; ++i) {
            memcpy(&c, o.r + i * L + 2 * W, sizeof c);
            if (fabs(c) > cmax) cmax = fabs(c);
        }
        double thr = rel_drop * cmax;
        size_t k = 0;
        for (size_t i = 0; i < o.n; ++i) {
            memcpy(&c, o.r + i * L + 2 * W, sizeof c);
            if (c == 0.0 || fabs(c) < thr) continue;
            if (k != i) memmove(o.r + k * L, o.r + i * L, sizeof(uint64_t) * L);
            ++k;
        }
        if (k == 0) { free(o.r); o.r = (uint64_t*)malloc(sizeof(uint64_t) * L); if (!o.r) return -1; }
        *out_rows = o.r;
        return (long long)k;
    }
fail:
    free(t.s);
    free(o.r);
    return -1;
}

void hamgen_free(uint64_t* p) { free(p); }
