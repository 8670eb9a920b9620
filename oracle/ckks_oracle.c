/*
 * ckks_oracle.c -- plain CPU reference of the RNS-CKKS server path.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The GPU library never
 * links, loads or calls it, and the two share no source, header or table.
 *
 * Everything here works in the coefficient domain: a polynomial of
 * R_q = Z_q[X]/(X^N + 1) (Section 2.2) is N residues in [0, q); an RNS
 * polynomial is [limbs][N], limb i reduced modulo moduli[i].  Ring products
 * are negacyclic convolutions, computed with a textbook number-theoretic
 * transform used as a library primitive (evaluation at the odd powers of a
 * primitive 2N-th root psi).  Limb loops carry OpenMP pragmas; they compute
 * independent limbs and change no result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Modular arithmetic.  q is an odd prime below 2^62.                    */
/* Barrett reduction of x < q^2 (Menezes, van Oorschot, Vanstone,        */
/* Handbook of Applied Cryptography, Algorithm 14.42, radix 2):          */
/* k = bitlen(q), mu = floor(2^(2k) / q).                                */
/* ------------------------------------------------------------------ */
typedef struct { u64 q; u64 mu; int k; } modulus;

static modulus mk_mod(u64 q) {
    modulus m;
    m.q = q;
    m.k = 64 - __builtin_clzll(q);
    m.mu = (u64)(((u128)1 << (2 * m.k)) / q);
    return m;
}

static inline u64 barrett(u128 x, const modulus *m) {
    u128 q1 = x >> (m->k - 1);
    u128 q3 = (q1 * m->mu) >> (m->k + 1);
    u128 r = x - q3 * m->q;
    while (r >= m->q) r -= m->q;
    return (u64)r;
}

static inline u64 mulmod(u64 a, u64 b, const modulus *m) { return barrett((u128)a * b, m); }
static inline u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

static u64 powmod(u64 a, u64 e, const modulus *m) {
    u64 r = 1 % m->q;
    a %= m->q;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

static u64 invmod(u64 a, const modulus *m) { return powmod(a, m->q - 2, m); } /* q prime */

u64 or_mulmod(u64 a, u64 b, u64 q) { modulus m = mk_mod(q); return mulmod(a % q, b % q, &m); }
u64 or_powmod(u64 a, u64 e, u64 q) { modulus m = mk_mod(q); return powmod(a, e, &m); }

/* ------------------------------------------------------------------ */
/* NTT tables: pw[e] = psi^e, ipw[e] = psi^-e for 0 <= e < 2N.          */
/* ------------------------------------------------------------------ */
typedef struct { u64 q, psi, n; modulus m; u64 ninv; u64 *pw, *ipw; } ntt_table;

#define MAX_TABLES 256
static ntt_table g_tables[MAX_TABLES];
static int g_ntables = 0;

static const ntt_table *get_table(u64 q, u64 psi, u64 n) {
    const ntt_table *found = NULL;
#pragma omp critical(or_tables)
    {
        for (int i = 0; i < g_ntables; i++)
            if (g_tables[i].q == q && g_tables[i].psi == psi && g_tables[i].n == n) { found = &g_tables[i]; break; }
        if (!found && g_ntables < MAX_TABLES) {
            ntt_table *t = &g_tables[g_ntables];
            t->q = q; t->psi = psi; t->n = n; t->m = mk_mod(q);
            t->pw = (u64 *)malloc(2 * n * sizeof(u64));
            t->ipw = (u64 *)malloc(2 * n * sizeof(u64));
            u64 ipsi = invmod(psi, &t->m);
            t->pw[0] = 1; t->ipw[0] = 1;
            for (u64 e = 1; e < 2 * n; e++) {
                t->pw[e] = mulmod(t->pw[e - 1], psi, &t->m);
                t->ipw[e] = mulmod(t->ipw[e - 1], ipsi, &t->m);
            }
            t->ninv = invmod(n % q, &t->m);
            g_ntables++;
            found = t;
        }
    }
    return found;
}

static void bitrev_perm(u64 *a, u64 n) {
    for (u64 i = 1, j = 0; i < n; i++) {
        u64 bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* out[k] = sum_i a[i] psi^((2k+1) i): twist by psi^i, then a cyclic radix-2
   decimation-in-time transform with omega = psi^2 (natural order out). */
static void ntt_tab(u64 *a, const ntt_table *T) {
    const u64 n = T->n, q = T->q;
    const modulus *m = &T->m;
    for (u64 i = 0; i < n; i++) a[i] = mulmod(a[i], T->pw[i], m);
    bitrev_perm(a, n);
    for (u64 len = 2; len <= n; len <<= 1) {
        const u64 half = len >> 1, step = 2 * (n / len);
        for (u64 i = 0; i < n; i += len)
            for (u64 j = 0; j < half; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + half], T->pw[j * step], m);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
}

/* inverse of ntt_tab */
static void intt_tab(u64 *a, const ntt_table *T) {
    const u64 n = T->n, q = T->q;
    const modulus *m = &T->m;
    bitrev_perm(a, n);
    for (u64 len = 2; len <= n; len <<= 1) {
        const u64 half = len >> 1, step = 2 * (n / len);
        for (u64 i = 0; i < n; i += len)
            for (u64 j = 0; j < half; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + half], T->ipw[j * step], m);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
    for (u64 i = 0; i < n; i++) a[i] = mulmod(mulmod(a[i], T->ninv, m), T->ipw[i], m);
}

void or_ntt(u64 *a, u64 n, u64 q, u64 psi) { ntt_tab(a, get_table(q, psi, n)); }
void or_intt(u64 *a, u64 n, u64 q, u64 psi) { intt_tab(a, get_table(q, psi, n)); }

/* The definition, O(N^2): out[k] = sum_i a[i] psi^((2k+1) i mod 2N). */
void or_ntt_direct(const u64 *a, u64 *out, u64 n, u64 q, u64 psi) {
    modulus m = mk_mod(q);
    for (u64 k = 0; k < n; k++) {
        u64 acc = 0;
        for (u64 i = 0; i < n; i++)
            acc = addmod(acc, mulmod(a[i], powmod(psi, ((2 * k + 1) * i) % (2 * n), &m), &m), q);
        out[k] = acc;
    }
}

/* negacyclic product in Z_q[X]/(X^N+1) */
static void polymul_tab(const u64 *a, const u64 *b, u64 *out, const ntt_table *T) {
    const u64 n = T->n;
    u64 *fa = (u64 *)malloc(n * sizeof(u64)), *fb = (u64 *)malloc(n * sizeof(u64));
    memcpy(fa, a, n * sizeof(u64));
    memcpy(fb, b, n * sizeof(u64));
    ntt_tab(fa, T);
    ntt_tab(fb, T);
    for (u64 i = 0; i < n; i++) fa[i] = mulmod(fa[i], fb[i], &T->m);
    intt_tab(fa, T);
    memcpy(out, fa, n * sizeof(u64));
    free(fa);
    free(fb);
}

void or_polymul(const u64 *a, const u64 *b, u64 *out, u64 n, u64 q, u64 psi) {
    polymul_tab(a, b, out, get_table(q, psi, n));
}

/* ------------------------------------------------------------------ */
/* RNS polynomials [limbs][n]                                          */
/* ------------------------------------------------------------------ */
static void prepare_tables(const u64 *moduli, const u64 *psis, u64 limbs, u64 n) {
    for (u64 i = 0; i < limbs; i++) (void)get_table(moduli[i], psis[i], n);
}

void or_rns_polymul(const u64 *a, const u64 *b, u64 *out, u64 limbs, u64 n, const u64 *moduli, const u64 *psis) {
    prepare_tables(moduli, psis, limbs, n);
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 i = 0; i < (i64)limbs; i++)
        polymul_tab(a + i * n, b + i * n, out + i * n, get_table(moduli[i], psis[i], n));
}

/* out = a * c with c given by its residue per limb */
void or_rns_mul_scalar(const u64 *a, const u64 *cres, u64 *out, u64 limbs, u64 n, const u64 *moduli) {
    for (u64 i = 0; i < limbs; i++) {
        modulus m = mk_mod(moduli[i]);
        for (u64 k = 0; k < n; k++) out[i * n + k] = mulmod(a[i * n + k], cres[i], &m);
    }
}

/* a(X) -> a(X^g) for odd g: coefficient i moves to i*g mod 2N, negated
   when that index lands in [N, 2N) because X^N = -1. */
void or_rns_automorphism(const u64 *a, u64 *out, u64 limbs, u64 n, const u64 *moduli, u64 g) {
    for (u64 l = 0; l < limbs; l++) {
        const u64 q = moduli[l];
        for (u64 i = 0; i < n; i++) {
            u64 j = (i * (g % (2 * n))) % (2 * n);
            u64 v = a[l * n + i];
            if (j < n) out[l * n + j] = v;
            else out[l * n + (j - n)] = v ? q - v : 0;
        }
    }
}

/* Rescale (Section 2.5): drop limb l = top, rounding half up.
   a: [comps][l+1][n] -> out: [comps][l][n];
   out_i = (a_i + [floor(q_l/2)]_{q_i} - [[a_l + floor(q_l/2)]_{q_l}]_{q_i}) * q_l^{-1} mod q_i. */
void or_rescale(const u64 *a, u64 *out, u64 comps, u64 l, u64 n, const u64 *moduli) {
    const u64 ql = moduli[l], half = (ql - 1) / 2;
    for (u64 c = 0; c < comps; c++) {
        const u64 *top = a + (c * (l + 1) + l) * n;
        for (u64 i = 0; i < l; i++) {
            const u64 qi = moduli[i];
            modulus m = mk_mod(qi);
            const u64 inv = invmod(ql % qi, &m), hi = half % qi;
            const u64 *src = a + (c * (l + 1) + i) * n;
            u64 *dst = out + (c * l + i) * n;
            for (u64 k = 0; k < n; k++) {
                u64 r = addmod(top[k], half, ql) % qi;
                dst[k] = mulmod(submod(addmod(src[k], hi, qi), r, qi), inv, &m);
            }
        }
    }
}

/* Fast base conversion of x given by residues modulo the primes src[0..ns)
   to the prime p: sum_i [x_i * (Qs/q_i)^{-1}]_{q_i} * ((Qs/q_i) mod p)  mod p.
   The result is (x + u*Qs) mod p for some 0 <= u < ns. */
static void base_convert(const u64 *x, const u64 *src, u64 ns, u64 p, u64 n, u64 *out) {
    modulus mp = mk_mod(p);
    u64 inv_hat[64], hat_p[64];
    for (u64 i = 0; i < ns; i++) {
        modulus mi = mk_mod(src[i]);
        u64 hi = 1 % src[i], hp = 1 % p;
        for (u64 j = 0; j < ns; j++) if (j != i) {
            hi = mulmod(hi, src[j] % src[i], &mi);
            hp = mulmod(hp, src[j] % p, &mp);
        }
        inv_hat[i] = invmod(hi, &mi);
        hat_p[i] = hp;
    }
    for (u64 k = 0; k < n; k++) {
        u64 acc = 0;
        for (u64 i = 0; i < ns; i++) {
            modulus mi = mk_mod(src[i]);
            u64 y = mulmod(x[i * n + k], inv_hat[i], &mi);
            acc = addmod(acc, mulmod(y % p, hat_p[i], &mp), p);
        }
        out[k] = acc;
    }
}

void or_base_convert(const u64 *x, const u64 *src, u64 ns, const u64 *dst, u64 nd, u64 n, u64 *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 t = 0; t < (i64)nd; t++) base_convert(x, src, ns, dst[t], n, out + t * n);
}

/* ModDown: c given modulo q_0..q_{nq-1}, p_0..p_{K-1} ([nq+K][n]);
   out = floor((c + floor(P/2)) / P) up to the base-conversion excess,
   i.e. out_i = (c_i + [floor(P/2)]_{q_i} - Conv_{P->q_i}(c + floor(P/2))) * P^{-1} mod q_i. */
void or_moddown(const u64 *c, u64 nq, u64 K, const u64 *moduli, u64 n, u64 *out) {
    const u64 *ps = moduli + nq;
    u64 *v = (u64 *)malloc(K * n * sizeof(u64));
    for (u64 k = 0; k < K; k++) {
        modulus mk = mk_mod(ps[k]);
        /* floor(P/2) = (P-1)/2 since P is odd; mod p_k that is (p_k-1)/2 */
        u64 hk = mulmod(submod(0, 1, ps[k]), invmod(2, &mk), &mk);
        for (u64 t = 0; t < n; t++) v[k * n + t] = addmod(c[(nq + k) * n + t], hk, ps[k]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (i64 i = 0; i < (i64)nq; i++) {
        const u64 qi = moduli[i];
        modulus mi = mk_mod(qi);
        u64 pmod = 1 % qi;
        for (u64 k = 0; k < K; k++) pmod = mulmod(pmod, ps[k] % qi, &mi);
        const u64 hq = mulmod(submod(pmod, 1, qi), invmod(2, &mi), &mi); /* (P-1)/2 mod q_i */
        const u64 pinv = invmod(pmod, &mi);
        u64 *conv = (u64 *)malloc(n * sizeof(u64));
        base_convert(v, ps, K, qi, n, conv);
        for (u64 t = 0; t < n; t++)
            out[i * n + t] = mulmod(submod(addmod(c[i * n + t], hq, qi), conv[t], qi), pinv, &mi);
        free(conv);
    }
    free(v);
}

/* Hybrid SwitchKey (Section 2.4.1): the digits of d are its residues on the
   prime groups D_j = {q_{j*alpha}, ..., q_{j*alpha+alpha-1}} (cut at level l);
   each digit is lifted to Q_l*P by fast base conversion, the inner product
   with the key sum_j d~_j * swk_j is taken over Q_l*P, and the result is
   divided by P with rounding (ModDown).
   d: [l+1][n];  evk: [dnum_key][2][nQ+K][n] over q_0..q_{nQ-1}, p_0..p_{K-1};
   moduli/psis: nQ+K entries in that order;  out: [2][l+1][n]. */
void or_keyswitch(const u64 *d, u64 l, const u64 *evk, u64 dnum_key, u64 nQ, u64 K, u64 alpha,
                  const u64 *moduli, const u64 *psis, u64 n, u64 *out) {
    const u64 nl = l + 1, ntg = nl + K, dnum = (nl + alpha - 1) / alpha;
    if (dnum > dnum_key) return;
    u64 *tg_mod = (u64 *)malloc(ntg * sizeof(u64)), *tg_psi = (u64 *)malloc(ntg * sizeof(u64));
    u64 *tg_idx = (u64 *)malloc(ntg * sizeof(u64));
    for (u64 t = 0; t < ntg; t++) {
        tg_idx[t] = t < nl ? t : nQ + (t - nl);
        tg_mod[t] = moduli[tg_idx[t]];
        tg_psi[t] = psis[tg_idx[t]];
    }
    prepare_tables(tg_mod, tg_psi, ntg, n);
    u64 *acc = (u64 *)calloc(2 * ntg * n, sizeof(u64));
    for (u64 j = 0; j < dnum; j++) {
        const u64 lo = j * alpha, hi = (j + 1) * alpha < nl ? (j + 1) * alpha : nl;
#pragma omp parallel for schedule(dynamic, 1)
        for (i64 t = 0; t < (i64)ntg; t++) {
            const u64 p = tg_mod[t];
            const ntt_table *T = get_table(p, tg_psi[t], n);
            u64 *dt = (u64 *)malloc(n * sizeof(u64)), *prod = (u64 *)malloc(n * sizeof(u64));
            if ((u64)t >= lo && (u64)t < hi) memcpy(dt, d + t * n, n * sizeof(u64));
            else base_convert(d + lo * n, moduli + lo, hi - lo, p, n, dt);
            for (u64 c = 0; c < 2; c++) {
                const u64 *key = evk + ((j * 2 + c) * (nQ + K) + tg_idx[t]) * n;
                polymul_tab(dt, key, prod, T);
                u64 *a = acc + (c * ntg + t) * n;
                for (u64 k = 0; k < n; k++) a[k] = addmod(a[k], prod[k], p);
            }
            free(dt);
            free(prod);
        }
    }
    u64 *mods = (u64 *)malloc(ntg * sizeof(u64));
    for (u64 t = 0; t < ntg; t++) mods[t] = tg_mod[t];
    for (u64 c = 0; c < 2; c++) or_moddown(acc + c * ntg * n, nl, K, mods, n, out + c * nl * n);
    free(mods);
    free(acc);
    free(tg_mod);
    free(tg_psi);
    free(tg_idx);
}

int or_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
