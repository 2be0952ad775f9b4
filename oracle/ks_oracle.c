/*
 * ks_oracle.c -- plain CPU oracle for RNS hybrid key switching (HKS).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it (through oracle/oracle.py).  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Style: slow and obviously correct.  Every modular product is a 128-bit
 * product followed by the C `%` operator; no Shoup, Barrett, Montgomery or
 * lazy reduction; every value handed between steps is canonical in [0, m).
 *
 * What it follows (CiFlow, arxiv 2311.01598):
 *   - RNS representation of a ring element as one residue polynomial
 *     ("tower") per prime: Sec. II and Table I.
 *   - Digit decomposition into dnum digits of alpha towers: Sec. III-A,
 *     Table I (alpha = ceil((L+1)/dnum)).
 *   - ModUp P1 (iNTT), P2 (BConv alpha -> beta towers), P3 (NTT, digit
 *     towers bypassed), P4 (apply key), P5 (reduce over digits): Sec. III-B.
 *   - ModDown P1 (iNTT of the K special towers), P2 (BConv K -> l towers),
 *     P3 (NTT), P4 (subtract and scale by P^-1): Sec. III-C.
 * The paper gives these steps in prose only (it cites Han & Ki for the
 * algebra), so the formulas below are the standard hybrid key-switching
 * ones; readings where the paper is silent are listed at each function.
 *
 * Parity status: every exported function is pinned by tests that do not go
 * through this file's arithmetic (sympy primality, big-integer CRT identities,
 * schoolbook negacyclic products, published SplitMix64 vectors, decryption
 * noise bounds, the evk sizes of Table III).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Scalar modular arithmetic (m < 2^62 everywhere in this file).        */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * (u128)b) % m); }
static u64 addmod(u64 a, u64 b, u64 m) { return (a + b) % m; }
static u64 submod(u64 a, u64 b, u64 m) { return (a + (m - b)) % m; }
static u64 powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}
/* m prime: Fermat inverse. */
static u64 invmod(u64 a, u64 m) { return powmod(a % m, m - 2, m); }
/* Reduce a signed integer into [0, m). */
static u64 smod(i64 v, u64 m)
{
    i64 r = v % (i64)m;
    return (u64)(r < 0 ? r + (i64)m : r);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Primes and roots of unity (the paper fixes neither; reading R1/R2).  */
/* ------------------------------------------------------------------ */

/* Deterministic Miller-Rabin for 64-bit n (the first 12 prime bases are a
 * proven witness set below 3.3e24). */
int orc_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* The `count` largest primes q < 2^bits with q = 1 (mod 2N), descending.
 * Returns 0 on success, -1 if the progression runs out. */
int orc_gen_primes(int logN, int bits, int count, u64 *out)
{
    u64 step = (u64)2 << logN; /* 2N */
    u64 top = (bits >= 63) ? ((u64)1 << 63) : ((u64)1 << bits);
    u64 k = (top - 2) / step; /* largest k with 1 + k*2N < 2^bits */
    int got = 0;
    while (got < count) {
        if (k == 0) return -1;
        u64 c = 1 + k * step;
        if (orc_is_prime(c)) out[got++] = c;
        k--;
    }
    return 0;
}

/* psi = x^((q-1)/2N) for the smallest x >= 2 with psi^N = -1 (mod q):
 * a primitive 2N-th root of unity. */
u64 orc_find_psi(u64 q, int logN)
{
    u64 N = (u64)1 << logN;
    for (u64 x = 2; x < q; x++) {
        u64 psi = powmod(x, (q - 1) / (2 * N), q);
        if (powmod(psi, N, q) == q - 1) return psi;
    }
    return 0;
}

static u64 bitrev(u64 x, int bits)
{
    u64 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT.  Convention (reading R3): slot k holds the value of   */
/* the polynomial at psi^(2*brv(k)+1), brv = logN-bit reversal.          */
/* ------------------------------------------------------------------ */

/* Direct O(N^2) evaluation: the definition. */
void orc_ntt_naive(const u64 *a, u64 *out, int logN, u64 q, u64 psi)
{
    u64 N = (u64)1 << logN;
    for (u64 k = 0; k < N; k++) {
        u64 root = powmod(psi, 2 * bitrev(k, logN) + 1, q);
        u64 acc = 0, pw = 1;
        for (u64 i = 0; i < N; i++) {
            acc = addmod(acc, mulmod(a[i], pw, q), q);
            pw = mulmod(pw, root, q);
        }
        out[k] = acc;
    }
}

/* Direct O(N^2) inverse: a_i = N^-1 * sum_k ahat_k * root_k^-i. */
void orc_intt_naive(const u64 *ahat, u64 *out, int logN, u64 q, u64 psi)
{
    u64 N = (u64)1 << logN;
    u64 ninv = invmod(N, q);
    for (u64 i = 0; i < N; i++) out[i] = 0;
    for (u64 k = 0; k < N; k++) {
        u64 rinv = invmod(powmod(psi, 2 * bitrev(k, logN) + 1, q), q);
        u64 pw = 1;
        for (u64 i = 0; i < N; i++) {
            out[i] = addmod(out[i], mulmod(ahat[k], pw, q), q);
            pw = mulmod(pw, rinv, q);
        }
    }
    for (u64 i = 0; i < N; i++) out[i] = mulmod(out[i], ninv, q);
}

/* In-place radix-2 Cooley-Tukey NTT with psi powers in bit-reversed
 * order; produces the same slot order as orc_ntt_naive. */
void orc_ntt(u64 *a, int logN, u64 q, u64 psi)
{
    u64 N = (u64)1 << logN;
    u64 t = N;
    for (u64 m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (u64 i = 0; i < m; i++) {
            u64 w = powmod(psi, bitrev(m + i, logN), q);
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 u = a[j];
                u64 v = mulmod(a[j + t], w, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
    }
}

/* In-place Gentleman-Sande inverse of orc_ntt, including the N^-1 factor. */
void orc_intt(u64 *a, int logN, u64 q, u64 psi)
{
    u64 N = (u64)1 << logN;
    u64 psi_inv = invmod(psi, q);
    u64 t = 1;
    for (u64 m = N >> 1; m >= 1; m >>= 1) {
        for (u64 i = 0; i < m; i++) {
            u64 w = powmod(psi_inv, bitrev(m + i, logN), q);
            u64 j1 = 2 * i * t;
            for (u64 j = j1; j < j1 + t; j++) {
                u64 u = a[j];
                u64 v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), w, q);
            }
        }
        t <<= 1;
    }
    u64 ninv = invmod(N, q);
    for (u64 j = 0; j < N; j++) a[j] = mulmod(a[j], ninv, q);
}

/* ------------------------------------------------------------------ */
/* Fast base conversion (ModUp P2 / ModDown P2).                        */
/* ------------------------------------------------------------------ */

/* Fast base conversion without correction (reading R7): for source primes
 * s_0..s_{a-1} with product S and coefficient-form residues x_i, every
 * target prime r gets
 *     out_r = sum_i [x_i * (S/s_i)^-1]_{s_i} * (S/s_i)  mod r,
 * which equals (X + u*S) mod r for the CRT value X in [0,S) and one integer
 * u in [0, a) per coefficient.  x is [a][N], out is [b][N]. */
void orc_bconv(const u64 *src_primes, int a, const u64 *x, const u64 *dst_primes,
               int b, u64 *out, int logN)
{
    u64 N = (u64)1 << logN;
    u64 *y = (u64 *)malloc(sizeof(u64) * (size_t)a * N);
    for (int i = 0; i < a; i++) {
        u64 si = src_primes[i];
        u64 hat = 1; /* (S/s_i) mod s_i */
        for (int k = 0; k < a; k++)
            if (k != i) hat = mulmod(hat, src_primes[k] % si, si);
        u64 hinv = invmod(hat, si);
        for (u64 n = 0; n < N; n++) y[(size_t)i * N + n] = mulmod(x[(size_t)i * N + n], hinv, si);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < b; t++) {
        u64 r = dst_primes[t];
        u64 *o = out + (size_t)t * N;
        for (u64 n = 0; n < N; n++) o[n] = 0;
        for (int i = 0; i < a; i++) {
            u64 hat = 1; /* (S/s_i) mod r */
            for (int k = 0; k < a; k++)
                if (k != i) hat = mulmod(hat, src_primes[k] % r, r);
            for (u64 n = 0; n < N; n++)
                o[n] = addmod(o[n], mulmod(y[(size_t)i * N + n] % r, hat, r), r);
        }
    }
    free(y);
}

/* ------------------------------------------------------------------ */
/* Parameter context.                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    int logN;
    u64 N;
    int nq;    /* L+1 Q primes */
    int kp;    /* K special primes */
    int dnum;
    int alpha; /* ceil(nq/dnum) */
    int ndig;  /* ceil(nq/alpha): digits that hold at least one tower */
    u64 *q, *p, *psi_q, *psi_p;
} orc_ctx;

/* Prime rule (reading R1): the nq+kp largest primes below 2^bits that are
 * 1 mod 2N, in descending order; the first kp become P (p_0 largest), the
 * rest q_0, q_1, ...  Explicit primes may be passed instead. */
orc_ctx *orc_ctx_create(int logN, int nq, int kp, int dnum, int bits, const u64 *q_or_null,
                        const u64 *p_or_null)
{
    if (logN < 1 || logN > 20 || nq < 1 || kp < 1 || dnum < 1 || dnum > nq) return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->logN = logN;
    c->N = (u64)1 << logN;
    c->nq = nq;
    c->kp = kp;
    c->dnum = dnum;
    c->alpha = (nq + dnum - 1) / dnum;
    c->ndig = (nq + c->alpha - 1) / c->alpha;
    c->q = (u64 *)malloc(sizeof(u64) * nq);
    c->p = (u64 *)malloc(sizeof(u64) * kp);
    c->psi_q = (u64 *)malloc(sizeof(u64) * nq);
    c->psi_p = (u64 *)malloc(sizeof(u64) * kp);
    if (q_or_null && p_or_null) {
        memcpy(c->q, q_or_null, sizeof(u64) * nq);
        memcpy(c->p, p_or_null, sizeof(u64) * kp);
    } else {
        u64 *all = (u64 *)malloc(sizeof(u64) * (nq + kp));
        if (orc_gen_primes(logN, bits, nq + kp, all) != 0) {
            free(all);
            free(c->q); free(c->p); free(c->psi_q); free(c->psi_p); free(c);
            return NULL;
        }
        memcpy(c->p, all, sizeof(u64) * kp);
        memcpy(c->q, all + kp, sizeof(u64) * nq);
        free(all);
    }
    for (int i = 0; i < nq; i++) c->psi_q[i] = orc_find_psi(c->q[i], logN);
    for (int k = 0; k < kp; k++) c->psi_p[k] = orc_find_psi(c->p[k], logN);
    return c;
}

void orc_ctx_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->q); free(c->p); free(c->psi_q); free(c->psi_p);
    free(c);
}

void orc_ctx_primes(const orc_ctx *c, u64 *q_out, u64 *p_out, u64 *psiq_out, u64 *psip_out)
{
    if (q_out) memcpy(q_out, c->q, sizeof(u64) * c->nq);
    if (p_out) memcpy(p_out, c->p, sizeof(u64) * c->kp);
    if (psiq_out) memcpy(psiq_out, c->psi_q, sizeof(u64) * c->nq);
    if (psip_out) memcpy(psip_out, c->psi_p, sizeof(u64) * c->kp);
}
int orc_ctx_alpha(const orc_ctx *c) { return c->alpha; }
int orc_ctx_ndig(const orc_ctx *c) { return c->ndig; }

/* Tower t of the level-l extended basis D_l = {q_0..q_{nact-1}} u {p_0..p_{K-1}},
 * compact order (Q first, then P). */
static u64 tower_prime(const orc_ctx *c, int nact, int t)
{
    return t < nact ? c->q[t] : c->p[t - nact];
}
static u64 tower_psi(const orc_ctx *c, int nact, int t)
{
    return t < nact ? c->psi_q[t] : c->psi_p[t - nact];
}
/* Index of compact tower t inside the full-level evaluation-key layout. */
static int tower_full_index(const orc_ctx *c, int nact, int t)
{
    return t < nact ? t : c->nq + (t - nact);
}

/* ------------------------------------------------------------------ */
/* ModUp (Sec. III-B, stages P1-P3).                                    */
/* ------------------------------------------------------------------ */

/* Digit j at level nact covers Q towers [j*alpha, min((j+1)*alpha, nact))
 * (reading R8: the last active digit may be short; digits past nact are
 * inactive).  Returns the number of active digits. */
int orc_active_digits(const orc_ctx *c, int nact)
{
    return (nact + c->alpha - 1) / c->alpha;
}

/* d: [nact][N] evaluation form.  Dout: [ndig_act][nact+K][N] evaluation
 * form over D_l, where row j is digit j raised to the whole basis:
 *   P1  x_i = iNTT_{q_i}(d_i) for the digit's towers,
 *   P2  fast base conversion of x (over the digit's active primes) to every
 *       tower outside the digit,
 *   P3  NTT of the converted towers; the digit's own towers are the input
 *       towers themselves (bypass). */
void orc_modup(const orc_ctx *c, int nact, const u64 *d, u64 *Dout)
{
    u64 N = c->N;
    int nd = orc_active_digits(c, nact);
    int nt = nact + c->kp;
    for (int j = 0; j < nd; j++) {
        int lo = j * c->alpha;
        int hi = lo + c->alpha < nact ? lo + c->alpha : nact;
        int a = hi - lo;
        u64 *x = (u64 *)malloc(sizeof(u64) * (size_t)a * N);
        u64 *src = (u64 *)malloc(sizeof(u64) * a);
        for (int i = 0; i < a; i++) {
            src[i] = c->q[lo + i];
            memcpy(x + (size_t)i * N, d + (size_t)(lo + i) * N, sizeof(u64) * N);
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < a; i++) orc_intt(x + (size_t)i * N, c->logN, c->q[lo + i], c->psi_q[lo + i]);
        int b = nt - a;
        u64 *dst = (u64 *)malloc(sizeof(u64) * b);
        int *dst_t = (int *)malloc(sizeof(int) * b);
        int nb = 0;
        for (int t = 0; t < nt; t++) {
            if (t >= lo && t < hi) continue;
            dst[nb] = tower_prime(c, nact, t);
            dst_t[nb] = t;
            nb++;
        }
        u64 *z = (u64 *)malloc(sizeof(u64) * (size_t)b * N);
        orc_bconv(src, a, x, dst, b, z, c->logN);
        u64 *row = Dout + (size_t)j * nt * N;
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < b; k++) {
            int t = dst_t[k];
            orc_ntt(z + (size_t)k * N, c->logN, dst[k], tower_psi(c, nact, t));
            memcpy(row + (size_t)t * N, z + (size_t)k * N, sizeof(u64) * N);
        }
        for (int t = lo; t < hi; t++) memcpy(row + (size_t)t * N, d + (size_t)t * N, sizeof(u64) * N);
        free(x); free(src); free(dst); free(dst_t); free(z);
    }
}

/* ModUp P4 + P5: c'_{x,t} = sum_j D_{j,t} * evk_{j,x,t} for x in {b, a}.
 * evk: [ndig][2][nq+kp][N] (full level, evaluation form); only the towers of
 * D_l are read.  cb, ca: [nact+K][N]. */
void orc_apply_key(const orc_ctx *c, int nact, const u64 *D, const u64 *evk, u64 *cb, u64 *ca)
{
    u64 N = c->N;
    int nd = orc_active_digits(c, nact);
    int nt = nact + c->kp;
    int nfull = c->nq + c->kp;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nt; t++) {
        u64 r = tower_prime(c, nact, t);
        int tf = tower_full_index(c, nact, t);
        for (u64 n = 0; n < N; n++) {
            u64 sb = 0, sa = 0;
            for (int j = 0; j < nd; j++) {
                u64 dv = D[((size_t)j * nt + t) * N + n];
                u64 kb = evk[(((size_t)j * 2 + 0) * nfull + tf) * N + n];
                u64 ka = evk[(((size_t)j * 2 + 1) * nfull + tf) * N + n];
                sb = addmod(sb, mulmod(dv, kb, r), r);
                sa = addmod(sa, mulmod(dv, ka, r), r);
            }
            cb[(size_t)t * N + n] = sb;
            ca[(size_t)t * N + n] = sa;
        }
    }
}

/* ------------------------------------------------------------------ */
/* ModDown (Sec. III-C): cp [nact+K][N] evaluation form -> out [nact][N]. */
/*   P1 w = iNTT of the K special towers,                                */
/*   P2 v = fast base conversion of w from P to each q_i,                */
/*   P3 NTT_{q_i}(v_i),                                                   */
/*   P4 out_i = (cp_i - NTT(v_i)) * P^-1 mod q_i.                         */
/* ------------------------------------------------------------------ */
void orc_moddown(const orc_ctx *c, int nact, const u64 *cp, u64 *out)
{
    u64 N = c->N;
    int K = c->kp;
    u64 *w = (u64 *)malloc(sizeof(u64) * (size_t)K * N);
    memcpy(w, cp + (size_t)nact * N, sizeof(u64) * (size_t)K * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; k++) orc_intt(w + (size_t)k * N, c->logN, c->p[k], c->psi_p[k]);
    u64 *v = (u64 *)malloc(sizeof(u64) * (size_t)nact * N);
    orc_bconv(c->p, K, w, c->q, nact, v, c->logN);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < nact; i++) {
        u64 q = c->q[i];
        u64 *vi = v + (size_t)i * N;
        orc_ntt(vi, c->logN, q, c->psi_q[i]);
        u64 pm = 1;
        for (int k = 0; k < K; k++) pm = mulmod(pm, c->p[k] % q, q);
        u64 pinv = invmod(pm, q);
        for (u64 n = 0; n < N; n++)
            out[(size_t)i * N + n] = mulmod(submod(cp[(size_t)i * N + n], vi[n], q), pinv, q);
    }
    free(w);
    free(v);
}

/* Whole key switch at level nact (nact = l+1 active Q towers):
 * d [nact][N] evaluation form under s', evk [ndig][2][nq+kp][N]
 * -> (out0, out1) [nact][N] with out0 + out1*s ~ d*s' (mod Q_l). */
void orc_keyswitch(const orc_ctx *c, int nact, const u64 *d, const u64 *evk, u64 *out0, u64 *out1)
{
    u64 N = c->N;
    int nd = orc_active_digits(c, nact);
    int nt = nact + c->kp;
    u64 *D = (u64 *)malloc(sizeof(u64) * (size_t)nd * nt * N);
    u64 *cb = (u64 *)malloc(sizeof(u64) * (size_t)nt * N);
    u64 *ca = (u64 *)malloc(sizeof(u64) * (size_t)nt * N);
    orc_modup(c, nact, d, D);
    orc_apply_key(c, nact, D, evk, cb, ca);
    orc_moddown(c, nact, cb, out0);
    orc_moddown(c, nact, ca, out1);
    free(D); free(cb); free(ca);
}

/* ------------------------------------------------------------------ */
/* Rotations with hoisting (Sec. II: every rotation needs the key switch */
/* of a Galois automorphism; hoisting shares one ModUp among them).     */
/* ------------------------------------------------------------------ */

/* X -> X^g on an evaluation-form tower.  Slot k holds a(psi^e_k) with
 * e_k = 2 brv(k) + 1; a(X^g) there equals a at psi^(e_k g mod 2N), i.e. the
 * slot k' with e_k' = e_k g mod 2N: a permutation of slots (g odd). */
void orc_automorph_eval(const u64 *in, u64 *out, int logN, u64 g)
{
    u64 N = 1ull << logN, two_n = 2 * N;
    u64 gg = g % two_n;
    for (u64 k = 0; k < N; k++) {
        u64 e = ((2 * bitrev(k, logN) + 1) * gg) % two_n;
        out[k] = in[bitrev((e - 1) / 2, logN)];
    }
}

/* Hoisted key switches of nrot rotations of one polynomial d (evaluation
 * form, nact towers): the digits are raised once, D_j = ModUp_j(d); for
 * rotation r every raised tower is mapped by X -> X^g_r and switched with
 * key r:  out_r = ModDown(sum_j phi_r(D_j) * evk_r,j).  evks:
 * [nrot][ndig][2][nq+kp][N]; out0, out1: [nrot][nact][N].  With g_r = 1 this
 * is orc_keyswitch. */
void orc_keyswitch_hoisted(const orc_ctx *c, int nact, const u64 *d, int nrot, const u64 *evks, const u64 *gal,
                           u64 *out0, u64 *out1)
{
    u64 N = c->N;
    int nd = orc_active_digits(c, nact);
    int nt = nact + c->kp;
    size_t key_words = (size_t)c->ndig * 2 * (c->nq + c->kp) * N;
    u64 *D = (u64 *)malloc(sizeof(u64) * (size_t)nd * nt * N);
    u64 *Dg = (u64 *)malloc(sizeof(u64) * (size_t)nd * nt * N);
    u64 *cb = (u64 *)malloc(sizeof(u64) * (size_t)nt * N);
    u64 *ca = (u64 *)malloc(sizeof(u64) * (size_t)nt * N);
    orc_modup(c, nact, d, D);
    for (int r = 0; r < nrot; r++) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int l = 0; l < nd * nt; l++) orc_automorph_eval(D + (size_t)l * N, Dg + (size_t)l * N, c->logN, gal[r]);
        orc_apply_key(c, nact, Dg, evks + (size_t)r * key_words, cb, ca);
        orc_moddown(c, nact, cb, out0 + (size_t)r * nact * N);
        orc_moddown(c, nact, ca, out1 + (size_t)r * nact * N);
    }
    free(D); free(Dg); free(cb); free(ca);
}

/* ------------------------------------------------------------------ */
/* Key generation (the paper is silent on sampling; reading R9).        */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a Weyl sequence with
 * increment 0x9E3779B97F4A7C15 passed through a 64-bit finaliser. */
typedef struct { u64 s; } orc_rng;
static u64 orc_rng_next(orc_rng *g)
{
    g->s += 0x9E3779B97F4A7C15ULL;
    u64 z = g->s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
void orc_splitmix64(u64 seed, int n, u64 *out)
{
    orc_rng g = {seed};
    for (int i = 0; i < n; i++) out[i] = orc_rng_next(&g);
}

static int bitlen(u64 x)
{
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}
/* Uniform in [0, m): rejection of a 64-bit draw masked to bitlen(m). */
static u64 orc_uniform(orc_rng *g, u64 m)
{
    int b = bitlen(m);
    u64 mask = b >= 64 ? ~(u64)0 : (((u64)1 << b) - 1);
    for (;;) {
        u64 v = orc_rng_next(g) & mask;
        if (v < m) return v;
    }
}
/* Rounded Gaussian, sigma 3.2, by Box-Muller from two 53-bit draws,
 * rounded half away from zero, redrawn while |e| > 19. */
static i64 orc_gauss(orc_rng *g)
{
    const double sigma = 3.2;
    for (;;) {
        double u1 = (double)((orc_rng_next(g) >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(orc_rng_next(g) >> 11) * 0x1.0p-53;
        double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
        i64 e = (i64)llround(sigma * z);
        if (e >= -19 && e <= 19) return e;
    }
}
void orc_sample_gauss(u64 seed, int n, i64 *out)
{
    orc_rng g = {seed};
    for (int i = 0; i < n; i++) out[i] = orc_gauss(&g);
}

/* Evaluation key for switching from s' to s (Han & Ki hybrid key):
 *   b_j = -a_j * s + e_j + [P * g_j] * s'   (evaluation form, per tower),
 * g_j the CRT idempotent of digit j: [P*g_j]_{q_i} = [P]_{q_i} if q_i is in
 * digit j of the full level, 0 otherwise; 0 on the P towers.
 * Draw order: stream seed^0 gives a_j for j, then tower in D_L order, then
 * coefficient; stream seed^1 gives e_j (one integer polynomial per digit).
 * s: [N] in {-1,0,1}; sp: [N] signed coefficients of s'.
 * evk_out: [ndig][2][nq+kp][N] with index 0 = b, 1 = a. */
/* b_j = -a_j*s + e_j + [P g_j] s' on every tower, given a_j in the a-slots
 * of evk_out and e_j drawn from stream seed^1 (digit, then coefficient). */
static void keygen_b(const orc_ctx *c, const int8_t *s, const i64 *sp, u64 seed, u64 *evk_out)
{
    u64 N = c->N;
    int nfull = c->nq + c->kp;
    int nd = c->ndig;
    orc_rng ge = {seed ^ 1};
    i64 *e = (i64 *)malloc(sizeof(i64) * (size_t)nd * N);
    for (int j = 0; j < nd; j++)
        for (u64 n = 0; n < N; n++) e[(size_t)j * N + n] = orc_gauss(&ge);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nfull; t++) {
        u64 r = tower_prime(c, c->nq, t);
        u64 psi = tower_psi(c, c->nq, t);
        u64 *sh = (u64 *)malloc(sizeof(u64) * N);
        u64 *sph = (u64 *)malloc(sizeof(u64) * N);
        u64 *eh = (u64 *)malloc(sizeof(u64) * N);
        for (u64 n = 0; n < N; n++) {
            sh[n] = smod(s[n], r);
            sph[n] = smod(sp[n], r);
        }
        orc_ntt(sh, c->logN, r, psi);
        orc_ntt(sph, c->logN, r, psi);
        u64 pm = 1;
        for (int k = 0; k < c->kp; k++) pm = mulmod(pm, c->p[k] % r, r);
        for (int j = 0; j < nd; j++) {
            for (u64 n = 0; n < N; n++) eh[n] = smod(e[(size_t)j * N + n], r);
            orc_ntt(eh, c->logN, r, psi);
            int in_digit = (t < c->nq) && (t / c->alpha == j);
            u64 g = in_digit ? pm : 0;
            const u64 *a = evk_out + (((size_t)j * 2 + 1) * nfull + t) * N;
            u64 *b = evk_out + (((size_t)j * 2 + 0) * nfull + t) * N;
            for (u64 n = 0; n < N; n++) {
                u64 v = submod(eh[n], mulmod(a[n], sh[n], r), r);
                b[n] = addmod(v, mulmod(g, sph[n], r), r);
            }
        }
        free(sh); free(sph); free(eh);
    }
    free(e);
}

/* Evaluation key for switching from s' to s (Han & Ki hybrid key):
 *   b_j = -a_j * s + e_j + [P * g_j] * s'   (evaluation form, per tower),
 * g_j the CRT idempotent of digit j: [P*g_j]_{q_i} = [P]_{q_i} if q_i is in
 * digit j of the full level, 0 otherwise; 0 on the P towers.
 * Draw order: stream seed^0 gives a_j for j, then tower in D_L order, then
 * coefficient; stream seed^1 gives e_j (one integer polynomial per digit).
 * s: [N] in {-1,0,1}; sp: [N] signed coefficients of s'.
 * evk_out: [ndig][2][nq+kp][N] with index 0 = b, 1 = a. */
void orc_keygen(const orc_ctx *c, const int8_t *s, const i64 *sp, u64 seed, u64 *evk_out)
{
    u64 N = c->N;
    int nfull = c->nq + c->kp;
    orc_rng ga = {seed ^ 0};
    /* a_j, drawn straight into the a-slot */
    for (int j = 0; j < c->ndig; j++)
        for (int t = 0; t < nfull; t++) {
            u64 r = tower_prime(c, c->nq, t);
            u64 *dst = evk_out + (((size_t)j * 2 + 1) * nfull + t) * N;
            for (u64 n = 0; n < N; n++) dst[n] = orc_uniform(&ga, r);
        }
    keygen_b(c, s, sp, seed, evk_out);
}

/* Compressed keys (Sec. IV-D: regenerating the key's uniform half from a
 * seed halves the key's data movement; the sampling is reading R16).
 * SplitMix64's state after k outputs is seed + k*0x9E3779B97F4A7C15, so
 * output number c+1 of the stream is reached directly:
 *   SM(x, c) = finaliser(x + (c+1)*0x9E3779B97F4A7C15).
 * a_j at full tower t (q_0..q_L, p_0..p_{K-1}), slot n: the first of the
 * draws v_m = SM(seed^2, ((j*nfull + t)*N + n)*64 + m) & mask(bitlen(r)),
 * m = 0..63, with v_m < r; if all 64 reject (probability below 2^-64 for
 * primes above 2^(bits-1)) the last one reduced mod r. */
static u64 splitmix_at(u64 x, u64 c)
{
    orc_rng g = {x + c * 0x9E3779B97F4A7C15ULL};
    return orc_rng_next(&g);
}
u64 orc_key_a_word(u64 seed, int j, int t, u64 n, int logN, int nfull, u64 r)
{
    int b = bitlen(r);
    u64 mask = b >= 64 ? ~(u64)0 : (((u64)1 << b) - 1);
    u64 base = (((u64)j * (u64)nfull + (u64)t) * ((u64)1 << logN) + n) * 64;
    u64 v = 0;
    for (int m = 0; m < 64; m++) {
        v = splitmix_at(seed ^ 2, base + (u64)m) & mask;
        if (v < r) return v;
    }
    return v % r;
}
/* The full evaluation key of a compressed key: a_j regenerated as above,
 * e_j and b_j as orc_keygen.  Same layout as orc_keygen. */
void orc_keygen_compressed(const orc_ctx *c, const int8_t *s, const i64 *sp, u64 seed, u64 *evk_out)
{
    u64 N = c->N;
    int nfull = c->nq + c->kp;
    for (int j = 0; j < c->ndig; j++)
#pragma omp parallel for schedule(dynamic, 1)
        for (int t = 0; t < nfull; t++) {
            u64 r = tower_prime(c, c->nq, t);
            u64 *dst = evk_out + (((size_t)j * 2 + 1) * nfull + t) * N;
            for (u64 n = 0; n < N; n++) dst[n] = orc_key_a_word(seed, j, t, n, c->logN, nfull, r);
        }
    keygen_b(c, s, sp, seed, evk_out);
}

/* Negacyclic schoolbook product mod q (a*b mod X^N+1): pins the NTT. */
void orc_negacyclic_mul(const u64 *a, const u64 *b, u64 *out, int logN, u64 q)
{
    u64 N = (u64)1 << logN;
    for (u64 k = 0; k < N; k++) out[k] = 0;
    for (u64 i = 0; i < N; i++)
        for (u64 j = 0; j < N; j++) {
            u64 v = mulmod(a[i], b[j], q);
            u64 k = i + j;
            if (k < N) out[k] = addmod(out[k], v, q);
            else out[k - N] = submod(out[k - N], v, q);
        }
}
