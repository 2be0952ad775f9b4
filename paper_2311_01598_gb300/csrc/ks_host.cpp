// ks_host.cpp -- host-side number theory and table construction.
//
// Primes (rule fixed by the library, the paper does not give one): the
// n_q + k_p largest primes below 2^bits that are 1 mod 2N, descending; the
// first k_p become p_0.., the rest q_0, q_1, ...  psi is x^((q-1)/2N) for the
// smallest x >= 2 whose power is a primitive 2N-th root (psi^N = -1).
#include <algorithm>
#include <cstring>

#include "ks_internal.h"
#include "ks_launch.h"

namespace ks {

typedef unsigned __int128 u128;

u64 mulmod_h(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }

u64 powmod_h(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod_h(r, b, m);
        b = mulmod_h(b, b, m);
        e >>= 1;
    }
    return r;
}

u64 invmod_h(u64 a, u64 m) { return powmod_h(a % m, m - 2, m); }

u64 shoup_h(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Miller-Rabin with the first twelve primes as bases: deterministic for
// every 64-bit input (Sorenson & Webster bound 3.3e24).
bool is_prime_u64(u64 n)
{
    static const u64 a[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : a) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    for (u64 b : a) {
        u64 x = powmod_h(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s && composite; ++r) {
            x = mulmod_h(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

// The count largest primes below 2^bits of the form k*2^32 + 1, descending
// (each is 1 mod 2N for every supported N).
int gen_special_primes(int bits, int count, std::vector<u64> &out)
{
    out.clear();
    if (bits <= 32) return -1;
    u64 k = (((u64)1 << bits) - 2) >> 32;
    while ((int)out.size() < count && k > 0) {
        const u64 c = (k << 32) + 1;
        if (is_prime_u64(c)) out.push_back(c);
        --k;
    }
    return (int)out.size() == count ? 0 : -1;
}

int gen_primes(int logN, int bits, int count, std::vector<u64> &out)
{
    out.clear();
    const u64 step = (u64)2 << logN;
    u64 k = (((u64)1 << bits) - 2) / step;
    while ((int)out.size() < count && k > 0) {
        u64 c = 1 + k * step;
        if (is_prime_u64(c)) out.push_back(c);
        --k;
    }
    return (int)out.size() == count ? 0 : -1;
}

u64 find_psi(u64 q, int logN)
{
    const u64 N = (u64)1 << logN;
    for (u64 x = 2; x < q; ++x) {
        u64 psi = powmod_h(x, (q - 1) / (2 * N), q);
        if (powmod_h(psi, N, q) == q - 1) return psi;
    }
    return 0;
}

static u64 brv(u64 x, int bits)
{
    u64 r = 0;
    for (int i = 0; i < bits; ++i) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

static u64 split28(u64 c) { return (c & ((1ull << kSplit) - 1)) | ((c >> kSplit) << 32); }

// c * 2^64 mod r: base-conversion constants are stored in Montgomery form, so
// one Montgomery reduction of the 128-bit sum of products yields the sum mod r.
static u64 to_mont(u64 c, u64 r) { return (u64)((((unsigned __int128)c) << 64) % r); }

static ulonglong2 shoup_pair(u64 w, u64 q)
{
    ulonglong2 r;
    r.x = w;
    r.y = shoup_h(w, q);
    return r;
}

template <class T>
static int upload(T **dst, const std::vector<T> &src)
{
    if (src.empty()) {
        *dst = nullptr;
        return KS_OK;
    }
    if (cudaMalloc((void **)dst, sizeof(T) * src.size()) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return fail(KS_ENOMEM, "cudaMalloc failed for a parameter table");
    }
    if (cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaMemcpy of a parameter table failed");
    }
    return KS_OK;
}

int build_tables(ks_params *P)
{
    const int nt = P->nq + P->kp;
    const u64 N = P->N;
    std::vector<u64> prim(nt);
    for (int i = 0; i < P->nq; ++i) prim[i] = P->q[i];
    for (int k = 0; k < P->kp; ++k) prim[P->nq + k] = P->p[k];
    P->psi.resize(nt);
    for (int t = 0; t < nt; ++t) {
        P->psi[t] = find_psi(prim[t], P->logN);
        if (!P->psi[t]) return fail(KS_EINVAL, "no primitive 2N-th root for a prime");
    }

    // per-tower constants
    std::vector<ModC> modc(nt);
    for (int t = 0; t < nt; ++t) {
        u64 q = prim[t];
        ModC &m = modc[t];
        m.q = q;
        m.q2 = 2 * q;
        u64 x = q;  // Newton iteration for q^-1 mod 2^64
        for (int i = 0; i < 6; ++i) x *= 2 - q * x;
        m.mont = (u64)0 - x;
        m.one_sh = shoup_h(1, q);
        m.r28 = ((u64)1 << 28) % q;
        m.r28_sh = shoup_h(m.r28, q);
        m.r56 = ((u64)1 << 56) % q;
        m.r56_sh = shoup_h(m.r56, q);
        m.ninv = invmod_h(N % q, q);
        m.ninv_sh = shoup_h(m.ninv, q);
        u64 r64 = (u64)((((u128)1) << 64) % q);
        m.r2 = mulmod_h(r64, r64, q);
        m.pad = 0;
    }

    // twiddles
    std::vector<ulonglong2> tw((size_t)nt * N), itw((size_t)nt * N);
    std::vector<u64> pw(N), ipw(N);
    for (int t = 0; t < nt; ++t) {
        u64 q = prim[t], psi = P->psi[t], psii = invmod_h(psi, q);
        pw[0] = 1;
        ipw[0] = 1;
        for (u64 e = 1; e < N; ++e) {
            pw[e] = mulmod_h(pw[e - 1], psi, q);
            ipw[e] = mulmod_h(ipw[e - 1], psii, q);
        }
        for (u64 i = 0; i < N; ++i) {
            u64 r = brv(i, P->logN);
            tw[(size_t)t * N + i] = shoup_pair(pw[r], q);
            itw[(size_t)t * N + i] = shoup_pair(ipw[r], q);
        }
    }

    // ModUp tables per (digit j, active towers a)
    const int A = P->alpha;
    std::vector<ulonglong2> pre;
    std::vector<u64> mat;
    P->up_off.pre.assign((size_t)P->ndig * (A + 1), -1);
    P->up_off.mat.assign((size_t)P->ndig * (A + 1), -1);
    for (int j = 0; j < P->ndig; ++j) {
        int lo = j * A;
        int full = std::min(A, P->nq - lo);
        for (int a = 1; a <= full; ++a) {
            P->up_off.pre[j * (A + 1) + a] = (int)pre.size();
            P->up_off.mat[j * (A + 1) + a] = (int)mat.size();
            for (int i = 0; i < a; ++i) {
                u64 qi = prim[lo + i];
                u64 hat = 1;
                for (int k = 0; k < a; ++k)
                    if (k != i) hat = mulmod_h(hat, prim[lo + k] % qi, qi);
                u64 s = mulmod_h(invmod_h(N % qi, qi), invmod_h(hat, qi), qi);
                pre.push_back(shoup_pair(s, qi));
            }
            for (int i = 0; i < a; ++i)
                for (int t = 0; t < nt; ++t) {
                    u64 r = prim[t];
                    u64 hat = 1;
                    for (int k = 0; k < a; ++k)
                        if (k != i) hat = mulmod_h(hat, prim[lo + k] % r, r);
                    mat.push_back(split28(to_mont(hat, r)));
                }
        }
    }

    // the same P1 factors laid out per level: row nact-1 holds towers 0..nact-1
    std::vector<ulonglong2> pre_lvl((size_t)P->nq * P->nq);
    for (int nact = 1; nact <= P->nq; ++nact)
        for (int i = 0; i < nact; ++i) {
            int j = i / A, lo = j * A;
            int a = std::min(A, nact - lo);
            pre_lvl[(size_t)(nact - 1) * P->nq + i] = pre[P->up_off.pre[j * (A + 1) + a] + (i - lo)];
        }

    // ModUp matrix offset of each active digit, per level
    std::vector<int> mat_lvl((size_t)P->nq * P->ndig, 0);
    for (int nact = 1; nact <= P->nq; ++nact)
        for (int j = 0; j * A < nact; ++j) {
            int a = std::min(A, nact - j * A);
            mat_lvl[(size_t)(nact - 1) * P->ndig + j] = P->up_off.mat[j * (A + 1) + a];
        }

    // ModDown matrix: (P/p_k) * P^-1 = p_k^-1 mod q_i
    std::vector<u64> dn((size_t)P->kp * P->nq);
    for (int k = 0; k < P->kp; ++k)
        for (int i = 0; i < P->nq; ++i)
            dn[(size_t)k * P->nq + i] = split28(to_mont(invmod_h(P->p[k] % P->q[i], P->q[i]), P->q[i]));

    // tensor-core base conversion: one B slab per (digit j, active towers a,
    // full tower t) for ModUp and per Q tower for ModDown (<= 18 sources; one
    // K block of 64 slice columns up to 9, two up to 18)
    std::vector<uint16_t> up_tc, dn_tc;
    std::vector<int> up_tc_lvl((size_t)P->nq * P->ndig, 0);
    const int kb_up = tc_kblocks(A), kb_dn = tc_kblocks(P->kp);
    int below54 = 1;
    for (u64 q : P->q) below54 = below54 && q < (1ull << 54);
    for (u64 p : P->p) below54 = below54 && p < (1ull << 54);
    const int bits_up = tc_slice_bits(kb_up, below54), bits_dn = tc_slice_bits(kb_dn, below54);
    const size_t SLAB = (size_t)kTcSlabHalves * kb_up, DSLAB = (size_t)kTcSlabHalves * kb_dn;
    if (A <= 18) {
        std::vector<int> off((size_t)P->ndig * (A + 1), -1);
        for (int j = 0; j < P->ndig; ++j) {
            int lo = j * A;
            int full = std::min(A, P->nq - lo);
            for (int a = 1; a <= full; ++a) {
                off[j * (A + 1) + a] = (int)(up_tc.size() / SLAB);
                for (int t = 0; t < nt; ++t) {
                    u64 r = prim[t];
                    std::vector<u64> c(a);
                    for (int i = 0; i < a; ++i) {
                        u64 hat = 1;
                        for (int k = 0; k < a; ++k)
                            if (k != i) hat = mulmod_h(hat, prim[lo + k] % r, r);
                        c[i] = to_mont(hat, r);
                    }
                    up_tc.resize(up_tc.size() + SLAB);
                    tc_slab(c, r, kb_up, bits_up, up_tc.data() + up_tc.size() - SLAB);
                }
            }
        }
        for (int nact = 1; nact <= P->nq; ++nact)
            for (int j = 0; j * A < nact; ++j)
                up_tc_lvl[(size_t)(nact - 1) * P->ndig + j] = off[j * (A + 1) + std::min(A, nact - j * A)];
    }
    if (P->kp <= 18) {
        dn_tc.resize((size_t)P->nq * DSLAB);
        for (int i = 0; i < P->nq; ++i) {
            std::vector<u64> c(P->kp);
            for (int k = 0; k < P->kp; ++k) c[k] = to_mont(invmod_h(P->p[k] % P->q[i], P->q[i]), P->q[i]);
            tc_slab(c, P->q[i], kb_dn, bits_dn, dn_tc.data() + (size_t)i * DSLAB);
        }
    }

    // factors folded into the stored key
    std::vector<ulonglong2> ksc(nt), psc(nt);
    for (int t = 0; t < nt; ++t) {
        u64 r = prim[t];
        u64 f;
        if (t < P->nq) {
            u64 pm = 1;
            for (int k = 0; k < P->kp; ++k) pm = mulmod_h(pm, P->p[k] % r, r);
            f = invmod_h(pm, r);
        } else {
            int kk = t - P->nq;
            u64 hat = 1;
            for (int k = 0; k < P->kp; ++k)
                if (k != kk) hat = mulmod_h(hat, P->p[k] % r, r);
            f = mulmod_h(invmod_h(N % r, r), invmod_h(hat, r), r);
        }
        psc[t] = shoup_pair(f, r);
        u64 fm = (u64)((((u128)f) << 64) % r);
        ksc[t] = shoup_pair(fm, r);
    }

    int rc;
    if ((rc = upload(&P->d_modc, modc)) != KS_OK) return rc;
    if ((rc = upload(&P->d_tw, tw)) != KS_OK) return rc;
    if ((rc = upload(&P->d_itw, itw)) != KS_OK) return rc;
    if ((rc = upload(&P->d_up_pre, pre)) != KS_OK) return rc;
    if ((rc = upload(&P->d_up_pre_lvl, pre_lvl)) != KS_OK) return rc;
    if ((rc = upload(&P->d_up_mat_lvl, mat_lvl)) != KS_OK) return rc;
    if ((rc = upload(&P->d_up_mat, mat)) != KS_OK) return rc;
    if ((rc = upload(&P->d_dn_mat, dn)) != KS_OK) return rc;
    if ((rc = upload(&P->d_key_sc, ksc)) != KS_OK) return rc;
    if ((rc = upload(&P->d_plain_sc, psc)) != KS_OK) return rc;
    if (!up_tc.empty()) {
        uint16_t *d = nullptr;
        if ((rc = upload(&d, up_tc)) != KS_OK) return rc;
        P->d_up_tc = reinterpret_cast<uint4 *>(d);  // 256-byte aligned allocation
        if ((rc = upload(&P->d_up_tc_lvl, up_tc_lvl)) != KS_OK) return rc;
    }
    if (!dn_tc.empty()) {
        uint16_t *d = nullptr;
        if ((rc = upload(&d, dn_tc)) != KS_OK) return rc;
        P->d_dn_tc = reinterpret_cast<uint4 *>(d);
    }

    Tables &T = P->tables;
    T.modc = P->d_modc;
    T.tw = P->d_tw;
    T.itw = P->d_itw;
    T.up_pre = P->d_up_pre;
    T.up_mat = P->d_up_mat;
    T.dn_mat = P->d_dn_mat;
    T.key_sc = P->d_key_sc;
    T.plain_sc = P->d_plain_sc;
    T.up_mat_lvl = P->d_up_mat_lvl;
    T.up_tc = P->bconv_tensor ? P->d_up_tc : nullptr;
    T.up_tc_lvl = P->d_up_tc_lvl;
    T.dn_tc = P->bconv_tensor ? P->d_dn_tc : nullptr;
    T.ntt_cluster = P->ntt_cluster;
    T.row_stage = P->row_stage;
    T.tc_below54 = 1;
    for (u64 q : P->q) T.tc_below54 = T.tc_below54 && q < (1ull << 54);
    for (u64 p : P->p) T.tc_below54 = T.tc_below54 && p < (1ull << 54);
    T.spq = 1;
    for (u64 q : P->q) T.spq = T.spq && (q & 0xFFFFFFFFull) == 1;
    for (u64 p : P->p) T.spq = T.spq && (p & 0xFFFFFFFFull) == 1;
    T.logN = P->logN;
    T.nq = P->nq;
    T.kp = P->kp;
    T.alpha = P->alpha;
    T.ndig = P->ndig;
    return KS_OK;
}

void free_tables(ks_params *P)
{
    void *ptrs[] = {P->d_modc,   P->d_tw,     P->d_itw,    P->d_up_pre,   P->d_up_pre_lvl, P->d_up_mat,
                    P->d_dn_mat, P->d_key_sc, P->d_plain_sc, P->d_up_mat_lvl, P->d_up_tc,      P->d_up_tc_lvl,
                    P->d_dn_tc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    P->d_modc = nullptr;
    P->d_tw = P->d_itw = P->d_up_pre = P->d_up_pre_lvl = P->d_key_sc = P->d_plain_sc = nullptr;
    P->d_up_mat = P->d_dn_mat = nullptr;
    P->d_up_mat_lvl = nullptr;
    P->d_up_tc = P->d_dn_tc = nullptr;
    P->d_up_tc_lvl = nullptr;
}

}  // namespace ks

extern "C" int ks_special_primes(uint32_t bits, uint32_t count, uint64_t *h_out)
{
    if (!h_out || count == 0) return ks::fail(KS_EINVAL, "ks_special_primes: NULL output or count 0");
    if (bits < 33 || bits > (uint32_t)ks::kMaxPrimeBits) return ks::fail(KS_EINVAL, "ks_special_primes: bits must be in 33..56");
    std::vector<ks::u64> v;
    if (ks::gen_special_primes((int)bits, (int)count, v) != 0)
        return ks::fail(KS_EINVAL, "ks_special_primes: not enough primes of the form k*2^32 + 1 below 2^bits");
    for (uint32_t i = 0; i < count; ++i) h_out[i] = v[i];
    return KS_OK;
}
