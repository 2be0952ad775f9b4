// ks_device.cuh -- device arithmetic and the register/shared-memory NTT core.
//
// Modular arithmetic (all moduli q < 2^56, one uint64 per residue):
//   * Shoup multiplication by a known constant w with w' = floor(w*2^64/q):
//     a*w - floor(a*w'/2^64)*q lies in [0, 2q) for every a < 2^64 (Shoup).
//     The NTT butterflies use an estimate of that quotient built from three
//     of the four 32x32-bit partial products of a*w' (shoup_est), which
//     widens the range to [0, 4q) and saves a full 64x64 high product.
//   * Lazy butterflies (after Harvey): the forward (Cooley-Tukey) butterfly
//     lets values grow by at most 4q per stage and is reduced once at the
//     end; the inverse (Gentleman-Sande) one keeps them in [0, 4q).
//   * Montgomery reduction (REDC) of a 128-bit sum of products with the
//     stored key, whose factor 2^64 is folded in at upload.
//   * Base conversion accumulates 28-bit-split partial products in three
//     64-bit accumulators (no carries; the middle one in Karatsuba form) and
//     reduces once per output with a Montgomery reduction (constants stored
//     times 2^64).
//
// NTT structure.  The negacyclic NTT of N = 2^(LA+LB) points is the in-place
// Cooley-Tukey network whose stage s pairs indices differing in bit
// logN-1-s, with twiddle psi^brv(2^s + i) for butterfly group i.  Stages
// 0..LA-1 act within columns (fixed low LB index bits), stages LA..logN-1
// within rows (fixed high LA bits), so the transform splits into a column
// pass and a row pass over the limb viewed as a 2^LA x 2^LB matrix.  Inside a
// pass each sub-transform of 2^L points is held in registers by 2^(L-RR)
// threads (2^RR values each), RR = ceil(L/2): the first RR stages run in
// registers, one shared-memory transpose regroups the values, and the
// remaining L-RR stages run in registers again.  In sub-transform-local
// terms the twiddle of local stage s and local group i is tw[G*2^s + i] with
// G = 1 for the column pass and G = 2^LA + row for the row pass.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ks_internal.h"

namespace ks {

// ------------------------------------------------------------------ scalar
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q)
{
    return a * w - __umul64hi(a, wp) * q;  // [0, 2q)
}

__device__ __forceinline__ u64 reduce2(u64 x, u64 q)  // [0, 2q) -> [0, q)
{
    return x >= q ? x - q : x;
}

__device__ __forceinline__ u64 reduce4(u64 x, u64 q, u64 q2)  // [0, 4q) -> [0, q)
{
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// Shoup product with an estimated quotient.  Write a = a1*2^32 + a0 and
// w' = floor(w*2^64/q) = p1*2^32 + p0 (32-bit halves).  The exact Shoup
// quotient is Q = floor(a*w'/2^64), and
//   a*w'/2^64 = a1*p1 + (a1*p0 + a0*p1)/2^32 + a0*p0/2^64.
// The estimate E = a1*p1 + floor(a1*p0/2^32) + floor(a0*p1/2^32) drops two
// fractional parts below 1 each and a term below 1, so a*w'/2^64 - E lies in
// [0, 3) and Q - E is 0, 1 or 2.  Shoup's bound gives a*w - Q*q in [0, 2q),
// hence t = a*w - E*q lies in [0, 4q) for every a < 2^64, w < q < 2^56; as
// 4q < 2^64, t is computed exactly modulo 2^64 (nq = 2^64 - q).  Cost: one
// 32x32->64 and two high 32x32 products for E instead of a 64x64 high
// product (three partial products and their carries).
__device__ __forceinline__ u64 shoup_est(u64 a, u64 w, u64 wp, u64 nq)
{
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), p0 = (u32)wp, p1 = (u32)(wp >> 32);
    u64 e = (u64)a1 * p1 + __umulhi(a1, p0);
    e += __umulhi(a0, p1);
    return a * w + e * nq;
}

// The same product for a modulus of the special form q = q1*2^32 + 1
// (every prime of such a parameter set; ks_special_primes lists them):
// E*q mod 2^64 = E + ((E0*q1 mod 2^32) << 32), one 32-bit multiply instead of
// a 64-bit one, so t = a*w - E*q is the low 64 bits of a*w (one 32x32->64
// and two 32-bit products) with E and E0*q1 subtracted.  Same range [0, 4q).
__device__ __forceinline__ u64 shoup_est_sp(u64 a, u64 w, u64 wp, u64 q)
{
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), p0 = (u32)wp, p1 = (u32)(wp >> 32);
    u64 e = (u64)a1 * p1 + __umulhi(a1, p0);
    e += __umulhi(a0, p1);
    const u32 w0 = (u32)w, w1 = (u32)(w >> 32);
    const u64 lo = (u64)a0 * w0;
    const u32 hi = (u32)(lo >> 32) + a0 * w1 + a1 * w0 + (u32)e * (0u - (u32)(q >> 32));
    return ((((u64)hi) << 32) | (u32)lo) - e;
}

// Forward NTT outputs before the final reduction are below kFwdLazy * q:
// inputs below 4q grow by less than 4q per stage, 4q + 17*4q = 72q for the
// 17 stages of N = 2^17, and 76q < 2^63 for q < 2^56.
constexpr u64 kFwdLazy = 72;

// Forward Cooley-Tukey butterfly without a per-stage correction of X: with
// X, Y < B the outputs are below B + 4q (the estimated Shoup product is below
// 4q for any 64-bit Y), so a transform of at most 17 stages fed with values
// below 4q ends below kFwdLazy*q.  Consumers reduce with reduce_any.  SP:
// the modulus has the special form (shoup_est_sp).
template <bool SP = false>
__device__ __forceinline__ void fwd_bfly(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 q2)
{
    const u64 t = SP ? shoup_est_sp(Y, w, wp, q) : shoup_est(Y, w, wp, 0 - q);
    Y = X + (q2 + q2) - t;
    X = X + t;
}

// Any 64-bit x -> [0, q): Shoup product by 1 (into [0, 2q)), one correction.
__device__ __forceinline__ u64 reduce_any(u64 x, u64 q, u64 one_sh)
{
    const u64 r = x - __umul64hi(x, one_sh) * q;
    return r >= q ? r - q : r;
}

// Inverse Harvey butterfly on [0, 4q): X, Y in [0, 4q) -> [0, 4q) (the sum
// below 8q takes one conditional subtraction of 4q; the difference plus 4q
// is below 8q and its estimated Shoup product below 4q).
template <bool SP = false>
__device__ __forceinline__ void inv_bfly(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 q2)
{
    const u64 q4 = q2 + q2;
    u64 s = X + Y;
    s = s >= q4 ? s - q4 : s;
    const u64 d = X - Y + q4;
    X = s;
    Y = SP ? shoup_est_sp(d, w, wp, q) : shoup_est(d, w, wp, 0 - q);
}

// 128-bit accumulator.
struct U128 {
    u64 lo, hi;
};
__device__ __forceinline__ void mac128(U128 &acc, u64 a, u64 b)
{
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1 : 0);
}
// Montgomery reduction: returns T * 2^-64 mod q in [0, q + T/2^64).
__device__ __forceinline__ u64 redc(U128 T, u64 q, u64 mont)
{
    u64 m = T.lo * mont;
    return T.hi + __umul64hi(m, q) + (T.lo != 0 ? 1 : 0);
}
// Canonical key product of the a half from its 128-bit sum (see key_a).
template <bool CK>
__device__ __forceinline__ u64 key_a_finish(const KeyView &K, U128 sa, const ModC &mc, const ulonglong2 *fold, int t)
{
    u64 x = redc(sa, mc.q, mc.mont);
    if (CK && K.comp) x = shoup_lazy(x, fold[t].x, fold[t].y, mc.q);
    return reduce_any(x, mc.q, mc.one_sh);
}

// ------------------------------------------------------------------ keys
// Compressed keys store b_j ([digit][tower][N], stored form) and regenerate
// a_j (canonical, evaluation form) from a seed.  a-word (j, t, n), t the full
// tower index, is the first of the draws
//   v_m = SM(seed ^ 2, ((j*nfull + t)*N + n)*64 + m) & mask(bitlen(r)),
// m = 0..63, with v_m < r (the last one mod r if all reject, probability
// below 2^-64), where SM(x, c) is output c (from 0) of the SplitMix64 stream
// seeded with x (Steele, Lea & Flood 2014): the stream's state after c+1
// steps is x + (c+1)*0x9E3779B97F4A7C15, so any output is reached directly.
__device__ __forceinline__ u64 splitmix_out(u64 x, u64 c)
{
    u64 z = x + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ u64 key_a_word(u64 seed, int j, int t, size_t n, int logN, int nfull, u64 r)
{
    const int b = 64 - __clzll((long long)r);
    const u64 mask = b >= 64 ? ~0ull : ((1ull << b) - 1);
    const u64 base = (((((u64)j * (u64)nfull + (u64)t) << logN) + (u64)n) * 64);
    u64 v = 0;
    for (int m = 0; m < 64; ++m) {
        v = splitmix_out(seed ^ 2, base + (u64)m) & mask;
        if (v < r) return v;
    }
    return v % r;
}
// The same words for V consecutive slots n..n+V-1.  Slot n's first draw is
// output 64n' of the stream (n' the slot's global index), whose state is
// x + (64n'+1)*gamma: consecutive slots' first states differ by 64*gamma, so
// one multiply serves the V slots and each further slot costs an addition.
// A first draw that is rejected (at least r) takes the per-slot path for the
// remaining draws.
template <int V>
__device__ __forceinline__ void key_a_words(u64 seed, int j, int t, size_t n, int logN, int nfull, u64 r,
                                            u64 (&out)[V])
{
    constexpr u64 kGamma = 0x9E3779B97F4A7C15ull;
    const int b = 64 - __clzll((long long)r);
    const u64 mask = b >= 64 ? ~0ull : ((1ull << b) - 1);
    const u64 base = (((((u64)j * (u64)nfull + (u64)t) << logN) + (u64)n) * 64);
    u64 st = (seed ^ 2) + (base + 1) * kGamma;
#pragma unroll
    for (int c = 0; c < V; ++c) {
        u64 z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        u64 v = (z ^ (z >> 31)) & mask;
        if (v >= r) v = key_a_word(seed, j, t, n + c, logN, nfull, r);
        out[c] = v;
        st += 64 * kGamma;
    }
}
// Key words of digit j, full tower t, slot n.  Full keys hold both halves
// times the tower's fold factor and 2^64; a compressed key's a-word is
// canonical, so its sum of products is multiplied by that factor once per
// output (key_a_finish).
// CK: the launch may contain compressed keys (otherwise every key is full
// and the regeneration code is left out of the kernel).
template <bool CK>
__device__ __forceinline__ u64 key_b(const KeyView &K, int j, int t, size_t n, int nfull, int logN)
{
    return K.evk[(((size_t)((CK && K.comp) ? j : 2 * j) * nfull + t) << logN) + n];
}
template <bool CK>
__device__ __forceinline__ u64 key_a(const KeyView &K, int j, int t, size_t n, int nfull, int logN, u64 r)
{
    if (CK && K.comp) return key_a_word(K.a_seed, j, t, n, logN, nfull, r);
    return K.evk[(((size_t)(2 * j + 1) * nfull + t) << logN) + n];
}

// Base-conversion accumulator: sum of y*c with y, c < 2^56 split at 28 bits.
struct BAcc {
    u64 a0, a1, a2;
};
__device__ __forceinline__ void bacc_zero(BAcc &A) { A.a0 = A.a1 = A.a2 = 0; }
// Karatsuba form: the middle column is accumulated as (y0+y1)(c0+c1) and the
// outer columns are subtracted at the end, three 32x32->64 products per term
// instead of four.  Factors below 2^29 give products below 2^58, so up to 64
// terms fit in 64 bits.
__device__ __forceinline__ void bacc_mac(BAcc &A, u32 y0, u32 y1, u64 csplit)
{
    const u32 c0 = (u32)csplit, c1 = (u32)(csplit >> 32);
    // one multiply-add of 32x32 bits into 64 bits each (mad.wide.u32): the
    // C form of the same sums is not always compiled to it
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(A.a0) : "r"(y0), "r"(c0));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(A.a2) : "r"(y1), "r"(c1));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(A.a1) : "r"(y0 + y1), "r"(c0 + c1));
}
// Constants are stored times 2^64 (Montgomery form), so the accumulated value
// S = a0 + a1*2^28 + a2*2^56 is reduced by one Montgomery reduction:
// REDC(S) = S*2^-64 mod q = sum y*c mod q.  With at most 64 terms of
// 56-bit factors S < 2^119 and S*2^-64 < q*(64q/2^64) < q, so the result lies
// in [0, 2q).
__device__ __forceinline__ u64 bacc_reduce(const BAcc &A, const ModC &m)
{
    // 128-bit S from the three column sums (middle column recovered first)
    const u64 a1 = A.a1 - A.a0 - A.a2;
    const u64 t1 = a1 << 28;
    u64 lo = A.a0 + t1;
    u64 hi = (a1 >> 36) + (lo < t1 ? 1 : 0);
    const u64 t2 = A.a2 << 56;
    lo += t2;
    hi += (A.a2 >> 8) + (lo < t2 ? 1 : 0);
    U128 S = {lo, hi};
    return redc(S, m.q, m.mont);
}
__device__ __forceinline__ void split_y(u64 y, u32 &y0, u32 &y1)
{
    y0 = (u32)y & ((1u << kSplit) - 1);
    y1 = (u32)(y >> kSplit);
}

// Bulk prefetch of a contiguous block into L2 (TMA, one instruction for the
// whole block).  The bulk copy needs a 16-byte aligned address and a size
// that is a multiple of 16 bytes; blocks of caller buffers that are only
// 8-byte aligned are simply not prefetched.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    if ((((uintptr_t)p) & 15) != 0 || (bytes & 15) != 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ------------------------------------------------------------------ NTT shape
template <int LA_, int LB_>
struct Shape {
    static constexpr int LA = LA_, LB = LB_, LOGN = LA_ + LB_;
    static constexpr int N = 1 << LOGN;
    static constexpr int RA = (LA + 1) / 2, RB = (LB + 1) / 2;
    static constexpr int REGA = 1 << RA, REGB = 1 << RB;
    static constexpr int TA = 1 << (LA - RA), TB = 1 << (LB - RB);  // threads per sub-transform
    static constexpr int COLS_W = (256 / TA) < 16 ? 16 : (256 / TA);
    static constexpr int COLS = COLS_W > (1 << LB) ? (1 << LB) : COLS_W;  // columns per column-pass CTA
    static constexpr int ROWS_W = 64 / TB < 1 ? 1 : 64 / TB;
    static constexpr int ROWS = ROWS_W > (1 << LA) ? (1 << LA) : ROWS_W;  // rows per row-pass CTA
    static constexpr int THREADS_A = COLS * TA;
    static constexpr int THREADS_B = ROWS * TB;
    static constexpr int MB = 1 << (LB - RB);         // group size of the row pass, 2nd round
    static constexpr int ROWPAD = (1 << LB) + (1 << LB) / MB;  // padded row in shared memory
    static constexpr int SMEM_A = (1 << LA) * COLS * 8 + (1 << LA) * 16;
    static constexpr int SMEM_B = ROWS * ROWPAD * 8;
    // CTAs per SM requested from the register allocator: 64 registers a
    // thread (four 256-thread column-pass CTAs; sixteen row-pass CTAs of 64
    // threads, 4 rows at 2^16: each block barrier holds only two warps, and
    // the forward row pass ran 6% faster with 8-row and 2% faster again with
    // 4-row blocks than with 16-row ones; 8-column column-pass blocks were
    // slower); the 32-value column pass of 2^17 stays at the compiler's
    // default (it would spill).
    static constexpr int MINB_A = LA <= 8 ? 4 : 1;
    static constexpr int MINB_B = 16;
    // The forward row kernel stages its rows' first-round twiddles (REGB
    // entries a row, REGB-1 used) in shared memory after the row buffers.
    static constexpr int SMEM_BT = SMEM_B + ROWS * REGB * 16;
};

template <int LOGN>
struct ShapeOf;
template <> struct ShapeOf<10> { typedef Shape<5, 5> T; };
template <> struct ShapeOf<11> { typedef Shape<6, 5> T; };
template <> struct ShapeOf<12> { typedef Shape<6, 6> T; };
template <> struct ShapeOf<13> { typedef Shape<7, 6> T; };
template <> struct ShapeOf<14> { typedef Shape<7, 7> T; };
template <> struct ShapeOf<15> { typedef Shape<8, 7> T; };
template <> struct ShapeOf<16> { typedef Shape<8, 8> T; };
template <> struct ShapeOf<17> { typedef Shape<9, 8> T; };

// ------------------------------------------------------------------ rounds
// Round 1 in registers: x[k], k = the high RR bits of the sub-transform index.
// tw(s, i) returns the (w, w') pair of local stage s, local group i.
template <int RR, bool SP = false, class TW>
__device__ __forceinline__ void fwd_round1(u64 (&x)[1 << RR], const TW &tw, u64 q, u64 q2)
{
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        const int half = (1 << RR) >> (s + 1);
#pragma unroll
        for (int g = 0; g < (1 << s); ++g) {
            const ulonglong2 W = tw(s, g);
#pragma unroll
            for (int k = 0; k < half; ++k) fwd_bfly<SP>(x[g * 2 * half + k], x[g * 2 * half + k + half], W.x, W.y, q, q2);
        }
    }
}

// Round 2 in registers: NG groups of M = 2^(L-RR) values; group gg has
// global group id gid0 + gg (the high RR bits of the index).
template <int L, int RR, bool SP = false, class TW>
__device__ __forceinline__ void fwd_round2(u64 (&x)[1 << RR], int gid0, const TW &tw, u64 q, u64 q2)
{
    constexpr int M = 1 << (L - RR);
    constexpr int NG = (1 << RR) / M;
#pragma unroll
    for (int s2 = 0; s2 < L - RR; ++s2) {
        const int half = M >> (s2 + 1);
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) {
#pragma unroll
            for (int g2 = 0; g2 < (1 << s2); ++g2) {
                const ulonglong2 W = tw(RR + s2, ((gid0 + gg) << s2) + g2);
#pragma unroll
                for (int k = 0; k < half; ++k)
                    fwd_bfly<SP>(x[gg * M + g2 * 2 * half + k], x[gg * M + g2 * 2 * half + k + half], W.x, W.y, q, q2);
            }
        }
    }
}

// Inverse of fwd_round2: local stages L-1 .. RR on the low bits.
template <int L, int RR, bool SP = false, class TW>
__device__ __forceinline__ void inv_round2(u64 (&x)[1 << RR], int gid0, const TW &tw, u64 q, u64 q2)
{
    constexpr int M = 1 << (L - RR);
    constexpr int NG = (1 << RR) / M;
#pragma unroll
    for (int s2 = L - RR - 1; s2 >= 0; --s2) {
        const int half = M >> (s2 + 1);
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) {
#pragma unroll
            for (int g2 = 0; g2 < (1 << s2); ++g2) {
                const ulonglong2 W = tw(RR + s2, ((gid0 + gg) << s2) + g2);
#pragma unroll
                for (int k = 0; k < half; ++k)
                    inv_bfly<SP>(x[gg * M + g2 * 2 * half + k], x[gg * M + g2 * 2 * half + k + half], W.x, W.y, q, q2);
            }
        }
    }
}

// Inverse of fwd_round1: local stages RR-1 .. 0 on the high bits.
template <int RR, bool SP = false, class TW>
__device__ __forceinline__ void inv_round1(u64 (&x)[1 << RR], const TW &tw, u64 q, u64 q2)
{
#pragma unroll
    for (int s = RR - 1; s >= 0; --s) {
        const int half = (1 << RR) >> (s + 1);
#pragma unroll
        for (int g = 0; g < (1 << s); ++g) {
            const ulonglong2 W = tw(s, g);
#pragma unroll
            for (int k = 0; k < half; ++k) inv_bfly<SP>(x[g * 2 * half + k], x[g * 2 * half + k + half], W.x, W.y, q, q2);
        }
    }
}

// Twiddle fetchers.  Column pass: the first 2^LA entries of the tower's table,
// staged in shared memory (G = 1).  Row pass: the forward row kernel stages
// its rows' first-round twiddles in shared memory (TwStaged,
// ks_ntt_core.cuh); TwRow reads straight from the tower's global table
// (G = 2^LA + row).
struct TwSmem {
    const ulonglong2 *t;
    __device__ __forceinline__ ulonglong2 operator()(int s, int i) const { return t[(1 << s) + i]; }
};
struct TwRow {
    const ulonglong2 *t;  // tower table
    int G;
    __device__ __forceinline__ ulonglong2 operator()(int s, int i) const { return __ldg(t + (G << s) + i); }
};
// Same table, fetched with a volatile load: kernels that run several row
// transforms of one tower in a loop would otherwise keep every twiddle of the
// row live in registers across iterations.
struct TwRowV {
    const ulonglong2 *t;
    int G;
    __device__ __forceinline__ ulonglong2 operator()(int s, int i) const
    {
        ulonglong2 r;
        asm volatile("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(t + (G << s) + i));
        return r;
    }
};

}  // namespace ks
