// ks_bconv_tc.cu -- fast base conversion (ModUp P2, ModDown P2) on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The conversion z_t = sum_i y_i c_{i,t} mod r_t is a product of a
// [coefficients x sources] matrix by a [sources x targets] matrix of
// constants below 2^56.  Exactness with f16 operands: y_i (canonical, < 2^56)
// is cut into 7 bytes y_{i,a}, so y_i c_{i,t} = sum_a y_{i,a} 2^(8a) c_{i,t}.
// The shift of byte a is folded into the constant, c'_{i,a,t} = 2^(8a)
// c_{i,t} mod r_t, and each c' is cut into W-bit slices c'_{i,a,t,b}
// (W = 8: 7 slices; W = 9: 6 slices, when every modulus is below 2^54 and the
// sources fit one K block); then
//   z_t == sum_b 2^(Wb) P_{t,b}  (mod r_t),
//   P_{t,b} = sum_i sum_a y_{i,a} c'_{i,a,t,b},
// and every P_{t,b} (at most 18 sources x 7 bytes x 255^2, or 9 x 7 x 255 x
// 511 with W = 9, below 2^23) is an exact integer in the fp32 accumulator.  One MMA of M=128 coefficients,
// K = 7*(sources) padded to 64 (up to 9 sources) or 128 (up to 18: two K
// blocks), N = 8 per target (7 byte rows used) computes
// all P_{t,b} of up to 32 targets: the A tile holds the byte slices of y
// (built by the CTA from the source limbs), the B tile the per-target slabs
// B[b][7i+a] = c'_{i,a,t,b} (precomputed on the host, 1 KB a K block).  The
// epilogue reads the 6 or 7 sums from tensor memory and recombines them into
// S = sum_{i,a} y_{i,a} c'_{i,a,t} exactly; S <= 126*255*r < 2^15 r, so one
// Montgomery step by 2^32 (constants carry 2^32) leaves (S + m r)/2^32 below
// 2r: a lazy [0, 2r) output like the CUDA-core kernels (the same residue; the
// representative may differ).
//
// Operand layout: the canonical K-major layout without swizzle: 8x16-byte
// core matrices, K-adjacent core matrices 128 bytes apart (LBO), 8-row
// groups 1024 bytes a K block apart (SBO); B slabs of 8 rows concatenate.
#include <cstdio>

#include "ks_device.cuh"
#include "ks_launch.h"

namespace ks {

namespace {

constexpr int TC_M = 128;            // coefficients per MMA tile
constexpr int TC_TB = 32;            // targets per MMA (8 accumulator columns each)
constexpr uint32_t TC_LBO = 128;
// KB K blocks of 64: K = 64*KB columns (7 x up to 9*KB sources, the last
// column the bias), 8-row groups K/8*128 bytes apart, slabs of 8 rows.
template <int KB> struct TcK {
    static constexpr int K = 64 * KB;
    static constexpr uint32_t SBO = (K / 8) * 128;
    static constexpr int SLAB = 8 * K * 2;  // bytes of one target slab
    static constexpr int NSV = KB == 1 ? 5 : 10;  // source words of one producer (half a row)
};
static_assert(TcK<1>::SLAB == 2 * kTcSlabHalves && TcK<2>::SLAB == 4 * kTcSlabHalves, "slab size");
constexpr int TC_WAIT_LIMIT = 1 << 24;  // mbarrier polls before giving up

__device__ int g_tc_error;  // set when an MMA completion wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int KB>
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((TcK<KB>::SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle
    return d;
}
// kind::f16 instruction descriptor: D f32, A and B f16, both K-major.
__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
template <int KB>
__host__ __device__ __forceinline__ uint32_t tc_off(int r, int k)
{
    return (uint32_t)((r / 8) * TcK<KB>::SBO + (k / 8) * TC_LBO + (r % 8) * 16 + (k % 8) * 2);
}
// Two bytes as an exact f16 pair: byte a0 of word x (low half) and byte a1 of
// word y (high half).  0x6400 | b is the f16 of 1024 + b (b < 1024), so one
// byte permute, one logic op and one packed subtraction of 1024 give (b0, b1).
// The selector is a constant once the callers' loops are unrolled.
__device__ __forceinline__ uint32_t f16x2_bytes(uint32_t x, uint32_t y, uint32_t a0, uint32_t a1)
{
    const uint32_t sel = a0 | ((4u + a1) << 8);  // x.byte[a0] -> byte 0, y.byte[a1] -> byte 2
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(y), "r"(sel));
    d = (d & 0x00FF00FFu) | 0x64006400u;
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(d), "r"(0x64006400u));
    return r;
}

// The shifted partial sums of one target (W-bit slices: 7 for W = 8, 6 for
// W = 9), recombined and reduced by one Montgomery step by 2^32.  v[b] are the
// raw accumulator bits 0x4B000000 + P_b (bias column); the bias is removed
// once per group (modulo 2^64: the exact sums fit).  qinv = -q^-1 mod 2^32.
template <int W>
__device__ __forceinline__ u64 tc_reduce(const uint32_t *v, u64 q, uint32_t qinv)
{
    constexpr u64 B = 0x4B000000ull;
    constexpr u64 B5 = B * (1ull + (1ull << W) + (1ull << (2 * W)) + (1ull << (3 * W)) + (1ull << (4 * W)));
    u64 a0 = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) a0 += (u64)v[b] << (W * b);
    a0 -= B5;                           // P_0 + ... + P_4 2^(4W) < 2^(23 + 4W + 1)
    u64 a1;                             // the sums above, at 2^(5W)
    if constexpr (W == 8)
        a1 = (u64)v[5] + ((u64)v[6] << 8) - B * 0x0101ull;
    else
        a1 = (u64)v[5] - B;
    const u64 t1 = a1 << (5 * W);
    const u64 lo = a0 + t1;
    const uint32_t hi = (uint32_t)(a1 >> (64 - 5 * W)) + (lo < t1 ? 1u : 0u);  // S = lo + hi 2^64
    // (S + m q) / 2^32 with m = -S q^-1 mod 2^32: the low word of S + m q is 0
    const uint32_t l0 = (uint32_t)lo, l1 = (uint32_t)(lo >> 32);
    const uint32_t m = l0 * qinv;
    const u64 w = (u64)m * (uint32_t)q + l0;
    return (u64)m * (uint32_t)(q >> 32) + (w >> 32) + l1 + ((u64)hi << 32);
}

// 16 consecutive accumulator columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase)
{
    uint32_t done = 0;
    for (int it = 0; it < TC_WAIT_LIMIT && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
    return done != 0;
}

// One unit of work: a tile of 128 coefficients for one block of <= 16
// targets of one (job, digit) (ModUp) or (job, polynomial) (ModDown).
struct TcItem {
    const u64 *src;     // source tower 0 at the tile's first coefficient; tower i at + i*N
    int nsrc;           // source towers (<= 18)
    int G;              // targets (0: nothing to do)
    int key;            // (job block, target block): the B slabs and targets change with it
    int sbase;          // slab index base (ModUp: of the digit at this level)
    int t_first, ov_at, ov, nact, t_base;  // target numbering (ModUp)
    u64 *dst0;          // output base: target t at dst0 + (t - t_base)*N
};

template <int MODE>
__device__ __forceinline__ TcItem tc_item(const Tables &T, const BUpJobs &bu, const BDnJobs &bd, int item, int XT,
                                          int TBN, int TB)
{
    const size_t N = (size_t)1 << T.logN;
    const int xt = item % XT, r = item / XT, tb = r % TBN, z = r / TBN;
    TcItem it;
    it.key = r;
    if (MODE == 0) {
        const int jb = find_slot(bu.zpre, bu.n, z);
        const BUpJob &J = bu.job[jb];
        const int j = J.jsel >= 0 ? J.jsel : z - bu.zpre[jb];
        const int lo = j * T.alpha, hi = min(lo + T.alpha, J.nact);
        const int olo = max(lo, J.t_begin), ohi = min(hi, J.t_end);
        it.ov = ohi > olo ? ohi - olo : 0;
        it.ov_at = olo;
        const int nb = (J.t_end - J.t_begin) - it.ov;
        const int u0 = tb * TB;
        it.G = max(0, min(TB, nb - u0));
        it.t_first = J.t_begin + u0;
        it.nact = J.nact;
        it.t_base = J.t_base;
        it.nsrc = hi - lo;
        it.src = J.y + (size_t)lo * N + (size_t)xt * TC_M;
        it.sbase = T.up_tc_lvl[(size_t)(J.nact - 1) * T.ndig + j];
        it.dst0 = J.D + (size_t)(J.jsel >= 0 ? 0 : j) * J.dstride + (size_t)xt * TC_M;
    } else {
        const int jb = find_slot(bd.zpre, bd.n, z);
        const BDnJob &J = bd.job[jb];
        const int x = z - bd.zpre[jb];
        const int i0 = tb * TB;
        it.G = max(0, min(TB, J.nact - i0));
        it.t_first = i0;
        it.ov = 0;
        it.ov_at = 0;
        it.nact = J.nact;
        it.t_base = 0;
        it.nsrc = T.kp;
        it.src = J.cp + (size_t)x * J.cp_stride + (size_t)J.nact * N + (size_t)xt * TC_M;
        it.sbase = 0;
        it.dst0 = J.v + (size_t)x * J.v_stride + (size_t)xt * TC_M;
    }
    return it;
}

// target g of an item: compact tower, full tower, slab
template <int MODE>
__device__ __forceinline__ void tc_target(const Tables &T, const TcItem &it, int g, int &t, int &tf, int &slab)
{
    if (MODE == 0) {
        t = it.t_first + g;
        if (it.ov > 0 && t >= it.ov_at) t += it.ov;
        tf = full_tower(t, it.nact, T.nq);
        slab = it.sbase + tf;
    } else {
        t = it.t_first + g;
        tf = t;
        slab = t;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// OR of a flag over the 256 producer threads (named barrier 1 with reduction).
__device__ __forceinline__ bool producers_or(bool f)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)f)
        : "memory");
    return r != 0;
}

constexpr int TC_PROD = 256;                  // producer threads (warps 0-7): two per tile row
constexpr int TC_CONS_WARPS = 16;             // consumer warps: 4 lane quarters x 4 target groups
constexpr int TC_PIPE_THREADS = TC_PROD + 32 * TC_CONS_WARPS;
constexpr uint32_t TC_PIPE_COLS = 512;        // two accumulators of 256 columns

// Half H of A-tile row m: K chunks CH*H..CH*H+CH-1 (CH = 4*KB chunks of 8
// columns) from the sources they touch, y[u] = source SB + u with SB =
// 8*CH*H/7 (zero past the item's sources).  Column K-1 is the bias.
template <int KB, int H>
struct TcHalf {
    static constexpr int SB = 8 * 4 * KB * H / 7;                          // first source
    static constexpr int LAST = H == 1 ? 64 * KB - 2 : 8 * 4 * KB * (H + 1) - 1;  // last slice column
    static_assert(LAST / 7 - SB < TcK<KB>::NSV, "source words of a half row");
};
template <int KB, int H>
__device__ __forceinline__ void tc_build_half(unsigned char *sa, int m, const u64 (&y)[TcK<KB>::NSV])
{
    constexpr int CH = 4 * KB, SB = TcHalf<KB, H>::SB, NSV = TcK<KB>::NSV, K = TcK<KB>::K;
    uint32_t wd[2 * NSV];
#pragma unroll
    for (int u = 0; u < NSV; ++u) {
        wd[2 * u] = (uint32_t)y[u];
        wd[2 * u + 1] = (uint32_t)(y[u] >> 32);
    }
#pragma unroll
    for (int c = CH * H; c < CH * H + CH; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const int k0 = 8 * c + e, k1 = k0 + 1;
            const int u0 = k0 / 7 - SB, a0 = k0 % 7, u1 = k1 / 7 - SB, a1 = k1 % 7;
            if (k1 == K - 1)  // the last slice byte, then the bias 2048 (f16 0x6800)
                w[e / 2] = (f16x2_bytes(wd[2 * u0 + a0 / 4], 0u, (uint32_t)(a0 % 4), 0u) & 0xFFFFu) | 0x68000000u;
            else
                w[e / 2] = f16x2_bytes(wd[2 * u0 + a0 / 4], wd[2 * u1 + a1 / 4], (uint32_t)(a0 % 4), (uint32_t)(a1 % 4));
        }
        *reinterpret_cast<uint4 *>(sa + tc_off<KB>(m, 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Walks a CTA's contiguous run of items: (xt, r) advance without divisions and
// the item is decoded again only when its (job block, target block) changes.
template <int MODE>
struct TcCursor {
    int xt, r, XT, TBN, TB;
    TcItem it;
    __device__ __forceinline__ void start(const Tables &T, const BUpJobs &bu, const BDnJobs &bd, int item, int XT_,
                                          int TBN_, int TB_)
    {
        XT = XT_;
        TBN = TBN_;
        TB = TB_;
        xt = item % XT;
        r = item / XT;
        it = tc_item<MODE>(T, bu, bd, item, XT, TBN, TB);
    }
    __device__ __forceinline__ void next(const Tables &T, const BUpJobs &bu, const BDnJobs &bd)
    {
        if (++xt == XT) {
            xt = 0;
            ++r;
            it = tc_item<MODE>(T, bu, bd, r * XT, XT, TBN, TB);
        } else {
            it.src += TC_M;
            it.dst0 += TC_M;
        }
    }
};

// Persistent pipelined base conversion: each CTA (one per SM) takes a
// contiguous run of items.  Producer warps load the next item's sources into
// registers while they build the current A tile, then one thread issues the
// MMAs into the accumulator buffer of the item (two buffers alternate) and
// commits them to acc_full; consumer warps wait on acc_full, run the
// epilogue and release the buffer through acc_empty.  Every wait is bounded:
// on timeout the kernel sets g_tc_error and its threads leave their loops.
template <int MODE, int KB, int W>
__global__ void __launch_bounds__(TC_PIPE_THREADS, 1) k_bconv_tc(Tables T, BUpJobs bu, BDnJobs bd, const uint4 *slabs,
                                                                int XT, int TBN, int TB, int items)
{
    constexpr int K = TcK<KB>::K, NSV = TcK<KB>::NSV;
    extern __shared__ unsigned char tc_dyn[];
    unsigned char *sa0 = tc_dyn + ((128 - (smem_u32(tc_dyn) & 127)) & 127);
    unsigned char *sb = sa0 + 2 * TC_M * K * 2;
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tbase_s;
    __shared__ u64 *s_dst[2][TC_TB];
    __shared__ u64 s_q[2][TC_TB], s_mont[2][TC_TB];
    __shared__ int s_G[2];
    const int per = (items + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(items, i0 + per);
    if (i0 >= i1) return;
    const size_t N = (size_t)1 << T.logN;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 2);              // MMA commit + producer release of the targets
            mbar_init(smem_u32(&acc_empty[b]), TC_CONS_WARPS);  // one arrival per consumer warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase_s)),
                     "r"(TC_PIPE_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tbase_s;

    if (tid < TC_PROD) {
        // ------------------------------------------------------------ producers
        const int m = tid % TC_M, h = tid / TC_M;  // row m, half h of its K columns
        const int sb0 = h == 0 ? TcHalf<KB, 0>::SB : TcHalf<KB, 1>::SB;  // first source of the half
        int k = 0, cur_r = -1;
        TcCursor<MODE> cur, nxt;
        nxt.start(T, bu, bd, i0, XT, TBN, TB);
        u64 y[NSV];
#pragma unroll
        for (int u = 0; u < NSV; ++u)
            y[u] = (nxt.it.G > 0 && sb0 + u < nxt.it.nsrc) ? nxt.it.src[(size_t)(sb0 + u) * N + m] : 0;
        bool ok = true;
        for (int item = i0; item < i1; ++item) {
            cur = nxt;
            u64 yc[NSV];
#pragma unroll
            for (int u = 0; u < NSV; ++u) yc[u] = y[u];
            if (item + 1 < i1) {  // the next item's sources are in flight while this one is built
                nxt.next(T, bu, bd);
#pragma unroll
                for (int u = 0; u < NSV; ++u)
                    y[u] = (nxt.it.G > 0 && sb0 + u < nxt.it.nsrc) ? nxt.it.src[(size_t)(sb0 + u) * N + m] : 0;
            }
            const TcItem &it = cur.it;
            if (it.G == 0) continue;
            const int buf = k & 1;
            const bool restage = cur.r != cur_r;
            bool bad = false;
            // the accumulator and A tile of this buffer were last used by item k-2
            if (k >= 2) bad = !tc_wait(smem_u32(&acc_empty[buf]), (uint32_t)(((k >> 1) - 1) & 1));
            // new targets: every earlier MMA must be done with the B slabs
            if (!bad && restage && k >= 1) bad = !tc_wait(smem_u32(&acc_empty[buf ^ 1]), (uint32_t)(((k - 1) >> 1) & 1));
            if (producers_or(bad)) {
                ok = false;
                break;
            }
            if (restage) {
                // G slabs, and a zero slab after an odd G (the MMA's N is a
                // multiple of 16 columns: two targets)
                constexpr int W = TcK<KB>::SLAB / 16;
                const int Gp = (it.G + 1) & ~1;
                for (int idx = tid; idx < Gp * W; idx += TC_PROD) {
                    const int g = idx / W, w = idx % W;
                    uint4 val = make_uint4(0u, 0u, 0u, 0u);
                    if (g < it.G) {
                        int t, tf, slab;
                        tc_target<MODE>(T, it, g, t, tf, slab);
                        val = slabs[(size_t)slab * W + w];
                    }
                    reinterpret_cast<uint4 *>(sb)[idx] = val;
                }
                cur_r = cur.r;
            }
            unsigned char *sa = sa0 + buf * (TC_M * K * 2);
            // A tile: row m, columns 7i+a = byte a of source i (f16); column 63 =
            // 2048, the bias with the slabs' 4096 there.  Sources past nsrc are 0.
            if (h == 0)
                tc_build_half<KB, 0>(sa, m, yc);
            else
                tc_build_half<KB, 1>(sa, m, yc);
            if (h == 0 && m < it.G) {
                int t, tf, slab;
                tc_target<MODE>(T, it, m, t, tf, slab);
                s_dst[buf][m] = it.dst0 + (size_t)(t - it.t_base) * N;
                s_q[buf][m] = T.modc[tf].q;
                s_mont[buf][m] = T.modc[tf].mont;
            }
            if (tid == 0) s_G[buf] = it.G;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            producers_sync();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t idesc = tc_idesc(8 * ((it.G + 1) & ~1));
                const uint32_t dcol = tbase + (uint32_t)(buf * 256);
#pragma unroll
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint64_t ad = tc_desc<KB>(smem_u32(sa) + kk * 2 * TC_LBO);
                    const uint64_t bdsc = tc_desc<KB>(smem_u32(sb) + kk * 2 * TC_LBO);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dcol),
                        "l"(ad), "l"(bdsc), "r"(idesc), "r"((uint32_t)kk));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&acc_full[buf]))
                             : "memory");
                mbar_arrive(smem_u32(&acc_full[buf]));  // releases s_dst/s_q/s_mont/s_G of this buffer
            }
            ++k;
        }
        if (!ok && tid == 0) {
            atomicExch(&g_tc_error, 1);
            // once more, bounded, for the last MMAs still in flight before the memory is freed
            if (k >= 1) tc_wait(smem_u32(&acc_full[(k - 1) & 1]), (uint32_t)(((k - 1) >> 1) & 1));
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int cw = warp - TC_PROD / 32, quarter = cw % 4, part = cw / 4;
        const int row = quarter * 32 + lane;
        int k = 0;
        bool ok = true;
        TcCursor<MODE> cur;
        cur.start(T, bu, bd, i0, XT, TBN, TB);
        for (int item = i0; item < i1; ++item) {
            if (item > i0) cur.next(T, bu, bd);
            if (cur.it.G == 0) continue;
            const int buf = k & 1;
            const bool got = tc_wait(smem_u32(&acc_full[buf]), (uint32_t)((k >> 1) & 1));
            if (__any_sync(0xffffffffu, !got)) {  // the warp's lanes agree (tcgen05.ld is warp-collective)
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int G = s_G[buf], NP = (G + 1) / 2;
            // target pairs (2p, 2p+1: 16 columns) strided over the four warps
            // of a lane quarter, two tensor-memory loads in flight per wait
            for (int p = part; p < NP; p += 8) {
                const bool two = p + 4 < NP;
                uint32_t v[16], w[16];
                const uint32_t taddr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256 + 16 * p);
                tmem_ld16(taddr, v);
                if (two) tmem_ld16(taddr + 64, w);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int g = 2 * p;
                s_dst[buf][g][row] = tc_reduce<W>(v, s_q[buf][g], (uint32_t)s_mont[buf][g]);
                if (g + 1 < G) s_dst[buf][g + 1][row] = tc_reduce<W>(v + 8, s_q[buf][g + 1], (uint32_t)s_mont[buf][g + 1]);
                if (two) {
                    s_dst[buf][g + 8][row] = tc_reduce<W>(w, s_q[buf][g + 8], (uint32_t)s_mont[buf][g + 8]);
                    if (g + 9 < G)
                        s_dst[buf][g + 9][row] = tc_reduce<W>(w + 8, s_q[buf][g + 9], (uint32_t)s_mont[buf][g + 9]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
            ++k;
        }
        if (!ok && lane == 0) atomicExch(&g_tc_error, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_PIPE_COLS));
}

// Dynamic shared memory: two A tiles (16 KB each) and up to 16 B slabs
// (32 KB), padded so that one CTA holds an SM (it takes all 512 columns of
// tensor memory).
// With two K blocks: two 32 KB A tiles and up to 32 slabs of 2 KB.
template <int KB> constexpr int tc_pipe_smem() { return KB == 1 ? 120 * 1024 : 132 * 1024; }
static_assert(tc_pipe_smem<1>() >= 2 * TC_M * TcK<1>::K * 2 + TC_TB * TcK<1>::SLAB + 128, "tile space");
static_assert(tc_pipe_smem<2>() >= 2 * TC_M * TcK<2>::K * 2 + TC_TB * TcK<2>::SLAB + 128, "tile space");

}  // namespace

bool bconv_tc_supported(const Tables &T, int nsrc)
{
    return nsrc <= 18 && (((size_t)1 << T.logN) % (size_t)TC_M) == 0;
}

static int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <int MODE, int KB, int W>
static int launch_tc(const Tables &T, const BUpJobs &bu, const BDnJobs &bd, int span, int Z, const uint4 *slabs,
                     cudaStream_t st, const char *name)
{
    // target blocks of equal size (at most 32): 38 targets run as 19 + 19
    const int TBN = (span + TC_TB - 1) / TC_TB;
    const int TB = (span + TBN - 1) / TBN;
    static std::atomic<uint64_t> attr{0};
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_bconv_tc<MODE, KB, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_pipe_smem<KB>());
    });
    const int XT = (int)(((size_t)1 << T.logN) / TC_M);
    const long long items = (long long)XT * TBN * Z;
    if (items <= 0) return KS_OK;
    const int grid = (int)std::min<long long>(items, sm_count());
    KS_LAUNCH(st, name, (k_bconv_tc<MODE, KB, W><<<grid, TC_PIPE_THREADS, tc_pipe_smem<KB>(), st>>>(T, bu, bd, slabs, XT,
                                                                                                 TBN, TB, (int)items)));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KS_OK : fail(KS_ECUDA, std::string(name) + " (tensor cores) launch: " + cudaGetErrorString(e));
}

int launch_bconv_up_tc(const Tables &T, const BUpJobs &b, const uint4 *slabs, const int *, cudaStream_t st)
{
    int span = 0;  // most targets of any (job, digit): the range minus the digit's own towers
    for (int i = 0; i < b.n; ++i) {
        const BUpJob &J = b.job[i];
        const int nd = (J.nact + T.alpha - 1) / T.alpha;
        for (int j = (J.jsel >= 0 ? J.jsel : 0); j < (J.jsel >= 0 ? J.jsel + 1 : nd); ++j) {
            const int lo = j * T.alpha, hi = std::min(lo + T.alpha, J.nact);
            const int olo = std::max(lo, J.t_begin), ohi = std::min(hi, J.t_end);
            span = std::max(span, (J.t_end - J.t_begin) - std::max(0, ohi - olo));
        }
    }
    if (span <= 0) return KS_OK;
    BDnJobs none;
    none.n = 0;
    Tables Tt = T;
    Tt.up_tc = slabs;
    if (tc_kblocks(T.alpha) == 2) return launch_tc<0, 2, 8>(Tt, b, none, span, b.zpre[b.n], slabs, st, "bconv_up");
    return tc_slice_bits(1, T.tc_below54) == 9 ? launch_tc<0, 1, 9>(Tt, b, none, span, b.zpre[b.n], slabs, st, "bconv_up")
                                               : launch_tc<0, 1, 8>(Tt, b, none, span, b.zpre[b.n], slabs, st, "bconv_up");
}

int launch_bconv_down_tc(const Tables &T, const BDnJobs &b, const uint4 *slabs, cudaStream_t st)
{
    int span = 0;
    for (int i = 0; i < b.n; ++i) span = std::max(span, b.job[i].nact);
    if (span <= 0) return KS_OK;
    BUpJobs none;
    none.n = 0;
    if (tc_kblocks(T.kp) == 2) return launch_tc<1, 2, 8>(T, none, b, span, b.zpre[b.n], slabs, st, "bconv_down");
    return tc_slice_bits(1, T.tc_below54) == 9 ? launch_tc<1, 1, 9>(T, none, b, span, b.zpre[b.n], slabs, st, "bconv_down")
                                               : launch_tc<1, 1, 8>(T, none, b, span, b.zpre[b.n], slabs, st, "bconv_down");
}

int tc_error_flag(bool clear)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    }
    return v;
}

// Host: the B slab of one target of modulus r: rows b (slice b of the
// folded constant, W bits; rows past the slices zero), columns k = 7i + a
// (source i, byte a of y): slice b of c_i * 2^(8a) * 2^-32 mod r (c_i carries
// 2^64, the epilogue's reduction takes 2^32 off); the last column holds the bias.
template <int KB>
static void tc_slab_kb(const std::vector<u64> &c, u64 r, int W, uint16_t *slab)
{
    constexpr int K = TcK<KB>::K;
    const int NSL = W == 8 ? 7 : 6;
    const u64 inv32 = invmod_h((u64)(((unsigned __int128)1 << 32) % r), r);
    for (int k = 0; k < K; ++k) {
        const int i = k / 7, a = k % 7;
        const u64 cf = (k < K - 1 && i < (int)c.size())
                           ? mulmod_h(mulmod_h(c[i] % r, inv32, r), powmod_h(2, 8 * (u64)a, r), r) : 0;
        for (int b = 0; b < 8; ++b) {
            const uint32_t sl = b < NSL ? (uint32_t)((cf >> (W * b)) & ((1u << W) - 1)) : 0u;
            // f16 of an integer below 2048
            uint16_t bits = 0;
            if (sl) {
                int e = 31 - __builtin_clz(sl);                   // exponent
                uint32_t mant = (sl << (10 - e)) & 0x3FF;          // 10 fraction bits
                bits = (uint16_t)(((15 + e) << 10) | mant);
            }
            slab[tc_off<KB>(b, k) / 2] = bits;
        }
    }
    // the last column (never a slice: 9*KB sources use the columns before it)
    // holds 4096 in the used slice rows; times the A tile's 2048 there it
    // adds 2^23, so the fp32 accumulator of P (< 2^23) reads 2^23 + P: its
    // bits are 0x4B000000 + P
    for (int b = 0; b < NSL; ++b) slab[tc_off<KB>(b, K - 1) / 2] = (uint16_t)((15 + 12) << 10);
}

void tc_slab(const std::vector<u64> &c, u64 r, int kblocks, int bits, uint16_t *slab)
{
    if (kblocks == 1)
        tc_slab_kb<1>(c, r, bits, slab);
    else
        tc_slab_kb<2>(c, r, 8, slab);
}

}  // namespace ks
