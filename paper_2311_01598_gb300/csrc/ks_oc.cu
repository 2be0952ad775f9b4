// ks_oc.cu -- Output-Centric dataflow (CiFlow Sec. IV-C), batched.
//
// OC computes the key-switch output tower by tower instead of stage by stage.
// GPU schedule (special towers first -- ModDown of every Q output tower needs
// all K special towers of c'), every launch covering all jobs of the batch:
//   1. prep       iNTT of every input tower with the (Q_j/q_i)^-1 prescale
//                 (ModUp P1) -> y, coefficient form;
//   2. P section  BConv of every digit to the special towers only (P2), the
//                 column pass of their NTT (P3), then one fused kernel per row
//                 block: row pass of each digit's limb, the key product summed
//                 over digits on chip (P4+P5), and the row pass of ModDown's
//                 iNTT (ModDown P1); the inverse column pass then yields w;
//   3. Q section  BConv of the other digits to each output tower and of w to
//                 it (ModUp P2, ModDown P2), column passes, then one fused
//                 kernel per row block: row pass, key product with the
//                 bypassed digit read straight from the input (P3-P5), row
//                 pass of the ModDown limbs (ModDown P3) and the subtraction
//                 (ModDown P4) written to the output.
// The key is read once, inside the fused row kernels, while they compute.
#include <algorithm>

#include "ks_ntt_core.cuh"

namespace ks {

// x * e with the stored key word e: REDC of the 128-bit product; x below
// kFwdLazy*q, so the result is below q + 72q^2/2^64 < 2q before the correction.
__device__ __forceinline__ u64 key_mul(u64 x, u64 e, u64 q, u64 mont)
{
    U128 t = {0, 0};
    mac128(t, x, e);
    return reduce2(redc(t, q, mont), q);
}

// Shared memory of the fused row kernels: the row-exchange buffer, then the
// two accumulators (b and a parts of c') of every element of the block's rows.
template <class S>
struct RowSmem {
    static constexpr int ACC = S::ROWS * (1 << S::LB);  // words per accumulator
    static constexpr int BYTES = S::SMEM_B + 2 * ACC * 8;
};

// The per-limb bodies of the fused row kernels are not inlined: each row
// transform then gets its own register allocation, instead of the compiler
// keeping values of one transform live across the next (which tripled the
// register count of the kernels and halved their occupancy).

// One digit's share of the key product for the block's rows: the row pass of
// the limb at gin (skipped for the bypassed digit, whose input is already in
// evaluation form), then x * evk_b and x * evk_a added into the accumulators.
template <class S>
__device__ __noinline__ void oc_digit(const u64 *gin, int transform, const ulonglong2 *twt, int G, u64 *srow, int tau,
                                      const u64 *eb, const u64 *ea, u64 *ab, u64 *aa, int first, u64 q, u64 mont)
{
    u64 x[S::REGB];
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) x[i] = gin[i * S::TB + tau];
    if (transform) row_fwd_core<S>(x, TwRow{twt, G}, srow, tau, q, 2 * q);
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) {
        const int c = i * S::TB + tau;
        const u64 pb = key_mul(x[i], __ldg(eb + c), q, mont);
        const u64 pa = key_mul(x[i], __ldg(ea + c), q, mont);
        ab[c] = first ? pb : reduce2(ab[c] + pb, q);
        aa[c] = first ? pa : reduce2(aa[c] + pa, q);
    }
}

// Row pass of the inverse NTT of an accumulator row, stored to out.
template <class S>
__device__ __noinline__ void oc_inv_store(const u64 *acc, const ulonglong2 *itwt, int G, u64 *srow, int tau, u64 *out,
                                          u64 q)
{
    u64 x[S::REGB];
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) x[i] = acc[i * S::TB + tau];
    row_inv_core<S>(x, TwRow{itwt, G}, srow, tau, q, 2 * q);
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) out[i * S::TB + tau] = x[i];
}

// Row pass of a ModDown limb, then out = acc - NTT(v) mod q.
template <class S>
__device__ __noinline__ void oc_down_store(const u64 *gin, const ulonglong2 *twt, int G, u64 *srow, int tau,
                                           const u64 *acc, u64 *out, u64 q, u64 one_sh)
{
    u64 v[S::REGB];
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) v[i] = gin[i * S::TB + tau];
    row_fwd_core<S>(v, TwRow{twt, G}, srow, tau, q, 2 * q);
    const u64 qlz = kFwdLazy * q;
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) {
        const int c = i * S::TB + tau;
        out[c] = reduce_any(acc[c] + qlz - v[i], q, one_sh);
    }
}

// P section, fused row kernel.  grid (2^LA/ROWS, jobs*K).
template <class S>
__global__ void __launch_bounds__(S::THREADS_B) k_oc_rowP(Tables T, OcJobs oj)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int K = T.kp;
    const OcJob &J = oj.job[blockIdx.y / K];
    const int k = blockIdx.y % K;
    const int nact = J.nact;
    const int t = nact + k;
    const int tf = T.nq + k;
    const int nt = nact + K;
    const int nfull = T.nq + K;
    const ModC &mc = T.modc[tf];
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    u64 *srow = sm + rr * S::ROWPAD;
    u64 *ab = sm + S::SMEM_B / 8 + rr * (1 << S::LB);
    u64 *aa = ab + RowSmem<S>::ACC;
    const int G = (1 << S::LA) + h;
    const size_t rowoff = (size_t)h << S::LB;
    const ulonglong2 *twt = T.tw + ((size_t)tf << S::LOGN);
    // the block's rows of one limb are one contiguous block of global memory
    const size_t brow = (size_t)blockIdx.x * S::ROWS << S::LB;
    constexpr uint32_t BLK = S::ROWS * (1 << S::LB) * 8;
    auto prefetch_digit = [&](int j) {
        prefetch_l2(J.tmp + ((size_t)(j * K + k) << S::LOGN) + brow, BLK);
        prefetch_l2(J.key.evk + ((size_t)((j * 2 + 0) * nfull + tf) << S::LOGN) + brow, BLK);
        prefetch_l2(J.key.evk + ((size_t)((j * 2 + 1) * nfull + tf) << S::LOGN) + brow, BLK);
    };
    if (threadIdx.x == 0) prefetch_digit(0);
    for (int j = 0; j < J.nd; ++j) {
        if (threadIdx.x == 0 && j + 1 < J.nd) prefetch_digit(j + 1);
        oc_digit<S>(J.tmp + ((size_t)(j * K + k) << S::LOGN) + rowoff, 1, twt, G, srow, tau,
                    J.key.evk + ((size_t)((j * 2 + 0) * nfull + tf) << S::LOGN) + rowoff,
                    J.key.evk + ((size_t)((j * 2 + 1) * nfull + tf) << S::LOGN) + rowoff, ab, aa, j == 0, mc.q, mc.mont);
    }
    const ulonglong2 *itwt = T.itw + ((size_t)tf << S::LOGN);
    oc_inv_store<S>(ab, itwt, G, srow, tau, J.cp + ((size_t)t << S::LOGN) + rowoff, mc.q);
    oc_inv_store<S>(aa, itwt, G, srow, tau, J.cp + ((size_t)(nt + t) << S::LOGN) + rowoff, mc.q);
}

// Q section, fused row kernel.  grid (2^LA/ROWS, sum of nact over jobs).
// tmp holds [nd + 2][nact] limbs: rows j < nd the ModUp limbs of digit j
// (the slot of the tower's own digit unused), rows nd and nd+1 the ModDown
// limbs of the two polynomials.
template <class S>
__global__ void __launch_bounds__(S::THREADS_B) k_oc_rowQ(Tables T, OcJobs oj)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int jb = find_slot(oj.pre, oj.n, blockIdx.y);
    const OcJob &J = oj.job[jb];
    const int t = blockIdx.y - oj.pre[jb];
    const int nact = J.nact;
    const int j0 = t / T.alpha;
    const int nfull = T.nq + T.kp;
    const ModC &mc = T.modc[t];
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    u64 *srow = sm + rr * S::ROWPAD;
    u64 *ab = sm + S::SMEM_B / 8 + rr * (1 << S::LB);
    u64 *aa = ab + RowSmem<S>::ACC;
    const int G = (1 << S::LA) + h;
    const size_t rowoff = (size_t)h << S::LB;
    const ulonglong2 *twt = T.tw + ((size_t)t << S::LOGN);
    const size_t brow = (size_t)blockIdx.x * S::ROWS << S::LB;
    constexpr uint32_t BLK = S::ROWS * (1 << S::LB) * 8;
    auto prefetch_digit = [&](int j) {
        const u64 *src = j == j0 ? J.d + ((size_t)t << S::LOGN) : J.tmp + ((size_t)(j * nact + t) << S::LOGN);
        prefetch_l2(src + brow, BLK);
        prefetch_l2(J.key.evk + ((size_t)((j * 2 + 0) * nfull + t) << S::LOGN) + brow, BLK);
        prefetch_l2(J.key.evk + ((size_t)((j * 2 + 1) * nfull + t) << S::LOGN) + brow, BLK);
    };
    if (threadIdx.x == 0) prefetch_digit(0);
    for (int j = 0; j < J.nd; ++j) {
        if (threadIdx.x == 0) {
            if (j + 1 < J.nd) {
                prefetch_digit(j + 1);
            } else {
                prefetch_l2(J.tmp + ((size_t)(J.nd * nact + t) << S::LOGN) + brow, BLK);
                prefetch_l2(J.tmp + ((size_t)((J.nd + 1) * nact + t) << S::LOGN) + brow, BLK);
            }
        }
        const u64 *gin = j == j0 ? J.d + ((size_t)t << S::LOGN) + rowoff
                                 : J.tmp + ((size_t)(j * nact + t) << S::LOGN) + rowoff;
        oc_digit<S>(gin, j != j0, twt, G, srow, tau, J.key.evk + ((size_t)((j * 2 + 0) * nfull + t) << S::LOGN) + rowoff,
                    J.key.evk + ((size_t)((j * 2 + 1) * nfull + t) << S::LOGN) + rowoff, ab, aa, j == 0, mc.q, mc.mont);
    }
    for (int xp = 0; xp < 2; ++xp)
        oc_down_store<S>(J.tmp + ((size_t)((J.nd + xp) * nact + t) << S::LOGN) + rowoff, twt, G, srow, tau,
                         xp == 0 ? ab : aa, (xp == 0 ? J.out0 : J.out1) + ((size_t)t << S::LOGN) + rowoff, mc.q,
                         mc.one_sh);
}

template <class S>
static void oc_rows_S(const Tables &T, const OcJobs &oj, bool p_section, cudaStream_t st)
{
    static std::atomic<uint64_t> attr{0};
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_oc_rowP<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowSmem<S>::BYTES);
        cudaFuncSetAttribute(k_oc_rowQ<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowSmem<S>::BYTES);
    });
    if (p_section)
        KS_LAUNCH(st, "oc_row_p",
                  k_oc_rowP<S><<<dim3((1 << S::LA) / S::ROWS, oj.n * T.kp), S::THREADS_B, RowSmem<S>::BYTES, st>>>(
                      T, oj));
    else
        KS_LAUNCH(st, "oc_row_q",
                  k_oc_rowQ<S><<<dim3((1 << S::LA) / S::ROWS, oj.pre[oj.n]), S::THREADS_B, RowSmem<S>::BYTES, st>>>(
                      T, oj));
}

static int oc_rows(const Tables &T, const OcJobs &oj, bool p_section, cudaStream_t st)
{
    switch (T.logN) {
    case 10: oc_rows_S<ShapeOf<10>::T>(T, oj, p_section, st); break;
    case 11: oc_rows_S<ShapeOf<11>::T>(T, oj, p_section, st); break;
    case 12: oc_rows_S<ShapeOf<12>::T>(T, oj, p_section, st); break;
    case 13: oc_rows_S<ShapeOf<13>::T>(T, oj, p_section, st); break;
    case 14: oc_rows_S<ShapeOf<14>::T>(T, oj, p_section, st); break;
    case 15: oc_rows_S<ShapeOf<15>::T>(T, oj, p_section, st); break;
    case 16: oc_rows_S<ShapeOf<16>::T>(T, oj, p_section, st); break;
    case 17: oc_rows_S<ShapeOf<17>::T>(T, oj, p_section, st); break;
    default: return fail(KS_EUNSUPPORTED, "logN outside 10..17");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string("OC row kernel launch: ") + cudaGetErrorString(e));
    return KS_OK;
}

// ------------------------------------------------------------------ split variant
// The same schedule with the row passes run by the plain row-pass kernel and
// the key product / ModDown subtraction by streaming combine kernels: more
// resident warps per SM than the fused row kernels, at the price of one more
// round trip of the section's limbs through L2/HBM.

// V consecutive coefficients per thread (V = 2: 16-byte loads and stores;
// limb bases and even coefficient indices keep them aligned).
template <int V>
__device__ __forceinline__ void ldv(const u64 *p, u64 (&o)[V])
{
    static_assert(V == 1 || V % 2 == 0, "one word or pairs");
    if constexpr (V == 1) {
        o[0] = *p;
    } else {
#pragma unroll
        for (int c = 0; c < V; c += 2) {
            const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p + c);
            o[c] = t.x;
            o[c + 1] = t.y;
        }
    }
}
template <int V>
__device__ __forceinline__ void stv(u64 *p, const u64 (&v)[V])
{
    static_assert(V == 1 || V % 2 == 0, "one word or pairs");
    if constexpr (V == 1) {
        *p = v[0];
    } else {
#pragma unroll
        for (int c = 0; c < V; c += 2) *reinterpret_cast<ulonglong2 *>(p + c) = make_ulonglong2(v[c], v[c + 1]);
    }
}
// key product of V coefficients: x * b_j and x * a_j added into sb, sa
template <bool CK, int V>
__device__ __forceinline__ void key_macv(const KeyView &K, int j, int t, size_t n, int nfull, int logN, u64 q,
                                         const u64 (&x)[V], U128 (&sb)[V], U128 (&sa)[V])
{
    const size_t N = (size_t)1 << logN;
    u64 kb[V], ka[V];
    if (CK && K.comp) {
        ldv<V>(K.evk + ((size_t)j * nfull + t) * N + n, kb);
        key_a_words<V>(K.a_seed, j, t, n, logN, nfull, q, ka);
    } else {
        ldv<V>(K.evk + ((size_t)(2 * j) * nfull + t) * N + n, kb);
        ldv<V>(K.evk + ((size_t)(2 * j + 1) * nfull + t) * N + n, ka);
    }
#pragma unroll
    for (int c = 0; c < V; ++c) {
        mac128(sb[c], x[c], kb[c]);
        mac128(sa[c], x[c], ka[c]);
    }
}

// the key words of V coefficients (regenerated a half for a compressed key)
template <bool CK, int V>
__device__ __forceinline__ void key_words(const KeyView &K, int j, int t, size_t n, int nfull, int logN, u64 q,
                                          u64 (&kb)[V], u64 (&ka)[V])
{
    const size_t N = (size_t)1 << logN;
    if (CK && K.comp) {
        ldv<V>(K.evk + ((size_t)j * nfull + t) * N + n, kb);
        key_a_words<V>(K.a_seed, j, t, n, logN, nfull, q, ka);
    } else {
        ldv<V>(K.evk + ((size_t)(2 * j) * nfull + t) * N + n, kb);
        ldv<V>(K.evk + ((size_t)(2 * j + 1) * nfull + t) * N + n, ka);
    }
}

static bool any_compressed(const OcJobs &oj)
{
    for (int i = 0; i < oj.n; ++i)
        if (oj.job[i].key.comp) return true;
    return false;
}

// P section combine: c'_{x,p_k} = sum_j NTT(z_{j,p_k}) * evk_{j,x,p_k} for
// every coefficient, written canonical to cp.  grid (N/(256V), jobs*K).
template <bool CK, int V>
__global__ void __launch_bounds__(256) k_oc_comb_p(Tables T, OcJobs oj)
{
    const int K = T.kp;
    const OcJob &J = oj.job[blockIdx.y / K];
    const int k = blockIdx.y % K;
    const int tf = T.nq + k;
    const int t = J.nact + k;
    const int nt = J.nact + K;
    const int nfull = T.nq + K;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[tf];
    U128 sb[V], sa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) sb[c] = sa[c] = U128{0, 0};
    for (int j = 0; j < J.nd; ++j) {
        u64 x[V];
        ldv<V>(J.tmp + (size_t)(j * K + k) * N + n, x);
        key_macv<CK, V>(J.key, j, tf, n, nfull, T.logN, mc.q, x, sb, sa);
    }
    u64 ob[V], oa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        ob[c] = reduce_any(redc(sb[c], mc.q, mc.mont), mc.q, mc.one_sh);
        oa[c] = key_a_finish<CK>(J.key, sa[c], mc, T.key_sc, tf);
    }
    stv<V>(J.cp + (size_t)t * N + n, ob);
    stv<V>(J.cp + (size_t)(nt + t) * N + n, oa);
}

// Q section combine: out_x = sum_j D_j * evk_{j,x} - NTT(v_x), D_j the
// transformed ModUp limb or the input tower for the own digit.
// grid (N/(256V), sum of nact over jobs).
template <bool CK, int V>
__global__ void __launch_bounds__(256) k_oc_comb_q(Tables T, OcJobs oj)
{
    const int jb = find_slot(oj.pre, oj.n, blockIdx.y);
    const OcJob &J = oj.job[jb];
    const int t = blockIdx.y - oj.pre[jb];
    const int nact = J.nact;
    const int j0 = t / T.alpha;
    const int nfull = T.nq + T.kp;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[t];
    U128 sb[V], sa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) sb[c] = sa[c] = U128{0, 0};
    for (int j = 0; j < J.nd; ++j) {
        u64 x[V];
        ldv<V>(j == j0 ? J.d + (size_t)t * N + n : J.tmp + (size_t)(j * nact + t) * N + n, x);
        key_macv<CK, V>(J.key, j, t, n, nfull, T.logN, mc.q, x, sb, sa);
    }
    u64 vb[V], va[V], o0[V], o1[V];
    ldv<V>(J.tmp + (size_t)(J.nd * nact + t) * N + n, vb);
    ldv<V>(J.tmp + (size_t)((J.nd + 1) * nact + t) * N + n, va);
    const u64 qlz = kFwdLazy * mc.q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
        const u64 cb = reduce_any(redc(sb[c], mc.q, mc.mont), mc.q, mc.one_sh);
        const u64 ca = key_a_finish<CK>(J.key, sa[c], mc, T.key_sc, t);
        o0[c] = reduce_any(cb + qlz - vb[c], mc.q, mc.one_sh);
        o1[c] = reduce_any(ca + qlz - va[c], mc.q, mc.one_sh);
    }
    stv<V>(J.out0 + (size_t)t * N + n, o0);
    stv<V>(J.out1 + (size_t)t * N + n, o1);
}

// ------------------------------------------------------------------ shared keys
// Combine kernels for jobs that share a key: one block reads each key word
// once and applies it to every job of its group (up to kGroupJobs), so a
// key's limbs cross HBM once per group instead of once per job.  Same
// arithmetic, per job, as the per-job kernels above.  Used when the
// schedule orders jobs by key.  On the 64-job mixed-level batch (16 keys),
// pairs at two coefficients a thread beat the per-job kernels at two (Q
// combine 0.99 against 1.08 ms) but not at four (8293 against 8329
// key-switches/s for the batch); groups of four were slower still, and
// pairs at four coefficients need 128 registers a thread.
constexpr int kGroupJobs = 2;  // jobs a block serves
constexpr int kGroupV = 2;     // coefficients a thread
struct KeyGroups {
    int n;                     // groups
    int pre[kMaxBatch + 1];    // Q-combine row blocks of group g: [pre[g], pre[g+1]) (largest nact)
    int first[kMaxBatch + 1];  // members of group g: mem[first[g] .. first[g+1])
    int mem[kMaxBatch];        // job indices into the launch's OcJobs
};

// Row n of the section's limbs: WHOLE = the whole-basis layout (D
// [nd][nact+K], then v [2][nact]); otherwise the split layout (P section D
// [nd][K]; Q section D [nd][nact], then v [2][nact]).
template <bool WHOLE>
__device__ __forceinline__ const u64 *p_limb(const OcJob &J, int j, int k, int K, size_t N)
{
    return WHOLE ? J.tmp + ((size_t)j * (J.nact + K) + J.nact + k) * N : J.tmp + ((size_t)j * K + k) * N;
}
template <bool WHOLE>
__device__ __forceinline__ const u64 *q_limb(const OcJob &J, int j, int t, int j0, int K, size_t N)
{
    if (j == j0) return J.d + (size_t)t * N;
    return J.tmp + ((size_t)j * (WHOLE ? J.nact + K : J.nact) + t) * N;
}
template <bool WHOLE>
__device__ __forceinline__ const u64 *v_limb(const OcJob &J, int x, int t, int K, size_t N)
{
    const size_t base = WHOLE ? (size_t)J.nd * (J.nact + K) : (size_t)J.nd * J.nact;
    return J.tmp + (base + (size_t)x * J.nact + t) * N;
}

// P towers.  grid (N/(256V), groups*K).
template <bool CK, bool WHOLE, int V>
__global__ void __launch_bounds__(256) k_oc_comb_pg(Tables T, OcJobs oj, KeyGroups kg)
{
    const int K = T.kp;
    const int g = blockIdx.y / K, k = blockIdx.y % K;
    const int m0 = kg.first[g], cnt = kg.first[g + 1] - m0;
    const KeyView key = oj.job[kg.mem[m0]].key;
    const int tf = T.nq + k;
    const int nfull = T.nq + K;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[tf];
    int ndm = 0;
    for (int i = 0; i < cnt; ++i) ndm = max(ndm, oj.job[kg.mem[m0 + i]].nd);
    U128 sb[kGroupJobs][V], sa[kGroupJobs][V];
#pragma unroll
    for (int i = 0; i < kGroupJobs; ++i)
#pragma unroll
        for (int c = 0; c < V; ++c) sb[i][c] = sa[i][c] = U128{0, 0};
    for (int j = 0; j < ndm; ++j) {
        u64 kb[V], ka[V];
        key_words<CK, V>(key, j, tf, n, nfull, T.logN, mc.q, kb, ka);
#pragma unroll
        for (int i = 0; i < kGroupJobs; ++i)
            if (i < cnt) {
                const OcJob &J = oj.job[kg.mem[m0 + i]];
                if (j < J.nd) {
                    u64 x[V];
                    ldv<V>(p_limb<WHOLE>(J, j, k, K, N) + n, x);
#pragma unroll
                    for (int c = 0; c < V; ++c) {
                        mac128(sb[i][c], x[c], kb[c]);
                        mac128(sa[i][c], x[c], ka[c]);
                    }
                }
            }
    }
#pragma unroll
    for (int i = 0; i < kGroupJobs; ++i)
        if (i < cnt) {
            const OcJob &J = oj.job[kg.mem[m0 + i]];
            const int t = J.nact + k, nt = J.nact + K;
            u64 ob[V], oa[V];
#pragma unroll
            for (int c = 0; c < V; ++c) {
                ob[c] = reduce_any(redc(sb[i][c], mc.q, mc.mont), mc.q, mc.one_sh);
                oa[c] = key_a_finish<CK>(key, sa[i][c], mc, T.key_sc, tf);
            }
            stv<V>(J.cp + (size_t)t * N + n, ob);
            stv<V>(J.cp + (size_t)(nt + t) * N + n, oa);
        }
}

// Q towers and the ModDown subtraction.  grid (N/(256V), kg.pre[kg.n]).
template <bool CK, bool WHOLE, int V>
__global__ void __launch_bounds__(256) k_oc_comb_qg(Tables T, OcJobs oj, KeyGroups kg)
{
    const int K = T.kp;
    const int g = find_slot(kg.pre, kg.n, blockIdx.y);
    const int t = blockIdx.y - kg.pre[g];
    const int m0 = kg.first[g], cnt = kg.first[g + 1] - m0;
    const KeyView key = oj.job[kg.mem[m0]].key;
    const int j0 = t / T.alpha;
    const int nfull = T.nq + K;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[t];
    int ndm = 0;
    for (int i = 0; i < cnt; ++i) {
        const OcJob &J = oj.job[kg.mem[m0 + i]];
        if (J.nact > t) ndm = max(ndm, J.nd);
    }
    U128 sb[kGroupJobs][V], sa[kGroupJobs][V];
#pragma unroll
    for (int i = 0; i < kGroupJobs; ++i)
#pragma unroll
        for (int c = 0; c < V; ++c) sb[i][c] = sa[i][c] = U128{0, 0};
    for (int j = 0; j < ndm; ++j) {
        u64 kb[V], ka[V];
        key_words<CK, V>(key, j, t, n, nfull, T.logN, mc.q, kb, ka);
#pragma unroll
        for (int i = 0; i < kGroupJobs; ++i)
            if (i < cnt) {
                const OcJob &J = oj.job[kg.mem[m0 + i]];
                if (J.nact > t && j < J.nd) {
                    u64 x[V];
                    ldv<V>(q_limb<WHOLE>(J, j, t, j0, K, N) + n, x);
#pragma unroll
                    for (int c = 0; c < V; ++c) {
                        mac128(sb[i][c], x[c], kb[c]);
                        mac128(sa[i][c], x[c], ka[c]);
                    }
                }
            }
    }
    const u64 qlz = kFwdLazy * mc.q;
#pragma unroll
    for (int i = 0; i < kGroupJobs; ++i)
        if (i < cnt) {
            const OcJob &J = oj.job[kg.mem[m0 + i]];
            if (J.nact > t) {
                u64 vb[V], va[V], o0[V], o1[V];
                ldv<V>(v_limb<WHOLE>(J, 0, t, K, N) + n, vb);
                ldv<V>(v_limb<WHOLE>(J, 1, t, K, N) + n, va);
#pragma unroll
                for (int c = 0; c < V; ++c) {
                    const u64 cb = reduce_any(redc(sb[i][c], mc.q, mc.mont), mc.q, mc.one_sh);
                    const u64 ca = key_a_finish<CK>(key, sa[i][c], mc, T.key_sc, t);
                    o0[c] = reduce_any(cb + qlz - vb[c], mc.q, mc.one_sh);
                    o1[c] = reduce_any(ca + qlz - va[c], mc.q, mc.one_sh);
                }
                stv<V>(J.out0 + (size_t)t * N + n, o0);
                stv<V>(J.out1 + (size_t)t * N + n, o1);
            }
        }
}

// Groups of jobs sharing a key (by stored key address), members in
// descending level, at most kGroupJobs each.  Returns false when no two jobs
// share a key (the per-job kernels are used then).
static bool key_groups(const OcJobs &oj, KeyGroups &kg)
{
    std::vector<std::vector<int>> by_key;
    std::vector<const u64 *> keys;
    for (int i = 0; i < oj.n; ++i) {
        const u64 *k = oj.job[i].key.evk;
        size_t at = 0;
        while (at < keys.size() && keys[at] != k) ++at;
        if (at == keys.size()) {
            keys.push_back(k);
            by_key.emplace_back();
        }
        by_key[at].push_back(i);
    }
    if ((int)keys.size() == oj.n) return false;
    kg.n = 0;
    kg.pre[0] = 0;
    kg.first[0] = 0;
    int m = 0;
    for (auto &members : by_key) {
        std::stable_sort(members.begin(), members.end(),
                         [&](int a, int b) { return oj.job[a].nact > oj.job[b].nact; });
        for (size_t s = 0; s < members.size(); s += kGroupJobs) {
            const size_t e = std::min(members.size(), s + kGroupJobs);
            int top = 0;
            for (size_t i = s; i < e; ++i) {
                kg.mem[m++] = members[i];
                top = std::max(top, oj.job[members[i]].nact);
            }
            kg.first[kg.n + 1] = m;
            kg.pre[kg.n + 1] = kg.pre[kg.n] + top;
            ++kg.n;
        }
    }
    return true;
}

template <bool WHOLE>
static void comb_grouped(const Tables &T, const OcJobs &oj, const KeyGroups &kg, bool p_section, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const bool ck = any_compressed(oj);
    constexpr int V = kGroupV;
    if (p_section) {
        const dim3 g((unsigned)(N / (256 * V)), kg.n * T.kp);
        if (ck)
            KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_pg<true, WHOLE, V><<<g, 256, 0, st>>>(T, oj, kg)));
        else
            KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_pg<false, WHOLE, V><<<g, 256, 0, st>>>(T, oj, kg)));
    } else {
        const dim3 g((unsigned)(N / (256 * V)), kg.pre[kg.n]);
        if (ck)
            KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_qg<true, WHOLE, V><<<g, 256, 0, st>>>(T, oj, kg)));
        else
            KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_qg<false, WHOLE, V><<<g, 256, 0, st>>>(T, oj, kg)));
    }
}

static int oc_combine(const Tables &T, const OcJobs &oj, bool p_section, bool share_keys, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    // Q towers: four coefficients a thread (two 16-byte accesses per
    // stream: 0.42 ms against 0.47 ms with two at the benchmark step); the
    // P-tower combine has few rows and keeps one (two measured slower)
    const dim3 gp((unsigned)(N / 256), oj.n * T.kp), gq((unsigned)(N / 1024), oj.pre[oj.n]);
    KeyGroups kg;
    if (share_keys && key_groups(oj, kg)) {
        comb_grouped<false>(T, oj, kg, p_section, st);
    } else if (p_section) {
        if (any_compressed(oj))
            KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_p<true, 1><<<gp, 256, 0, st>>>(T, oj)));
        else
            KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_p<false, 1><<<gp, 256, 0, st>>>(T, oj)));
    } else {
        if (any_compressed(oj))
            KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_q<true, 4><<<gq, 256, 0, st>>>(T, oj)));
        else
            KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_q<false, 4><<<gq, 256, 0, st>>>(T, oj)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string("OC combine launch: ") + cudaGetErrorString(e));
    return KS_OK;
}

size_t oc_scratch_words(const Tables &T, int nact)
{
    const size_t N = (size_t)1 << T.logN;
    const size_t nd = (size_t)(nact + T.alpha - 1) / T.alpha;
    const size_t tmp = nd * ((size_t)nact + T.kp) + 2 * (size_t)nact;
    return ((size_t)nact + tmp + 2 * ((size_t)nact + T.kp)) * N;
}

// Whole-basis variant: tmp holds D [nd][nact+K] then v [2][nact].
// P-tower combine of this layout: c'_{x,p_k} from D rows at tower nact+k.
// grid (N/(256V), jobs*K).
template <bool CK, int V>
__global__ void __launch_bounds__(256) k_oc_comb_pw(Tables T, OcJobs oj)
{
    const int K = T.kp;
    const OcJob &J = oj.job[blockIdx.y / K];
    const int k = blockIdx.y % K;
    const int tf = T.nq + k;
    const int t = J.nact + k;
    const int nt = J.nact + K;
    const int nfull = T.nq + K;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[tf];
    U128 sb[V], sa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) sb[c] = sa[c] = U128{0, 0};
    for (int j = 0; j < J.nd; ++j) {
        u64 x[V];
        ldv<V>(J.tmp + ((size_t)j * nt + t) * N + n, x);
        key_macv<CK, V>(J.key, j, tf, n, nfull, T.logN, mc.q, x, sb, sa);
    }
    u64 ob[V], oa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) {
        ob[c] = reduce_any(redc(sb[c], mc.q, mc.mont), mc.q, mc.one_sh);
        oa[c] = key_a_finish<CK>(J.key, sa[c], mc, T.key_sc, tf);
    }
    stv<V>(J.cp + (size_t)t * N + n, ob);
    stv<V>(J.cp + (size_t)(nt + t) * N + n, oa);
}

// Q-tower combine of the whole-basis layout.  grid (N/(256V), sum of nact).
// Four CTAs per SM (64 registers, a few spilled words): more loads in flight
// than three CTAs at the compiler's 74 registers (0.92 -> 0.95 of the copy
// bandwidth on the benchmark step).
template <bool CK, int V>
__global__ void __launch_bounds__(256, 4) k_oc_comb_qw(Tables T, OcJobs oj)
{
    const int jb = find_slot(oj.pre, oj.n, blockIdx.y);
    const OcJob &J = oj.job[jb];
    const int t = blockIdx.y - oj.pre[jb];
    const int nact = J.nact;
    const int nt = nact + T.kp;
    const int j0 = t / T.alpha;
    const int nfull = T.nq + T.kp;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    const ModC &mc = T.modc[t];
    U128 sb[V], sa[V];
#pragma unroll
    for (int c = 0; c < V; ++c) sb[c] = sa[c] = U128{0, 0};
    for (int j = 0; j < J.nd; ++j) {
        u64 x[V];
        ldv<V>(j == j0 ? J.d + (size_t)t * N + n : J.tmp + ((size_t)j * nt + t) * N + n, x);
        key_macv<CK, V>(J.key, j, t, n, nfull, T.logN, mc.q, x, sb, sa);
    }
    const u64 *v = J.tmp + (size_t)J.nd * nt * N;
    u64 vb[V], va[V], o0[V], o1[V];
    ldv<V>(v + (size_t)t * N + n, vb);
    ldv<V>(v + (size_t)(nact + t) * N + n, va);
    const u64 qlz = kFwdLazy * mc.q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
        const u64 cb = reduce_any(redc(sb[c], mc.q, mc.mont), mc.q, mc.one_sh);
        const u64 ca = key_a_finish<CK>(J.key, sa[c], mc, T.key_sc, t);
        o0[c] = reduce_any(cb + qlz - vb[c], mc.q, mc.one_sh);
        o1[c] = reduce_any(ca + qlz - va[c], mc.q, mc.one_sh);
    }
    stv<V>(J.out0 + (size_t)t * N + n, o0);
    stv<V>(J.out1 + (size_t)t * N + n, o1);
}

static int launch_oc_whole(const Tables &T, int n, const OcJob *jobs, bool share_keys, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const int K = T.kp;
    int rc;
    LimbMaps m1, mD, mw, mv;
    m1.n = mD.n = mw.n = mv.n = 0;
    BUpJobs bu;
    bu.n = 0;
    BDnJobs bd;
    bd.n = 0;
    OcJobs oj;
    oj.n = n;
    oj.pre[0] = 0;
    for (int i = 0; i < n; ++i) {
        const OcJob &J = jobs[i];
        const int nt = J.nact + K;
        add_map(m1, LimbMap{J.d, J.y, J.pre, J.nact, 0, 0, 0, J.nact, -1}, J.nact);
        add_bup(bu, T, BUpJob{J.y, J.tmp, (size_t)nt * N, J.nact, 0, nt, 0, -1});
        add_map(mD, LimbMap{J.tmp, J.tmp, nullptr, nt, nt, 0, 0, J.nact, 0}, J.nd * nt);
        add_map(mw, LimbMap{J.cp, J.cp, nullptr, K, nt, J.nact, J.nact, J.nact, -1}, 2 * K);
        u64 *v = J.tmp + (size_t)J.nd * nt * N;
        add_bdn(bd, BDnJob{J.cp, (size_t)nt * N, v, (size_t)J.nact * N, J.nact, 2});
        add_map(mv, LimbMap{v, v, nullptr, J.nact, J.nact, 0, 0, J.nact, -1}, 2 * J.nact);
        oj.job[i] = J;
        oj.pre[i + 1] = oj.pre[i] + J.nact;
    }
    if ((rc = launch_ntt_inv(T, m1, false, st)) != KS_OK) return rc;   // ModUp P1
    if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;          // P2, every tower
    if ((rc = launch_ntt_fwd(T, mD, false, st)) != KS_OK) return rc;    // P3
    const bool ck = any_compressed(oj);
    KeyGroups kg;
    const bool grouped = share_keys && key_groups(oj, kg);
    // Q towers four coefficients a thread, P towers one (as in oc_combine)
    const dim3 gp((unsigned)(N / 256), n * K), gq((unsigned)(N / 1024), oj.pre[n]);
    if (grouped)  // P4+P5, P towers
        comb_grouped<true>(T, oj, kg, true, st);
    else if (ck)
        KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_pw<true, 1><<<gp, 256, 0, st>>>(T, oj)));
    else
        KS_LAUNCH(st, "oc_comb_p", (k_oc_comb_pw<false, 1><<<gp, 256, 0, st>>>(T, oj)));
    if ((rc = launch_ntt_inv(T, mw, false, st)) != KS_OK) return rc;    // ModDown P1
    if ((rc = launch_bconv_down(T, bd, st)) != KS_OK) return rc;        // ModDown P2
    if ((rc = launch_ntt_fwd(T, mv, false, st)) != KS_OK) return rc;    // ModDown P3
    if (grouped)  // P4+P5 Q, ModDown P4
        comb_grouped<true>(T, oj, kg, false, st);
    else if (ck)
        KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_qw<true, 4><<<gq, 256, 0, st>>>(T, oj)));
    else
        KS_LAUNCH(st, "oc_comb_q", (k_oc_comb_qw<false, 4><<<gq, 256, 0, st>>>(T, oj)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string("OC whole-basis launch: ") + cudaGetErrorString(e));
    return KS_OK;
}

static int launch_oc_chunk(const Tables &T, int n, const OcJob *jobs, int variant, bool share_keys, cudaStream_t st)
{
    if (variant == KS_OC_WHOLE) return launch_oc_whole(T, n, jobs, share_keys, st);
    const size_t N = (size_t)1 << T.logN;
    const int K = T.kp;
    int rc;
    // 1. prep (ModUp P1)
    LimbMaps m1;
    m1.n = 0;
    for (int i = 0; i < n; ++i) {
        const OcJob &J = jobs[i];
        add_map(m1, LimbMap{J.d, J.y, J.pre, J.nact, 0, 0, 0, J.nact, -1}, J.nact);
    }
    if ((rc = launch_ntt_inv(T, m1, false, st)) != KS_OK) return rc;
    // 2. P section
    BUpJobs bp;
    bp.n = 0;
    LimbMaps mp, mw;
    mp.n = 0;
    mw.n = 0;
    OcJobs oj;
    oj.n = n;
    oj.pre[0] = 0;
    for (int i = 0; i < n; ++i) {
        const OcJob &J = jobs[i];
        const int nt = J.nact + K;
        add_bup(bp, T, BUpJob{J.y, J.tmp, (size_t)K * N, J.nact, J.nact, nt, J.nact, -1});
        add_map(mp, LimbMap{J.tmp, J.tmp, nullptr, K, K, 0, J.nact, J.nact, -1}, J.nd * K);
        add_map(mw, LimbMap{J.cp, J.cp, nullptr, K, nt, J.nact, J.nact, J.nact, -1}, 2 * K);
        oj.job[i] = J;
        oj.pre[i + 1] = oj.pre[i] + J.nact;
    }
    if ((rc = launch_bconv_up(T, bp, st)) != KS_OK) return rc;
    if (variant == KS_OC_FUSED) {
        if ((rc = launch_fwd_col(T, mp, st)) != KS_OK) return rc;
        if ((rc = oc_rows(T, oj, true, st)) != KS_OK) return rc;
        if ((rc = launch_inv_col(T, mw, false, st)) != KS_OK) return rc;
    } else {
        if ((rc = launch_ntt_fwd(T, mp, false, st)) != KS_OK) return rc;
        if ((rc = oc_combine(T, oj, true, share_keys, st)) != KS_OK) return rc;
        if ((rc = launch_ntt_inv(T, mw, false, st)) != KS_OK) return rc;
    }
    // 3. Q section: one cluster kernel per output tower (TOWER), else the
    // split or fused form below
    if (variant == KS_OC_TOWER) {
        rc = launch_oc_tower(T, oj, st);
        if (rc != KS_EUNSUPPORTED) return rc;
    }
    BUpJobs bq;
    bq.n = 0;
    BDnJobs bd;
    bd.n = 0;
    LimbMaps mq;
    mq.n = 0;
    for (int i = 0; i < n; ++i) {
        const OcJob &J = jobs[i];
        const int nt = J.nact + K;
        add_bup(bq, T, BUpJob{J.y, J.tmp, (size_t)J.nact * N, J.nact, 0, J.nact, 0, -1});
        add_bdn(bd, BDnJob{J.cp, (size_t)nt * N, J.tmp + (size_t)J.nd * J.nact * N, (size_t)J.nact * N, J.nact, 2});
        add_map(mq, LimbMap{J.tmp, J.tmp, nullptr, J.nact, J.nact, 0, 0, J.nact, 0}, (J.nd + 2) * J.nact);
    }
    if ((rc = launch_bconv_up(T, bq, st)) != KS_OK) return rc;
    if ((rc = launch_bconv_down(T, bd, st)) != KS_OK) return rc;
    if (variant == KS_OC_FUSED) {
        if ((rc = launch_fwd_col(T, mq, st)) != KS_OK) return rc;
        return oc_rows(T, oj, false, st);
    }
    if ((rc = launch_ntt_fwd(T, mq, false, st)) != KS_OK) return rc;
    return oc_combine(T, oj, false, share_keys, st);
}

int launch_oc(const Tables &T, int njobs, const OcJob *jobs, int variant, cudaStream_t st, bool share_keys)
{
    // The tower kernel needs a ring degree with a cluster geometry and full
    // keys; otherwise its launch group runs the split variant (same result).
    if (variant == KS_OC_TOWER) {
        bool ok = oc_tower_supported(T);
        for (int i = 0; i < njobs && ok; ++i) ok = !jobs[i].key.comp;
        if (!ok) variant = KS_OC_SPLIT;
    }
    // The fused row kernels read the key's a half from memory: batches with
    // a compressed key run the split variant instead.
    if (variant == KS_OC_FUSED)
        for (int i = 0; i < njobs; ++i)
            if (jobs[i].key.comp) {
                variant = KS_OC_SPLIT;
                break;
            }
    for (int i0 = 0; i0 < njobs; i0 += kMaxBatch) {
        int rc = launch_oc_chunk(T, std::min(kMaxBatch, njobs - i0), jobs + i0, variant, share_keys, st);
        if (rc != KS_OK) return rc;
    }
    return KS_OK;
}

}  // namespace ks
