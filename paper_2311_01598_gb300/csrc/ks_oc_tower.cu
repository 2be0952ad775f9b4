// ks_oc_tower.cu -- Output-Centric key switching, one output tower on chip
// (CiFlow Sec. IV-C).
//
// The Output-Centric dataflow computes the key-switch output tower by tower:
// for output tower t everything that feeds it -- the base conversion of the
// other digits to t (ModUp P2), their NTTs (P3), the key product summed over
// digits (P4+P5), the base conversion of the special part w to t (ModDown
// P2), its NTT (P3) and the subtraction (P4) -- is done while the tower's
// data stays on chip, and the key limbs of t are streamed from memory once.
//
// GPU form: one thread-block cluster of C CTAs per (job, Q tower t), C the
// cluster NTT's geometry (16 CTAs of 256 threads at N = 2^16).  A limb of t
// is spread over the cluster: CTA r holds columns [r*COLS, (r+1)*COLS) for
// the column pass and rows [r*ROWS, (r+1)*ROWS) for the row pass, the rows
// gathered from the other CTAs' shared memory (distributed shared memory)
// between the passes.  Per CTA:
//   * the key product accumulators of its rows (both polynomials) live in
//     shared memory for the whole kernel;
//   * bypassed digit (the one holding t): the input tower d_t, already in
//     evaluation form, goes straight into the key product;
//   * every other digit j: base conversion of y_j (coefficient form, read
//     from L2) to t for the CTA's columns, column pass, cluster exchange,
//     row pass, key product;
//   * ModDown, for each polynomial: base conversion of w (the special
//     section's output) to t for the CTA's columns, column pass, exchange,
//     row pass, subtraction from the accumulator, output written.
// Only y and w (read from L2, shared by all towers of the job), the key rows
// and the input/output rows touch memory; the raised limbs and the ModDown
// limbs of t never do.  The butterflies, base-conversion arithmetic and key
// product are those of the other kernels, so outputs are bit-identical.
#include "ks_cluster.cuh"

namespace ks {

namespace {

template <class S>
struct TowerShape {
    typedef Cl<S, 1> G;
    static constexpr bool OK = G::OK;
    static constexpr int ACCW = G::ROWS << S::LB;  // words of one accumulator (the CTA's rows)
    static constexpr int CONSTS = kMaxQ > kMaxP ? kMaxQ : kMaxP;
    static constexpr int SMEM = G::SMEM + 2 * ACCW * 8 + CONSTS * 8;
};

// x * e (e a stored key word, Montgomery form with the tower's fold factor):
// REDC of the 128-bit product; x below kFwdLazy*q gives a result below 2q.
__device__ __forceinline__ u64 key_prod(u64 x, u64 e, u64 q, u64 mont)
{
    U128 t = {0, 0};
    mac128(t, x, e);
    return reduce2(redc(t, q, mont), q);
}

// Forward NTT of one limb of tower t spread over the cluster.  Enters with
// xc[k] = element (row k*TA + tauc, column c) of the CTA's column block
// (below 4q) and leaves with xr[k] = element k*TB + tau of row h (below
// kFwdLazy*q).  Contains block and cluster barriers: every thread of every CTA of
// the cluster calls it.
template <class S>
__device__ __forceinline__ void tower_ntt(u64 (&xc)[S::REGA], u64 (&xr)[S::REGB], u64 *buf,
                                          const ulonglong2 *tws, const ulonglong2 *tsh, const ulonglong2 *twt,
                                          int G, int cc, int tauc, int rr, int tau, int h, u64 q, u64 q2)
{
    typedef Cl<S, 1> G_;
    constexpr int COLS = G_::COLS;
    fwd_round1<S::RA>(xc, TwSmem{tws}, q, q2);
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) buf[(k * S::TA + tauc) * COLS + cc] = xc[k];
    __syncthreads();
    constexpr int M = S::TA, NG = S::REGA / S::TA;
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) xc[gg * M + k2] = buf[((tauc * NG + gg) * M + k2) * COLS + cc];
    fwd_round2<S::LA, S::RA>(xc, tauc * NG, TwSmem{tws}, q, q2);
    __syncthreads();  // every read of the transpose precedes the block's writes
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) buf[((tauc * NG + gg) * M + k2) * COLS + cc] = xc[gg * M + k2];
    cluster_barrier();  // every CTA's column block is complete
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) {
        const int c = k * S::TB + tau;
        xr[k] = ld_dsmem(dsmem_addr(buf + h * COLS + c % COLS, c / COLS));
    }
    cluster_barrier();  // no CTA reads another's block after this point
    row_fwd_core<S>(xr, TwStaged<S>{tsh, twt, G}, buf + rr * S::ROWPAD, tau, q, q2);
}

// Base conversion at the CTA's column positions: xc[k] = sum_i src_i[n] *
// cst[i] for n = (row k*TA + tauc, column c), i < nsrc, reduced once into
// [0, 2q) (Montgomery: the constants carry 2^64).  The sources' loads of one
// i are issued together (REGA independent loads in flight per thread).
template <class S>
__device__ __forceinline__ void tower_bconv(u64 (&xc)[S::REGA], const u64 *src, int nsrc, const u64 *cst, int c,
                                            int tauc, const ModC &mc)
{
    const size_t N = (size_t)1 << S::LOGN;
    BAcc A[S::REGA];
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) bacc_zero(A[k]);
    for (int i = 0; i < nsrc; ++i) {
        const u64 *s = src + (size_t)i * N + c;
        const u64 ci = cst[i];
        u64 v[S::REGA];
#pragma unroll
        for (int k = 0; k < S::REGA; ++k) v[k] = s[(size_t)(k * S::TA + tauc) << S::LB];
#pragma unroll
        for (int k = 0; k < S::REGA; ++k) {
            u32 y0, y1;
            split_y(v[k], y0, y1);
            bacc_mac(A[k], y0, y1, ci);
        }
    }
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) xc[k] = bacc_reduce(A[k], mc);
}

// grid (C, sum of nact over jobs), cluster (C, 1, 1): every CTA of a
// cluster has the same (job, tower), so all control flow below is uniform
// over the cluster.  Full keys only (the launcher checks).
template <class S>
__global__ void __launch_bounds__(Cl<S, 1>::THREADS, 2) k_oc_tower(Tables T, OcJobs oj)
{
    typedef Cl<S, 1> G_;
    typedef TowerShape<S> TS;
    constexpr int COLS = G_::COLS, ROWS = G_::ROWS, THREADS = G_::THREADS;
    constexpr int LBW = 1 << S::LB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *buf = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(buf + G_::BUFW);
    ulonglong2 *tsh_all = tws + (1 << S::LA);
    u64 *accb = reinterpret_cast<u64 *>(tsh_all + ROWS * S::REGB);
    u64 *acca = accb + TS::ACCW;
    u64 *cst = acca + TS::ACCW;  // base-conversion constants of the current digit (or of ModDown)

    const int jb = find_slot(oj.pre, oj.n, blockIdx.y);
    const OcJob &J = oj.job[jb];
    const int t = blockIdx.y - oj.pre[jb];
    const int nact = J.nact, K = T.kp;
    const int nt = nact + K, nfull = T.nq + K;
    const int alpha = T.alpha, j0 = t / alpha;
    const ModC &mc = T.modc[t];
    const u64 q = mc.q, q2 = 2 * q;
    const size_t N = (size_t)1 << S::LOGN;
    const int r = cluster_rank();
    const ulonglong2 *twt = T.tw + ((size_t)t << S::LOGN);

    // column-pass coordinates: column c, rows k*TA + tauc
    const int cc = threadIdx.x % COLS, tauc = threadIdx.x / COLS;
    const int c = r * COLS + cc;
    // row-pass coordinates: row h, elements k*TB + tau
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = r * ROWS + rr;
    const int G = (1 << S::LA) + h;
    ulonglong2 *tsh = tsh_all + rr * S::REGB;
    const size_t rowoff = (size_t)h << S::LB;
    u64 *ab = accb + rr * LBW, *aa = acca + rr * LBW;

    // the key rows of this CTA for every active digit are prefetched into L2
    // up front (one contiguous block per limb)
    if (threadIdx.x == 0) {
        const size_t brow = (size_t)r * ROWS << S::LB;
        constexpr uint32_t BLK = ROWS * LBW * 8;
        for (int j = 0; j < J.nd; ++j) {
            prefetch_l2(J.key.evk + ((size_t)((2 * j) * nfull + t) << S::LOGN) + brow, BLK);
            prefetch_l2(J.key.evk + ((size_t)((2 * j + 1) * nfull + t) << S::LOGN) + brow, BLK);
        }
    }
    // twiddles of tower t: the column pass's (shared by the whole CTA) and
    // the first round of each row (shared by every NTT of this kernel)
    for (int i = threadIdx.x; i < (1 << S::LA); i += THREADS) tws[i] = twt[i];
    stage_row_round1<S>(tsh, twt, G, tau);

    // bypassed digit: D = d_t (evaluation form), the accumulators' first term
    {
        const u64 *dr = J.d + ((size_t)t << S::LOGN) + rowoff;
        const u64 *eb = J.key.evk + ((size_t)((2 * j0) * nfull + t) << S::LOGN) + rowoff;
        const u64 *ea = J.key.evk + ((size_t)((2 * j0 + 1) * nfull + t) << S::LOGN) + rowoff;
#pragma unroll
        for (int k = 0; k < S::REGB; ++k) {
            const int e = k * S::TB + tau;
            const u64 x = dr[e];
            ab[e] = key_prod(x, __ldg(eb + e), q, mc.mont);
            aa[e] = key_prod(x, __ldg(ea + e), q, mc.mont);
        }
    }

    // One loop over the phases that need a base conversion and an NTT: the
    // non-bypassed digits (ModUp), then the two polynomials' ModDown limbs.
    // A single copy of the base-conversion and NTT code keeps the kernel
    // within the instruction cache (two inlined copies stalled on
    // instruction fetch).
    u64 xc[S::REGA], xr[S::REGB];
    const int nup = J.nd - 1;
    const u64 qlz = kFwdLazy * q;
    for (int p = 0; p < nup + 2; ++p) {
        const bool down = p >= nup;
        const int j = down ? 0 : (p < j0 ? p : p + 1);
        const int x = down ? p - nup : 0;
        const u64 *src;
        int nsrc;
        __syncthreads();  // the previous phase's reads of cst are done
        if (!down) {
            const int lo = j * alpha;
            nsrc = min(alpha, nact - lo);
            const u64 *mat = T.up_mat + T.up_mat_lvl[(size_t)(nact - 1) * T.ndig + j];
            for (int i = threadIdx.x; i < nsrc; i += THREADS) cst[i] = mat[(size_t)i * nfull + t];
            src = J.y + (size_t)lo * N;
        } else {
            nsrc = K;
            for (int k = threadIdx.x; k < K; k += THREADS) cst[k] = T.dn_mat[(size_t)k * T.nq + t];
            src = J.cp + ((size_t)x * nt + nact) * N;
        }
        __syncthreads();
        // base conversion to t at the CTA's column positions, then the NTT
        tower_bconv<S>(xc, src, nsrc, cst, c, tauc, mc);
        tower_ntt<S>(xc, xr, buf, tws, tsh, twt, G, cc, tauc, rr, tau, h, q, q2);
        if (!down) {
            // key product of digit j added into the accumulators
            const u64 *eb = J.key.evk + ((size_t)((2 * j) * nfull + t) << S::LOGN) + rowoff;
            const u64 *ea = J.key.evk + ((size_t)((2 * j + 1) * nfull + t) << S::LOGN) + rowoff;
#pragma unroll
            for (int k = 0; k < S::REGB; ++k) {
                const int e = k * S::TB + tau;
                ab[e] = reduce2(ab[e] + key_prod(xr[k], __ldg(eb + e), q, mc.mont), q);
                aa[e] = reduce2(aa[e] + key_prod(xr[k], __ldg(ea + e), q, mc.mont), q);
            }
        } else {
            // ModDown P4: out_x = c'_x - NTT(v_x)
            const u64 *acc = x == 0 ? ab : aa;
            u64 *out = (x == 0 ? J.out0 : J.out1) + ((size_t)t << S::LOGN) + rowoff;
#pragma unroll
            for (int k = 0; k < S::REGB; ++k) {
                const int e = k * S::TB + tau;
                out[e] = reduce_any(acc[e] + qlz - xr[k], q, mc.one_sh);
            }
        }
    }
}

template <class S>
struct TowerKernel {
    // per device: attributes set and the cluster shape accepted
    static bool ready()
    {
        if constexpr (!TowerShape<S>::OK) {
            return false;
        } else {
            static std::atomic<uint64_t> done{0}, ok{0};
            once_per_device(done, [] {
                const bool r = cluster_prepare(k_oc_tower<S>, Cl<S, 1>::C, Cl<S, 1>::THREADS, TowerShape<S>::SMEM);
                int dev = 0;
                if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
                if (r) ok.fetch_or(1ull << (dev & 63));
            });
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
            return (ok.load() >> (dev & 63)) & 1;
        }
    }
};

template <class S>
int tower_S(const Tables &T, const OcJobs &oj, cudaStream_t st)
{
    if constexpr (!TowerShape<S>::OK) {
        return KS_EUNSUPPORTED;
    } else {
        if (!TowerKernel<S>::ready()) return KS_EUNSUPPORTED;
        typedef Cl<S, 1> G_;
        const int items = oj.pre[oj.n];
        if (items == 0) return KS_OK;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)G_::C, (unsigned)items, 1);
        cfg.blockDim = dim3((unsigned)G_::THREADS, 1, 1);
        cfg.dynamicSmemBytes = (size_t)TowerShape<S>::SMEM;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)G_::C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e;
        KS_LAUNCH(st, "oc_tower", e = cudaLaunchKernelEx(&cfg, k_oc_tower<S>, T, oj));
        if (e != cudaSuccess) return fail(KS_ECUDA, std::string("OC tower launch: ") + cudaGetErrorString(e));
        return KS_OK;
    }
}

template <class S>
bool tower_ready_S()
{
    return TowerKernel<S>::ready();
}

}  // namespace

bool oc_tower_supported(const Tables &T)
{
    switch (T.logN) {
    case 10: return tower_ready_S<ShapeOf<10>::T>();
    case 11: return tower_ready_S<ShapeOf<11>::T>();
    case 12: return tower_ready_S<ShapeOf<12>::T>();
    case 13: return tower_ready_S<ShapeOf<13>::T>();
    case 14: return tower_ready_S<ShapeOf<14>::T>();
    case 15: return tower_ready_S<ShapeOf<15>::T>();
    case 16: return tower_ready_S<ShapeOf<16>::T>();
    case 17: return tower_ready_S<ShapeOf<17>::T>();
    default: return false;
    }
}

int launch_oc_tower(const Tables &T, const OcJobs &oj, cudaStream_t st)
{
    for (int i = 0; i < oj.n; ++i)
        if (oj.job[i].key.comp) return KS_EUNSUPPORTED;
    switch (T.logN) {
    case 10: return tower_S<ShapeOf<10>::T>(T, oj, st);
    case 11: return tower_S<ShapeOf<11>::T>(T, oj, st);
    case 12: return tower_S<ShapeOf<12>::T>(T, oj, st);
    case 13: return tower_S<ShapeOf<13>::T>(T, oj, st);
    case 14: return tower_S<ShapeOf<14>::T>(T, oj, st);
    case 15: return tower_S<ShapeOf<15>::T>(T, oj, st);
    case 16: return tower_S<ShapeOf<16>::T>(T, oj, st);
    case 17: return tower_S<ShapeOf<17>::T>(T, oj, st);
    default: return KS_EUNSUPPORTED;
    }
}

}  // namespace ks
