// ks_ntt_cluster.cu -- one-launch NTT over thread-block clusters.
//
// The two-pass NTT (ks_kernels.cu) runs its column and row passes as two
// launches, the limb going through L2/HBM in between.  Here one cluster of C
// CTAs transforms one limb in a single launch: CTA r runs the column pass on
// columns [r*COLS, (r+1)*COLS) and keeps its block in shared memory; after a
// cluster barrier it gathers rows [r*ROWS, (r+1)*ROWS) from the blocks of all
// C CTAs through distributed shared memory and runs the row pass.  The
// inverse runs the row pass first and gathers columns.  The butterflies,
// twiddles and value ranges are those of the two-pass kernels, so the outputs
// are bit-identical to theirs.
//
// Shared memory per CTA: one buffer (the CTA's block of the limb, the column
// pass's transpose, then the row buffers), the column twiddles and the staged
// first-round row twiddles: 42 KB at N = 2^16.  A second cluster barrier
// after the gather frees the buffer for reuse and keeps every CTA alive while
// others read its block.
#include "ks_cluster.cuh"

namespace ks {

namespace {

// Forward NTT (input below 4q; output canonical with CANON, else below kFwdLazy*q).
// grid (C, limbs), cluster (C, 1, 1): every CTA of a cluster has the same
// limb, so the early exits below are uniform over the cluster.
template <class S, int MUL, bool CANON>
__global__ void __launch_bounds__(Cl<S, MUL>::THREADS, Cl<S, MUL>::MINB) k_fwd_cl(Tables T, LimbMaps ms)
{
    typedef Cl<S, MUL> G_;
    constexpr int COLS = G_::COLS, ROWS = G_::ROWS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *buf = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(buf + G_::BUFW);
    ulonglong2 *tsh_all = tws + (1 << S::LA);
    const int lg = blockIdx.y + blockIdx.z * gridDim.y;
    if (lg >= ms.pre[ms.n]) return;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const ModC &mc = T.modc[L.tf];
    const u64 q = mc.q, q2 = 2 * q;
    const int r = cluster_rank();
    const ulonglong2 *twt = T.tw + ((size_t)L.tf << S::LOGN);
    {
        // column pass on this CTA's columns; the block stays in buf as
        // buf[h*COLS + cc] (row h, column r*COLS + cc)
        for (int i = threadIdx.x; i < (1 << S::LA); i += G_::THREADS) tws[i] = twt[i];
        const int cc = threadIdx.x % COLS, tau = threadIdx.x / COLS;
        const int c = r * COLS + cc;
        u64 x[S::REGA];
#pragma unroll
        for (int k = 0; k < S::REGA; ++k) x[k] = L.src[((size_t)(k * S::TA + tau) << S::LB) + c];
        __syncthreads();
        fwd_round1<S::RA>(x, TwSmem{tws}, q, q2);
#pragma unroll
        for (int k = 0; k < S::REGA; ++k) buf[(k * S::TA + tau) * COLS + cc] = x[k];
        __syncthreads();
        constexpr int M = S::TA, NG = S::REGA / S::TA;
#pragma unroll
        for (int gg = 0; gg < NG; ++gg)
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) x[gg * M + k2] = buf[((tau * NG + gg) * M + k2) * COLS + cc];
        fwd_round2<S::LA, S::RA>(x, tau * NG, TwSmem{tws}, q, q2);
        __syncthreads();  // every read of the transpose precedes the block's writes
#pragma unroll
        for (int gg = 0; gg < NG; ++gg)
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) buf[((tau * NG + gg) * M + k2) * COLS + cc] = x[gg * M + k2];
    }
    cluster_barrier();  // every CTA's block is complete
    // row pass on rows [r*ROWS, (r+1)*ROWS): element c of row h lives in
    // CTA c / COLS at buf[h*COLS + c % COLS]
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = r * ROWS + rr;
    const int G = (1 << S::LA) + h;
    u64 x[S::REGB];
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) {
        const int c = k * S::TB + tau;
        x[k] = ld_dsmem(dsmem_addr(buf + h * COLS + c % COLS, c / COLS));
    }
    ulonglong2 *tsh = tsh_all + rr * S::REGB;
    stage_row_round1<S>(tsh, twt, G, tau);
    cluster_barrier();  // no CTA reads another's block after this point
    row_fwd_core<S>(x, TwStaged<S>{tsh, twt, G}, buf + rr * S::ROWPAD, tau, q, q2);
    u64 *gout = L.dst + ((size_t)h << S::LB);
    const u64 one_sh = CANON ? mc.one_sh : 0;
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) gout[k * S::TB + tau] = CANON ? reduce_any(x[k], q, one_sh) : x[k];
}

// Inverse NTT (input below 4q), then the scale (SC: 0 none, 1 the job's
// per-entry scale, 2 N^-1); output canonical.
template <class S, int MUL, int SC>
__global__ void __launch_bounds__(Cl<S, MUL>::THREADS, Cl<S, MUL>::MINB) k_inv_cl(Tables T, LimbMaps ms)
{
    typedef Cl<S, MUL> G_;
    constexpr int COLS = G_::COLS, ROWS = G_::ROWS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *buf = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(buf + G_::BUFW);
    const int lg = blockIdx.y + blockIdx.z * gridDim.y;
    if (lg >= ms.pre[ms.n]) return;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const ModC &mc = T.modc[L.tf];
    const u64 q = mc.q, q2 = 2 * q;
    const int r = cluster_rank();
    const ulonglong2 *itw = T.itw + ((size_t)L.tf << S::LOGN);
    for (int i = threadIdx.x; i < (1 << S::LA); i += G_::THREADS) tws[i] = itw[i];
    {
        // row pass on rows [r*ROWS, (r+1)*ROWS); the block stays in buf as
        // buf[(h - r*ROWS) * 2^LB + c]
        const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
        const int h = r * ROWS + rr;
        const TwRow tw{itw, (1 << S::LA) + h};
        const u64 *gin = L.src + ((size_t)h << S::LB);
        u64 x[S::REGB];
#pragma unroll
        for (int k = 0; k < S::REGB; ++k) x[k] = gin[k * S::TB + tau];
        row_inv_core<S>(x, tw, buf + rr * S::ROWPAD, tau, q, q2);  // ends with buf free
#pragma unroll
        for (int k = 0; k < S::REGB; ++k) buf[rr * (1 << S::LB) + k * S::TB + tau] = x[k];
    }
    cluster_barrier();  // every CTA's block (and tws) is complete
    // column pass on columns [r*COLS, (r+1)*COLS): row h lives in CTA h / ROWS
    const int cc = threadIdx.x % COLS, tau = threadIdx.x / COLS;
    const int c = r * COLS + cc;
    constexpr int M = S::TA, NG = S::REGA / S::TA;
    u64 x[S::REGA];
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
            const int h = (tau * NG + gg) * M + k2;
            x[gg * M + k2] = ld_dsmem(dsmem_addr(buf + (h % ROWS) * (1 << S::LB) + c, h / ROWS));
        }
    cluster_barrier();  // no CTA reads another's block after this point
    inv_round2<S::LA, S::RA>(x, tau * NG, TwSmem{tws}, q, q2);
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) buf[((tau * NG + gg) * M + k2) * COLS + cc] = x[gg * M + k2];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) x[k] = buf[(k * S::TA + tau) * COLS + cc];
    inv_round1<S::RA>(x, TwSmem{tws}, q, q2);
    u64 w = 0, wp = 0;
    if (SC == 1) {
        const ulonglong2 f = L.scale[L.b];
        w = f.x;
        wp = f.y;
    } else if (SC == 2) {
        w = mc.ninv;
        wp = mc.ninv_sh;
    }
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) {
        u64 v = x[k];
        if (SC != 0) v = shoup_lazy(v, w, wp, q);
        L.dst[((size_t)(k * S::TA + tau) << S::LB) + c] = reduce4(v, q, q2);
    }
}

template <class S, int MUL>
struct ClKernels {
    typedef Cl<S, MUL> G;
    // per device: attributes set and the cluster shape accepted
    static bool ready()
    {
        static std::atomic<uint64_t> done{0}, ok{0};
        once_per_device(done, [] {
            bool r = true;
            r = r && cluster_prepare(k_fwd_cl<S, MUL, false>, G::C, G::THREADS, G::SMEM);
            r = r && cluster_prepare(k_fwd_cl<S, MUL, true>, G::C, G::THREADS, G::SMEM);
            r = r && cluster_prepare(k_inv_cl<S, MUL, 0>, G::C, G::THREADS, G::SMEM);
            r = r && cluster_prepare(k_inv_cl<S, MUL, 1>, G::C, G::THREADS, G::SMEM);
            r = r && cluster_prepare(k_inv_cl<S, MUL, 2>, G::C, G::THREADS, G::SMEM);
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
            if (r) ok.fetch_or(1ull << (dev & 63));
        });
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
        return (ok.load() >> (dev & 63)) & 1;
    }
};

template <class KERN>
static cudaError_t launch_cluster(KERN kern, int C, int threads, int smem, int limbs, const Tables &T,
                                  const LimbMaps &m, cudaStream_t st)
{
    const unsigned gy = (unsigned)std::min(limbs, 32768);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, gy, (unsigned)((limbs + (int)gy - 1) / (int)gy));
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, T, m);
}

// Returns KS_EUNSUPPORTED (nothing launched) when the shape or the device
// cannot run the cluster form.
template <class S, int MUL>
static int fwd_cl_SM(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st)
{
    typedef Cl<S, MUL> G;
    if constexpr (!G::OK) {
        return KS_EUNSUPPORTED;
    } else {
        if (!ClKernels<S, MUL>::ready()) return KS_EUNSUPPORTED;
        cudaError_t e;
        const int limbs = m.pre[m.n];
        if (canonical)
            KS_LAUNCH(st, "ntt_fwd_cl",
                      e = launch_cluster(k_fwd_cl<S, MUL, true>, G::C, G::THREADS, G::SMEM, limbs, T, m, st));
        else
            KS_LAUNCH(st, "ntt_fwd_cl",
                      e = launch_cluster(k_fwd_cl<S, MUL, false>, G::C, G::THREADS, G::SMEM, limbs, T, m, st));
        if (e != cudaSuccess) return fail(KS_ECUDA, std::string("cluster NTT launch: ") + cudaGetErrorString(e));
        return KS_OK;
    }
}

template <class S, int MUL>
static int inv_cl_SM(const Tables &T, const LimbMaps &m, int sc, cudaStream_t st)
{
    typedef Cl<S, MUL> G;
    if constexpr (!G::OK) {
        return KS_EUNSUPPORTED;
    } else {
        if (!ClKernels<S, MUL>::ready()) return KS_EUNSUPPORTED;
        cudaError_t e;
        const int limbs = m.pre[m.n];
        constexpr int C = G::C, TH = G::THREADS, SM = G::SMEM;
        if (sc == 1)
            KS_LAUNCH(st, "ntt_inv_cl", e = launch_cluster(k_inv_cl<S, MUL, 1>, C, TH, SM, limbs, T, m, st));
        else if (sc == 2)
            KS_LAUNCH(st, "ntt_inv_cl", e = launch_cluster(k_inv_cl<S, MUL, 2>, C, TH, SM, limbs, T, m, st));
        else
            KS_LAUNCH(st, "ntt_inv_cl", e = launch_cluster(k_inv_cl<S, MUL, 0>, C, TH, SM, limbs, T, m, st));
        if (e != cudaSuccess) return fail(KS_ECUDA, std::string("cluster NTT launch: ") + cudaGetErrorString(e));
        return KS_OK;
    }
}

// T.ntt_cluster: 1 = CTAs of the two-pass size, 2 = CTAs twice as wide
template <class S>
static int fwd_cl_S(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st)
{
    return T.ntt_cluster == 2 ? fwd_cl_SM<S, 2>(T, m, canonical, st) : fwd_cl_SM<S, 1>(T, m, canonical, st);
}
template <class S>
static int inv_cl_S(const Tables &T, const LimbMaps &m, int sc, cudaStream_t st)
{
    return T.ntt_cluster == 2 ? inv_cl_SM<S, 2>(T, m, sc, st) : inv_cl_SM<S, 1>(T, m, sc, st);
}

#define KS_CL_DISPATCH(logN, FN, ...)                         \
    switch (logN) {                                           \
    case 10: return FN<ShapeOf<10>::T>(__VA_ARGS__);          \
    case 11: return FN<ShapeOf<11>::T>(__VA_ARGS__);          \
    case 12: return FN<ShapeOf<12>::T>(__VA_ARGS__);          \
    case 13: return FN<ShapeOf<13>::T>(__VA_ARGS__);          \
    case 14: return FN<ShapeOf<14>::T>(__VA_ARGS__);          \
    case 15: return FN<ShapeOf<15>::T>(__VA_ARGS__);          \
    case 16: return FN<ShapeOf<16>::T>(__VA_ARGS__);          \
    case 17: return FN<ShapeOf<17>::T>(__VA_ARGS__);          \
    default: return KS_EUNSUPPORTED;                          \
    }

}  // namespace

bool ntt_cluster_shape(int logN)
{
    switch (logN) {
    case 10: return Cl<ShapeOf<10>::T, 1>::OK;
    case 11: return Cl<ShapeOf<11>::T, 1>::OK;
    case 12: return Cl<ShapeOf<12>::T, 1>::OK;
    case 13: return Cl<ShapeOf<13>::T, 1>::OK;
    case 14: return Cl<ShapeOf<14>::T, 1>::OK;
    case 15: return Cl<ShapeOf<15>::T, 1>::OK;
    case 16: return Cl<ShapeOf<16>::T, 1>::OK;
    case 17: return Cl<ShapeOf<17>::T, 1>::OK;
    default: return false;
    }
}

int launch_ntt_fwd_cluster(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st)
{
    KS_CL_DISPATCH(T.logN, fwd_cl_S, T, m, canonical, st);
}

int launch_ntt_inv_cluster(const Tables &T, const LimbMaps &m, int sc, cudaStream_t st)
{
    KS_CL_DISPATCH(T.logN, inv_cl_S, T, m, sc, st);
}

}  // namespace ks
