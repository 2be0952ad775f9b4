// ks_kernels.cu -- NTT passes and the per-stage kernels of hybrid key
// switching (CiFlow Sec. III: ModUp P1-P5, ModDown P1-P4).  Stage launches
// take per-job descriptor tables (ks_launch.h), so one launch covers every
// job of a batch.  The Output-Centric fused kernels live in ks_oc.cu.
#include <algorithm>

#include "ks_ntt_core.cuh"

namespace ks {

// ------------------------------------------------------------------ NTT passes
// Forward column pass (stages 0..LA-1).  grid (2^LB/COLS, limbs).  SP: every
// modulus has the special form q1*2^32 + 1 (cheaper butterfly product).
template <class S, bool SP>
__global__ void __launch_bounds__(S::THREADS_A, S::MINB_A) k_fwd_col(Tables T, LimbMaps ms)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(sm + (1 << S::LA) * S::COLS);
    const int lg = blockIdx.y + blockIdx.z * gridDim.y;
    if (lg >= ms.pre[ms.n]) return;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const u64 q = T.modc[L.tf].q, q2 = 2 * q;
    const ulonglong2 *twt = T.tw + ((size_t)L.tf << S::LOGN);
    for (int i = threadIdx.x; i < (1 << S::LA); i += S::THREADS_A) tws[i] = twt[i];
    const int cc = threadIdx.x % S::COLS, tau = threadIdx.x / S::COLS;
    const int c = blockIdx.x * S::COLS + cc;
    u64 x[S::REGA];
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) x[k] = L.src[((size_t)(k * S::TA + tau) << S::LB) + c];
    __syncthreads();
    fwd_round1<S::RA, SP>(x, TwSmem{tws}, q, q2);
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) sm[(k * S::TA + tau) * S::COLS + cc] = x[k];
    __syncthreads();
    constexpr int M = S::TA, NG = S::REGA / S::TA;
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) x[gg * M + k2] = sm[((tau * NG + gg) * M + k2) * S::COLS + cc];
    fwd_round2<S::LA, S::RA, SP>(x, tau * NG, TwSmem{tws}, q, q2);
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) L.dst[((size_t)((tau * NG + gg) * M + k2) << S::LB) + c] = x[gg * M + k2];
}

// Forward row pass (stages LA..logN-1).  grid (2^LA/ROWS, limbs).  Output
// canonical (CANON) or lazy below kFwdLazy*q.  Loads and stores are coalesced (a
// second shared-memory exchange returns the values to the first-round
// layout; measured faster than storing each thread's consecutive values
// with strided vector stores).
template <class S, bool CANON, bool SP>
__global__ void __launch_bounds__(S::THREADS_B, S::MINB_B) k_fwd_row(Tables T, LimbMaps ms)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int lz = blockIdx.y + blockIdx.z * gridDim.y;
    if (lz >= ms.pre[ms.n]) return;
    // limbs in reverse order: the column pass wrote the last ones most
    // recently, so the first blocks find their rows in L2
    const int lg = ms.pre[ms.n] - 1 - lz;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const ModC &mc = T.modc[L.tf];
    const u64 q = mc.q, q2 = 2 * q;
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    const int G = (1 << S::LA) + h;
    const ulonglong2 *twt = T.tw + ((size_t)L.tf << S::LOGN);
    ulonglong2 *tsh = reinterpret_cast<ulonglong2 *>(sm + S::ROWS * S::ROWPAD) + rr * S::REGB;
    const u64 *gin = L.src + ((size_t)h << S::LB);
    u64 *gout = L.dst + ((size_t)h << S::LB);
    u64 x[S::REGB];
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) x[k] = gin[k * S::TB + tau];
    stage_row_round1<S>(tsh, twt, G, tau);
    static_assert(S::TB <= 32, "a row's threads share one warp");
    __syncwarp();
    row_fwd_core<S, SP>(x, TwStaged<S>{tsh, twt, G}, sm + rr * S::ROWPAD, tau, q, q2);
    const u64 one_sh = CANON ? mc.one_sh : 0;
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) gout[k * S::TB + tau] = CANON ? reduce_any(x[k], q, one_sh) : x[k];
}

// ------------------------------------------------------------------ staged row pass
// Forward row pass with its row blocks staged in shared memory by the bulk
// copy engine (TMA, one 1-D cp.async.bulk of ROWS contiguous rows per item).
// Persistent CTAs of ROWS rows walk the launch's row blocks (item b = limb
// b / (2^LA/ROWS), row block b % (2^LA/ROWS)) with stride gridDim.x: the
// next item's rows are copied into the second buffer while the current item
// is transformed, so the loads of a block overlap the butterflies of the
// previous one instead of stalling its warps.  A buffer, once its values are
// in registers, is the item's row-exchange buffer.  Same butterflies,
// twiddles and output as k_fwd_row.
__device__ int g_ntt_error;  // set when a staged load's wait gives up
constexpr int kStageWaitLimit = 1 << 22;

template <class S>
struct StagedRow {
    static constexpr int ROWW = S::ROWS * (1 << S::LB);  // words of one row block
    static constexpr int BUFW = ROWW > S::ROWS * S::ROWPAD ? ROWW : S::ROWS * S::ROWPAD;
    static constexpr int BYTES = ROWW * 8;
    static constexpr int SMEM = 2 * BUFW * 8 + S::ROWS * S::REGB * 16 + 16;
};

__device__ __forceinline__ bool stage_wait(uint32_t mbar, uint32_t phase)
{
    uint32_t done = 0;
    for (int it = 0; it < kStageWaitLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
    return done != 0;
}

// First item >= b whose limb is transformed (bypassed digit limbs are skipped).
template <class S>
__device__ __forceinline__ int staged_next(const Tables &T, const LimbMaps &ms, int b, int total, int nblk)
{
    for (; b < total; b += gridDim.x)
        if (!limb_ref(ms, b / nblk, T.nq, T.alpha, S::LOGN).skip) return b;
    return total;
}

template <class S>
__device__ __forceinline__ void staged_issue(const Tables &T, const LimbMaps &ms, int b, int nblk, u64 *dst,
                                             uint32_t mbar)
{
    const LimbRef L = limb_ref(ms, b / nblk, T.nq, T.alpha, S::LOGN);
    const u64 *src = L.src + (((size_t)(b % nblk) * S::ROWS) << S::LB);
    // the buffer was last read through the generic proxy: order those reads
    // before the copy engine's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"((uint32_t)StagedRow<S>::BYTES)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(dst)),
        "l"(src), "r"((uint32_t)StagedRow<S>::BYTES), "r"(mbar)
        : "memory");
}

// 12 resident CTAs per SM (18 KB of shared memory each at 2^16): at most 85
// registers a thread.
template <class S, bool CANON>
__global__ void __launch_bounds__(S::THREADS_B, 12) k_fwd_row_st(Tables T, LimbMaps ms)
{
    typedef StagedRow<S> SR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *buf0 = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tsh_all = reinterpret_cast<ulonglong2 *>(buf0 + 2 * SR::BUFW);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tsh_all + S::ROWS * S::REGB);
    constexpr int nblk = (1 << S::LA) / S::ROWS;
    const int total = ms.pre[ms.n] * nblk;
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    const uint32_t mb1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int b = staged_next<S>(T, ms, blockIdx.x, total, nblk);
    if (b < total && threadIdx.x == 0) staged_issue<S>(T, ms, b, nblk, buf0, mb0);
    uint32_t phase = 0;  // bit k: parity of buffer k's next completion
    int cur = 0;
    bool ok = true;
    while (b < total) {
        const int nb = staged_next<S>(T, ms, b + gridDim.x, total, nblk);
        // the other buffer's last reader (the previous item) finished at its
        // final block barrier
        if (nb < total && threadIdx.x == 0) staged_issue<S>(T, ms, nb, nblk, buf0 + (cur ^ 1) * SR::BUFW, cur ? mb0 : mb1);
        u64 *sb = buf0 + cur * SR::BUFW;
        if (!stage_wait(cur ? mb1 : mb0, (phase >> cur) & 1)) {
            ok = false;
            break;
        }
        phase ^= 1u << cur;
        const LimbRef L = limb_ref(ms, b / nblk, T.nq, T.alpha, S::LOGN);
        const ModC &mc = T.modc[L.tf];
        const u64 q = mc.q, q2 = 2 * q;
        const int h = (b % nblk) * S::ROWS + rr;
        const int G = (1 << S::LA) + h;
        const ulonglong2 *twt = T.tw + ((size_t)L.tf << S::LOGN);
        ulonglong2 *tsh = tsh_all + rr * S::REGB;
        u64 x[S::REGB];
#pragma unroll
        for (int k = 0; k < S::REGB; ++k) x[k] = sb[rr * (1 << S::LB) + k * S::TB + tau];
        stage_row_round1<S>(tsh, twt, G, tau);
        __syncthreads();  // every row is in registers before the buffer becomes the exchange buffer
        row_fwd_core<S>(x, TwStaged<S>{tsh, twt, G}, sb + rr * S::ROWPAD, tau, q, q2);
        u64 *gout = L.dst + ((size_t)h << S::LB);
        const u64 one_sh = CANON ? mc.one_sh : 0;
#pragma unroll
        for (int k = 0; k < S::REGB; ++k) gout[k * S::TB + tau] = CANON ? reduce_any(x[k], q, one_sh) : x[k];
        b = nb;
        cur ^= 1;
    }
    if (!ok && threadIdx.x == 0) {
        atomicExch(&g_ntt_error, 1);
        // bounded waits for the copies still in flight before the CTA exits
        stage_wait(mb0, phase & 1);
        stage_wait(mb1, (phase >> 1) & 1);
    }
}

int ntt_error_flag(bool clear)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ntt_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_ntt_error, &z, sizeof(int));
    }
    return v;
}

// Inverse row pass (stages logN-1..LA), first half of the iNTT.  Input below
// 4q; output below 4q.
template <class S, bool SP>
__global__ void __launch_bounds__(S::THREADS_B, S::MINB_B) k_inv_row(Tables T, LimbMaps ms)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int lg = blockIdx.y + blockIdx.z * gridDim.y;
    if (lg >= ms.pre[ms.n]) return;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const u64 q = T.modc[L.tf].q, q2 = 2 * q;
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    const int G = (1 << S::LA) + h;
    const ulonglong2 *itwt = T.itw + ((size_t)L.tf << S::LOGN);
    ulonglong2 *tsh = reinterpret_cast<ulonglong2 *>(sm + S::ROWS * S::ROWPAD) + rr * S::REGB;
    const u64 *gin = L.src + ((size_t)h << S::LB);
    u64 *gout = L.dst + ((size_t)h << S::LB);
    u64 x[S::REGB];
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) x[k] = gin[k * S::TB + tau];
    // the last round's twiddles (common to the row) staged beside the loads,
    // as in the forward row pass; the block barriers of the first round
    // order them before their use
    stage_row_round1<S>(tsh, itwt, G, tau);
    row_inv_core<S, SP>(x, TwStaged<S>{tsh, itwt, G}, sm + rr * S::ROWPAD, tau, q, q2);
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) gout[k * S::TB + tau] = x[k];
}

// Inverse column pass (stages LA-1..0), second half of the iNTT, then the
// scale (SC: 0 none, 1 the job's per-entry scale, 2 N^-1); output canonical.
template <class S, int SC, bool SP>
__global__ void __launch_bounds__(S::THREADS_A, S::MINB_A) k_inv_col(Tables T, LimbMaps ms)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(sm + (1 << S::LA) * S::COLS);
    const int lz = blockIdx.y + blockIdx.z * gridDim.y;
    if (lz >= ms.pre[ms.n]) return;
    // limbs in reverse order: the row pass wrote the last ones most recently
    const int lg = ms.pre[ms.n] - 1 - lz;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, S::LOGN);
    if (L.skip) return;
    const ModC &mc = T.modc[L.tf];
    const u64 q = mc.q, q2 = 2 * q;
    const ulonglong2 *twt = T.itw + ((size_t)L.tf << S::LOGN);
    for (int i = threadIdx.x; i < (1 << S::LA); i += S::THREADS_A) tws[i] = twt[i];
    const int cc = threadIdx.x % S::COLS, tau = threadIdx.x / S::COLS;
    const int c = blockIdx.x * S::COLS + cc;
    constexpr int M = S::TA, NG = S::REGA / S::TA;
    u64 x[S::REGA];
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) x[gg * M + k2] = L.src[((size_t)((tau * NG + gg) * M + k2) << S::LB) + c];
    __syncthreads();
    inv_round2<S::LA, S::RA, SP>(x, tau * NG, TwSmem{tws}, q, q2);
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) sm[((tau * NG + gg) * M + k2) * S::COLS + cc] = x[gg * M + k2];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::REGA; ++k) x[k] = sm[(k * S::TA + tau) * S::COLS + cc];
    inv_round1<S::RA, SP>(x, TwSmem{tws}, q, q2);
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

template <class S, bool SP>
static void set_smem_attrs_sp()
{
    cudaFuncSetAttribute(k_fwd_col<S, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_A);
    cudaFuncSetAttribute(k_inv_col<S, 0, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_A);
    cudaFuncSetAttribute(k_inv_col<S, 1, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_A);
    cudaFuncSetAttribute(k_inv_col<S, 2, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_A);
    cudaFuncSetAttribute(k_fwd_row<S, true, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_BT);
    cudaFuncSetAttribute(k_fwd_row<S, false, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_BT);
    cudaFuncSetAttribute(k_inv_row<S, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_BT);
}

template <class S>
static void set_smem_attrs()
{
    static std::atomic<uint64_t> done{0};  // per instantiation, per device
    once_per_device(done, [] {
        set_smem_attrs_sp<S, false>();
        set_smem_attrs_sp<S, true>();
    });
}

static int launch_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return KS_OK;
}

// Grid over a limb set: the limb index is blockIdx.y + blockIdx.z*gridDim.y
// (grid y and z are limited to 65535 each).
static dim3 limb_grid(unsigned gx, int limbs)
{
    const unsigned gy = (unsigned)std::min(limbs, 32768);
    return dim3(gx, gy, (unsigned)((limbs + gy - 1) / gy));
}

static bool any_scale(const LimbMaps &ms)
{
    for (int j = 0; j < ms.n; ++j)
        if (ms.m[j].scale) return true;
    return false;
}

template <class S>
static void fwd_col_S(const Tables &T, const LimbMaps &m, cudaStream_t st)
{
    set_smem_attrs<S>();
    const dim3 ga = limb_grid((1 << S::LB) / S::COLS, m.pre[m.n]);
    if (T.spq)
        KS_LAUNCH(st, "ntt_fwd_col", k_fwd_col<S, true><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
    else
        KS_LAUNCH(st, "ntt_fwd_col", k_fwd_col<S, false><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
}

// Persistent grid of the staged row pass: resident CTAs per SM x SMs, at
// most one CTA per item.
template <class S, bool CANON>
static int staged_grid(int items)
{
    static std::atomic<uint64_t> done{0};
    static int per_sm[64] = {0}, sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    once_per_device(done, [dev] {
        cudaFuncSetAttribute(k_fwd_row_st<S, CANON>, cudaFuncAttributeMaxDynamicSharedMemorySize, StagedRow<S>::SMEM);
        int n = 0, c = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fwd_row_st<S, CANON>, S::THREADS_B,
                                                          StagedRow<S>::SMEM) != cudaSuccess ||
            cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
            c = 1;
        }
        per_sm[dev & 63] = std::max(1, n);
        sms[dev & 63] = std::max(1, c);
    });
    return std::max(1, std::min(items, per_sm[dev & 63] * sms[dev & 63]));
}

template <class S>
static void fwd_row_S(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st)
{
    set_smem_attrs<S>();
    // the bulk copies need 16-byte aligned sources (row blocks of an aligned
    // limb are); maps over caller buffers that are not run the plain pass
    bool aligned = true;
    for (int j = 0; j < m.n; ++j) aligned = aligned && (((uintptr_t)m.m[j].src & 15) == 0);
    if (T.row_stage && aligned) {
        const int items = m.pre[m.n] * ((1 << S::LA) / S::ROWS);
        if (canonical)
            KS_LAUNCH(st, "ntt_fwd_row",
                      k_fwd_row_st<S, true><<<staged_grid<S, true>(items), S::THREADS_B, StagedRow<S>::SMEM, st>>>(T, m));
        else
            KS_LAUNCH(st, "ntt_fwd_row",
                      k_fwd_row_st<S, false><<<staged_grid<S, false>(items), S::THREADS_B, StagedRow<S>::SMEM, st>>>(T,
                                                                                                                   m));
        return;
    }
    const dim3 gb = limb_grid((1 << S::LA) / S::ROWS, m.pre[m.n]);
    if (canonical && T.spq)
        KS_LAUNCH(st, "ntt_fwd_row", k_fwd_row<S, true, true><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
    else if (canonical)
        KS_LAUNCH(st, "ntt_fwd_row", k_fwd_row<S, true, false><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
    else if (T.spq)
        KS_LAUNCH(st, "ntt_fwd_row", k_fwd_row<S, false, true><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
    else
        KS_LAUNCH(st, "ntt_fwd_row", k_fwd_row<S, false, false><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
}

template <class S>
static void inv_row_S(const Tables &T, const LimbMaps &m, cudaStream_t st)
{
    set_smem_attrs<S>();
    const dim3 gb = limb_grid((1 << S::LA) / S::ROWS, m.pre[m.n]);
    if (T.spq)
        KS_LAUNCH(st, "ntt_inv_row", k_inv_row<S, true><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
    else
        KS_LAUNCH(st, "ntt_inv_row", k_inv_row<S, false><<<gb, S::THREADS_B, S::SMEM_BT, st>>>(T, m));
}

template <class S>
static void inv_col_S(const Tables &T, const LimbMaps &m, bool ninv, cudaStream_t st)
{
    set_smem_attrs<S>();
    const dim3 ga = limb_grid((1 << S::LB) / S::COLS, m.pre[m.n]);
    const int sc = any_scale(m) ? 1 : ninv ? 2 : 0;
    if (T.spq) {
        if (sc == 1)
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 1, true><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
        else if (sc == 2)
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 2, true><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
        else
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 0, true><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
    } else {
        if (sc == 1)
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 1, false><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
        else if (sc == 2)
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 2, false><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
        else
            KS_LAUNCH(st, "ntt_inv_col", k_inv_col<S, 0, false><<<ga, S::THREADS_A, S::SMEM_A, st>>>(T, m));
    }
}

#define KS_DISPATCH_LOGN(logN, FN, ...)                                                                   \
    switch (logN) {                                                                                       \
    case 10: FN<ShapeOf<10>::T>(__VA_ARGS__); break;                                                      \
    case 11: FN<ShapeOf<11>::T>(__VA_ARGS__); break;                                                      \
    case 12: FN<ShapeOf<12>::T>(__VA_ARGS__); break;                                                      \
    case 13: FN<ShapeOf<13>::T>(__VA_ARGS__); break;                                                      \
    case 14: FN<ShapeOf<14>::T>(__VA_ARGS__); break;                                                      \
    case 15: FN<ShapeOf<15>::T>(__VA_ARGS__); break;                                                      \
    case 16: FN<ShapeOf<16>::T>(__VA_ARGS__); break;                                                      \
    case 17: FN<ShapeOf<17>::T>(__VA_ARGS__); break;                                                      \
    default: return fail(KS_EUNSUPPORTED, "logN outside 10..17");                                         \
    }

LimbMaps one_map(const LimbMap &m, int nlimbs)
{
    LimbMaps ms;
    ms.n = 0;
    ms.pre[0] = 0;
    add_map(ms, m, nlimbs);
    return ms;
}

void add_map(LimbMaps &ms, const LimbMap &m, int nlimbs)
{
    if (ms.n == 0) ms.pre[0] = 0;
    ms.m[ms.n] = m;
    ms.pre[ms.n + 1] = ms.pre[ms.n] + nlimbs;
    ms.n += 1;
}

int launch_fwd_col(const Tables &T, const LimbMaps &m, cudaStream_t st)
{
    if (m.n == 0 || m.pre[m.n] == 0) return KS_OK;
    KS_DISPATCH_LOGN(T.logN, fwd_col_S, T, m, st);
    return launch_status("forward column pass launch");
}

int launch_inv_col(const Tables &T, const LimbMaps &m, bool scale_by_ninv, cudaStream_t st)
{
    if (m.n == 0 || m.pre[m.n] == 0) return KS_OK;
    KS_DISPATCH_LOGN(T.logN, inv_col_S, T, m, scale_by_ninv, st);
    return launch_status("inverse column pass launch");
}

int launch_ntt_fwd(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st)
{
    if (m.n == 0 || m.pre[m.n] == 0) return KS_OK;
    if (T.ntt_cluster) {
        const int rc = launch_ntt_fwd_cluster(T, m, canonical, st);
        if (rc != KS_EUNSUPPORTED) return rc;
    }
    KS_DISPATCH_LOGN(T.logN, fwd_col_S, T, m, st);
    LimbMaps m2 = m;
    for (int j = 0; j < m2.n; ++j) m2.m[j].src = m2.m[j].dst;
    KS_DISPATCH_LOGN(T.logN, fwd_row_S, T, m2, canonical, st);
    return launch_status("forward NTT launch");
}

int launch_ntt_inv(const Tables &T, const LimbMaps &m, bool scale_by_ninv, cudaStream_t st)
{
    if (m.n == 0 || m.pre[m.n] == 0) return KS_OK;
    if (T.ntt_cluster) {
        const int rc = launch_ntt_inv_cluster(T, m, any_scale(m) ? 1 : scale_by_ninv ? 2 : 0, st);
        if (rc != KS_EUNSUPPORTED) return rc;
    }
    KS_DISPATCH_LOGN(T.logN, inv_row_S, T, m, st);
    LimbMaps m2 = m;
    for (int j = 0; j < m2.n; ++j) m2.m[j].src = m2.m[j].dst;
    KS_DISPATCH_LOGN(T.logN, inv_col_S, T, m2, scale_by_ninv, st);
    return launch_status("inverse NTT launch");
}

// ------------------------------------------------------------------ BConv
constexpr int BC_TT = 8;  // target towers per block
constexpr int BC_THREADS = 256;
// Both base-conversion kernels ask for 4 CTAs/SM (64 registers a thread): the
// extra warps hide the source loads better than the few spilled words cost.

void add_bup(BUpJobs &b, const Tables &T, const BUpJob &j)
{
    if (b.n == 0) b.zpre[0] = 0;
    const int nd = j.jsel >= 0 ? 1 : (j.nact + T.alpha - 1) / T.alpha;
    b.job[b.n] = j;
    b.zpre[b.n + 1] = b.zpre[b.n] + nd;
    b.n += 1;
}

// ModUp P2: grid (N/256, ceil(max targets/TT), digit blocks of all jobs).
__global__ void __launch_bounds__(BC_THREADS, 4) k_bconv_up(Tables T, BUpJobs bj)
{
    __shared__ u64 cs[kMaxQ][BC_TT];
    __shared__ int s_t[BC_TT];
    __shared__ int s_tf[BC_TT];
    const int jb = find_slot(bj.zpre, bj.n, blockIdx.z);
    const BUpJob &J = bj.job[jb];
    const int nact = J.nact;
    const int j = J.jsel >= 0 ? J.jsel : (int)blockIdx.z - bj.zpre[jb];
    const int lo = j * T.alpha;
    const int hi = min(lo + T.alpha, nact);
    const int a = hi - lo;
    const int olo = max(lo, J.t_begin), ohi = min(hi, J.t_end);
    const int ov = ohi > olo ? ohi - olo : 0;
    const int nb = (J.t_end - J.t_begin) - ov;
    const int u0 = blockIdx.y * BC_TT;
    if (u0 >= nb) return;
    const int nfull = T.nq + T.kp;
    const u64 *mat = T.up_mat + T.up_mat_lvl[(size_t)(nact - 1) * T.ndig + j];
    if (threadIdx.x < BC_TT) {
        const int u = min(u0 + (int)threadIdx.x, nb - 1);
        int t = J.t_begin + u;
        if (ov > 0 && t >= olo) t += ov;
        s_t[threadIdx.x] = t;
        s_tf[threadIdx.x] = full_tower(t, nact, T.nq);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < a * BC_TT; idx += blockDim.x) {
        const int i = idx / BC_TT, g = idx % BC_TT;
        cs[i][g] = (u0 + g < nb) ? mat[(size_t)i * nfull + s_tf[g]] : 0;
    }
    __syncthreads();
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    BAcc acc[BC_TT];
#pragma unroll
    for (int g = 0; g < BC_TT; ++g) bacc_zero(acc[g]);
    // sources in groups of four: the loads of a group are issued together
    int i = 0;
    for (; i + 4 <= a; i += 4) {
        u64 yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) yv[u] = J.y[(size_t)(lo + i + u) * N + n];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            u32 y0, y1;
            split_y(yv[u], y0, y1);
#pragma unroll
            for (int g = 0; g < BC_TT; ++g) bacc_mac(acc[g], y0, y1, cs[i + u][g]);
        }
    }
    for (; i < a; ++i) {
        u32 y0, y1;
        split_y(J.y[(size_t)(lo + i) * N + n], y0, y1);
#pragma unroll
        for (int g = 0; g < BC_TT; ++g) bacc_mac(acc[g], y0, y1, cs[i][g]);
    }
    u64 *Dj = J.D + (size_t)(J.jsel >= 0 ? 0 : j) * J.dstride;
#pragma unroll
    for (int g = 0; g < BC_TT; ++g) {
        if (u0 + g < nb) Dj[(size_t)(s_t[g] - J.t_base) * N + n] = bacc_reduce(acc[g], T.modc[s_tf[g]]);
    }
}

int launch_bconv_up(const Tables &T, const BUpJobs &b, cudaStream_t st)
{
    if (b.n == 0) return KS_OK;
    if (T.up_tc && bconv_tc_supported(T, T.alpha)) return launch_bconv_up_tc(T, b, T.up_tc, T.up_tc_lvl, st);
    int span = 0;
    for (int i = 0; i < b.n; ++i) span = std::max(span, b.job[i].t_end - b.job[i].t_begin);
    if (span <= 0) return KS_OK;
    const size_t N = (size_t)1 << T.logN;
    dim3 g((unsigned)(N / BC_THREADS), (unsigned)((span + BC_TT - 1) / BC_TT), (unsigned)b.zpre[b.n]);
    KS_LAUNCH(st, "bconv_up", k_bconv_up<<<g, BC_THREADS, 0, st>>>(T, b));
    return launch_status("ModUp BConv launch");
}

void add_bdn(BDnJobs &b, const BDnJob &j)
{
    if (b.n == 0) b.zpre[0] = 0;
    b.job[b.n] = j;
    b.zpre[b.n + 1] = b.zpre[b.n] + j.npoly;
    b.n += 1;
}

// ModDown P2: grid (N/256, ceil(max nact/TT), polynomials of all jobs).
__global__ void __launch_bounds__(BC_THREADS, 4) k_bconv_down(Tables T, BDnJobs bj)
{
    __shared__ u64 cs[kMaxP][BC_TT];
    const int jb = find_slot(bj.zpre, bj.n, blockIdx.z);
    const BDnJob &J = bj.job[jb];
    const int x = blockIdx.z - bj.zpre[jb];
    const int nact = J.nact;
    const int ib = J.i_begin, ie = J.i_end < 0 ? nact : J.i_end;
    const int i0 = ib + blockIdx.y * BC_TT;  // first target tower of the block
    if (i0 >= ie) return;
    const int K = T.kp;
    for (int idx = threadIdx.x; idx < K * BC_TT; idx += blockDim.x) {
        const int k = idx / BC_TT, g = idx % BC_TT;
        cs[k][g] = (i0 + g < ie) ? T.dn_mat[(size_t)k * T.nq + i0 + g] : 0;
    }
    __syncthreads();
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 *w = J.w ? J.w + (size_t)x * J.w_stride : J.cp + (size_t)x * J.cp_stride + (size_t)nact * N;
    BAcc acc[BC_TT];
#pragma unroll
    for (int g = 0; g < BC_TT; ++g) bacc_zero(acc[g]);
    int k = 0;
    for (; k + 4 <= K; k += 4) {
        u64 wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) wv[u] = w[(size_t)(k + u) * N + n];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            u32 y0, y1;
            split_y(wv[u], y0, y1);
#pragma unroll
            for (int g = 0; g < BC_TT; ++g) bacc_mac(acc[g], y0, y1, cs[k + u][g]);
        }
    }
    for (; k < K; ++k) {
        u32 y0, y1;
        split_y(w[(size_t)k * N + n], y0, y1);
#pragma unroll
        for (int g = 0; g < BC_TT; ++g) bacc_mac(acc[g], y0, y1, cs[k][g]);
    }
    u64 *vo = J.v + (size_t)x * J.v_stride;
#pragma unroll
    for (int g = 0; g < BC_TT; ++g)
        if (i0 + g < ie) vo[(size_t)(i0 + g - ib) * N + n] = bacc_reduce(acc[g], T.modc[i0 + g]);
}

int launch_bconv_down(const Tables &T, const BDnJobs &b, cudaStream_t st)
{
    if (b.n == 0) return KS_OK;
    bool ranged = false;
    for (int i = 0; i < b.n; ++i)
        ranged = ranged || b.job[i].i_begin != 0 || (b.job[i].i_end >= 0 && b.job[i].i_end != b.job[i].nact) ||
                 b.job[i].w != nullptr;
    if (!ranged && T.dn_tc && bconv_tc_supported(T, T.kp)) return launch_bconv_down_tc(T, b, T.dn_tc, st);
    int span = 0;
    for (int i = 0; i < b.n; ++i)
        span = std::max(span, (b.job[i].i_end < 0 ? b.job[i].nact : b.job[i].i_end) - b.job[i].i_begin);
    if (span <= 0) return KS_OK;
    const size_t N = (size_t)1 << T.logN;
    dim3 g((unsigned)(N / BC_THREADS), (unsigned)((span + BC_TT - 1) / BC_TT), (unsigned)b.zpre[b.n]);
    KS_LAUNCH(st, "bconv_down", k_bconv_down<<<g, BC_THREADS, 0, st>>>(T, b));
    return launch_status("ModDown BConv launch");
}

// ------------------------------------------------------------------ apply key
// ModUp P4+P5 (single job): grid (N/256, nact+K).  The stored key carries the
// folded factors and 2^64, so REDC of the 128-bit sum gives the folded c'.
// With galois = g != 1 the raised digits are read through the automorphism
// X -> X^g of the evaluation domain (slot n takes slot n' with
// 2brv(n')+1 = (2brv(n)+1)g mod 2N): the key product of a hoisted rotation.
__device__ __forceinline__ size_t galois_slot(size_t n, u64 g, int logN)
{
    const u64 two_n = 2ull << logN;
    const u64 e = ((2ull * (__brev((unsigned)n) >> (32 - logN)) + 1) * g) & (two_n - 1);
    return (size_t)(__brev((unsigned)((e - 1) >> 1)) >> (32 - logN));
}

// Evaluation-domain automorphism X -> X^g of n towers starting at full
// tower t0: out[t][n] = in[t][galois_slot(n)] (+ out[t][n] mod q_t with
// accumulate).  Inputs canonical; grid (N/256, towers).
__global__ void __launch_bounds__(256) k_automorph(Tables T, int t0, const u64 *in, u64 *out, u64 galois,
                                                   int accumulate)
{
    const int t = blockIdx.y;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = T.modc[t0 + t].q;
    const u64 v = in[(size_t)t * N + galois_slot(n, galois, T.logN)];
    u64 *o = out + (size_t)t * N + n;
    *o = accumulate ? reduce2(*o + v, q) : v;
}

template <bool CK>
__global__ void __launch_bounds__(256) k_apply_key(Tables T, int nact, int j0, int j1, const u64 *d, const u64 *D,
                                                   size_t dstride, KeyView key, u64 *cp, int accumulate, u64 galois)
{
    const int t = blockIdx.y;
    const int nt = nact + T.kp;
    const int nfull = T.nq + T.kp;
    const int tf = full_tower(t, nact, T.nq);
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t ns = galois == 1 ? n : galois_slot(n, galois, T.logN);
    const ModC &mc = T.modc[tf];
    U128 sb = {0, 0}, sa = {0, 0};
    for (int j = j0; j < j1; ++j) {
        const bool own = t < nact && t / T.alpha == j;
        const u64 dv = own ? d[(size_t)t * N + ns] : D[(size_t)(j - j0) * dstride + (size_t)t * N + ns];
        mac128(sb, dv, key_b<CK>(key, j, tf, n, nfull, T.logN));
        mac128(sa, dv, key_a<CK>(key, j, tf, n, nfull, T.logN, mc.q));
    }
    // D below kFwdLazy*q: the REDC result is below q + kFwdLazy*nd*q^2/2^64, reduced fully.
    u64 rb = reduce_any(redc(sb, mc.q, mc.mont), mc.q, mc.one_sh);
    u64 ra = key_a_finish<CK>(key, sa, mc, T.key_sc, tf);
    u64 *cb = cp + (size_t)t * N + n;
    u64 *ca = cp + ((size_t)nt + t) * N + n;
    if (accumulate) {
        rb = reduce2(rb + *cb, mc.q);
        ra = reduce2(ra + *ca, mc.q);
    }
    *cb = rb;
    *ca = ra;
}

int launch_automorph(const Tables &T, int t0, int ntowers, const u64 *in, u64 *out, uint64_t galois, bool accumulate,
                     cudaStream_t st)
{
    if (ntowers == 0) return KS_OK;
    const size_t N = (size_t)1 << T.logN;
    KS_LAUNCH(st, "automorph",
              k_automorph<<<dim3((unsigned)(N / 256), (unsigned)ntowers), 256, 0, st>>>(T, t0, in, out, galois,
                                                                                       accumulate ? 1 : 0));
    return launch_status("automorphism launch");
}

int launch_apply_key(const Tables &T, int nact, int j_begin, int j_end, const u64 *d, const u64 *D,
                     size_t D_digit_stride, const KeyView &key, u64 *cp, bool accumulate, cudaStream_t st,
                     uint64_t galois)
{
    const size_t N = (size_t)1 << T.logN;
    dim3 g((unsigned)(N / 256), (unsigned)(nact + T.kp));
    if (key.comp)
        KS_LAUNCH(st, "apply_key",
                  k_apply_key<true><<<g, 256, 0, st>>>(T, nact, j_begin, j_end, d, D, D_digit_stride, key, cp,
                                                       accumulate ? 1 : 0, galois));
    else
        KS_LAUNCH(st, "apply_key",
                  k_apply_key<false><<<g, 256, 0, st>>>(T, nact, j_begin, j_end, d, D, D_digit_stride, key, cp,
                                                        accumulate ? 1 : 0, galois));
    return launch_status("apply-key launch");
}

struct OutPtrs {
    u64 *p[2];
};

// ModDown P4: out = cp - v mod q (cp canonical, v lazy below kFwdLazy*q).
__global__ void __launch_bounds__(256) k_down_final(Tables T, const u64 *cp, size_t cp_stride, const u64 *v,
                                                    size_t v_stride, OutPtrs outs)
{
    const int i = blockIdx.y, x = blockIdx.z;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ModC &mc = T.modc[i];
    const u64 r = cp[x * cp_stride + (size_t)i * N + n] + kFwdLazy * mc.q - v[x * v_stride + (size_t)i * N + n];
    outs.p[x][(size_t)i * N + n] = reduce_any(r, mc.q, mc.one_sh);
}

int launch_down_final(const Tables &T, int nact, int npoly, const u64 *cp, size_t cp_stride, const u64 *v,
                      size_t v_stride, u64 *const *outs, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    OutPtrs o;
    o.p[0] = outs[0];
    o.p[1] = npoly > 1 ? outs[1] : outs[0];
    dim3 g((unsigned)(N / 256), (unsigned)nact, (unsigned)npoly);
    KS_LAUNCH(st, "down_final", k_down_final<<<g, 256, 0, st>>>(T, cp, cp_stride, v, v_stride, o));
    return launch_status("ModDown final launch");
}

// ------------------------------------------------------------------ helpers
// grid (N/256, limbs)
__global__ void k_scale(Tables T, LimbMaps ms, const ulonglong2 *fac)
{
    const int lg = blockIdx.y + blockIdx.z * gridDim.y;
    if (lg >= ms.pre[ms.n]) return;
    const LimbRef L = limb_ref(ms, lg, T.nq, T.alpha, T.logN);
    if (L.skip) return;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = T.modc[L.tf].q;
    const ulonglong2 f = fac[L.tf];
    L.dst[n] = reduce2(shoup_lazy(L.src[n], f.x, f.y, q), q);
}

int launch_scale(const Tables &T, const LimbMaps &m, const ulonglong2 *factors_full, cudaStream_t st)
{
    if (m.n == 0 || m.pre[m.n] == 0) return KS_OK;
    const size_t N = (size_t)1 << T.logN;
    KS_LAUNCH(st, "scale", k_scale<<<limb_grid((unsigned)(N / 256), m.pre[m.n]), 256, 0, st>>>(T, m, factors_full));
    return launch_status("scale launch");
}

// grid (N/256, nact, nd): D[j][t] = d[t] for t in digit j.
__global__ void k_bypass_copy(Tables T, int nact, const u64 *d, u64 *D)
{
    const int t = blockIdx.y, j = blockIdx.z;
    if (t / T.alpha != j) return;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = nact + T.kp;
    D[((size_t)j * nt + t) * N + n] = d[(size_t)t * N + n];
}

int launch_bypass_copy(const Tables &T, int nact, const u64 *d, u64 *D, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const int nd = (nact + T.alpha - 1) / T.alpha;
    KS_LAUNCH(st, "bypass_copy", k_bypass_copy<<<dim3((unsigned)(N / 256), nact, nd), 256, 0, st>>>(T, nact, d, D));
    return launch_status("bypass copy launch");
}

// ------------------------------------------------------------------ keys
// evk [ndig][2][nfull][N] canonical -> * key_sc[t] (Montgomery factor folded).
__global__ void k_key_convert(Tables T, u64 *evk)
{
    const int nfull = T.nq + T.kp;
    const int limb = blockIdx.y;
    const int tf = limb % nfull;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = T.modc[tf].q;
    const ulonglong2 f = T.key_sc[tf];
    u64 *p = evk + (size_t)limb * N + n;
    *p = reduce2(shoup_lazy(*p, f.x, f.y, q), q);
}

int launch_key_convert(const Tables &T, u64 *evk, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const int limbs = T.ndig * 2 * (T.nq + T.kp);
    KS_LAUNCH(st, "key_convert", k_key_convert<<<dim3((unsigned)(N / 256), limbs), 256, 0, st>>>(T, evk));
    return launch_status("key conversion launch");
}

// Pseudo-random canonical residues (SplitMix64 finaliser of seed + index).
__global__ void k_key_random(Tables T, u64 *evk, uint64_t seed)
{
    const int nfull = T.nq + T.kp;
    const int limb = blockIdx.y;
    const int tf = limb % nfull;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    u64 z = seed + ((size_t)limb * N + n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    evk[(size_t)limb * N + n] = z % T.modc[tf].q;
}

int launch_key_random(const Tables &T, u64 *evk, uint64_t seed, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const int limbs = T.ndig * 2 * (T.nq + T.kp);
    KS_LAUNCH(st, "key_random", k_key_random<<<dim3((unsigned)(N / 256), limbs), 256, 0, st>>>(T, evk, seed));
    return launch_status("synthetic key launch");
}

// a*b mod q for a, b < q (two Montgomery reductions).
__device__ __forceinline__ u64 mulmod_dev(u64 a, u64 b, const ModC &m)
{
    U128 t = {0, 0};
    mac128(t, a, b);
    u64 r = reduce2(redc(t, m.q, m.mont), m.q);  // a*b*2^-64
    U128 t2 = {0, 0};
    mac128(t2, r, m.r2);
    return reduce2(redc(t2, m.q, m.mont), m.q);  // * 2^128 * 2^-64
}

// grid (N/256, nfull, ndig)
__global__ void k_keygen_combine(Tables T, const u64 *s_hat, const u64 *sp_hat, const u64 *e_hat, const u64 *pmod,
                                 u64 *evk)
{
    const int tf = blockIdx.y, j = blockIdx.z;
    const int nfull = T.nq + T.kp;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ModC &mc = T.modc[tf];
    const u64 q = mc.q;
    const u64 a = evk[(((size_t)j * 2 + 1) * nfull + tf) * N + n];
    const u64 sh = s_hat[(size_t)tf * N + n];
    const u64 sph = sp_hat[(size_t)tf * N + n];
    const u64 eh = e_hat[((size_t)j * nfull + tf) * N + n];
    u64 b = eh + q - mulmod_dev(a, sh, mc);
    b = reduce2(b, q);
    const bool in_digit = tf < T.nq && tf / T.alpha == j;
    if (in_digit) b = reduce2(b + mulmod_dev(pmod[tf], sph, mc), q);
    evk[(((size_t)j * 2 + 0) * nfull + tf) * N + n] = b;
}

int launch_keygen_combine(const Tables &T, const u64 *s_hat, const u64 *sp_hat, const u64 *e_hat, const u64 *pmod,
                          u64 *evk, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    KS_LAUNCH(st, "keygen_combine", k_keygen_combine<<<dim3((unsigned)(N / 256), T.nq + T.kp, T.ndig), 256, 0, st>>>(
                                        T, s_hat, sp_hat, e_hat, pmod, evk));
    return launch_status("keygen combine launch");
}

// grid (N/256, nfull, nvec): out[v][t][n] = in[v][n] mod r_t (signed input).
__global__ void k_signed_to_towers(Tables T, const int64_t *in, u64 *out)
{
    const int tf = blockIdx.y, vi = blockIdx.z;
    const int nfull = T.nq + T.kp;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q = T.modc[tf].q;
    const int64_t v = in[(size_t)vi * N + n];
    const u64 mag = v < 0 ? (u64)(-(v + 1)) + 1 : (u64)v;
    u64 r = mag % q;
    if (v < 0 && r != 0) r = q - r;
    out[((size_t)vi * nfull + tf) * N + n] = r;
}

int launch_signed_to_towers(const Tables &T, const int64_t *v, int nvec, u64 *out, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    KS_LAUNCH(st, "signed_to_towers",
              k_signed_to_towers<<<dim3((unsigned)(N / 256), T.nq + T.kp, nvec), 256, 0, st>>>(T, v, out));
    return launch_status("signed residue launch");
}

}  // namespace ks
