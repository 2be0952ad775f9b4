// ks_oc.cu -- Output-Centric dataflow (CiFlow Sec. IV-C).
//
// OC computes the key-switch output tower by tower instead of stage by stage.
// The GPU schedule (P towers first, reading (v): ModDown of every Q output
// tower needs all K special towers of c'):
//   1. prep       iNTT of every input tower with the (Q_j/q_i)^-1 prescale
//                 (ModUp P1) -> y, coefficient form;
//   2. P section  for each special tower p_k only: BConv of every digit to
//                 p_k (P2), column pass of the NTT (P3), then one fused
//                 kernel per row block: row pass of each digit's limb, the
//                 key product accumulated over digits on chip (P4+P5), and
//                 the row pass of ModDown's iNTT (ModDown P1) -- c' of the
//                 special towers never leaves the kernel in evaluation form;
//                 the inverse column pass then yields w;
//   3. Q section  for each output tower t: BConv of the other digits to t
//                 and of w to t (ModUp P2, ModDown P2), column passes, then
//                 one fused kernel per row block: row pass, key product with
//                 the bypassed digit taken straight from the input (P3-P5),
//                 row pass of the ModDown limbs (ModDown P3) and the final
//                 subtraction (ModDown P4) written to the output.
// The key is read once, in the fused kernels, straight from device memory.
#include "ks_ntt_core.cuh"

namespace ks {

// Accumulate x * e (e the stored key word) into a canonical accumulator.
__device__ __forceinline__ u64 mac_redc(u64 acc, u64 x, u64 e, u64 q, u64 mont)
{
    U128 t = {0, 0};
    mac128(t, x, e);
    return reduce2(acc + reduce2(redc(t, q, mont), q), q);
}

// P section, fused row kernel.  grid (2^LA/ROWS, K).
template <class S>
__global__ void __launch_bounds__(S::THREADS_B) k_oc_rowP(Tables T, int nact, int nd, const u64 *tmp1, const u64 *evk,
                                                          u64 *cp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int K = T.kp;
    const int k = blockIdx.y;
    const int t = nact + k;
    const int tf = T.nq + k;
    const int nt = nact + K;
    const int nfull = T.nq + K;
    const ModC mc = T.modc[tf];
    const u64 q = mc.q, q2 = 2 * q;
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    u64 *srow = sm + rr * S::ROWPAD;
    const TwRow tw{T.tw + ((size_t)tf << S::LOGN), (1 << S::LA) + h};
    const size_t rowoff = (size_t)h << S::LB;
    u64 accb[S::REGB], acca[S::REGB];
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) accb[i] = acca[i] = 0;
    for (int j = 0; j < nd; ++j) {
        const u64 *gin = tmp1 + ((size_t)(j * K + k) << S::LOGN) + rowoff;
        u64 x[S::REGB];
#pragma unroll
        for (int i = 0; i < S::REGB; ++i) x[i] = gin[i * S::TB + tau];
        row_fwd_core<S>(x, tw, srow, tau, q, q2);
        const u64 *eb = evk + ((size_t)((j * 2 + 0) * nfull + tf) << S::LOGN) + rowoff;
        const u64 *ea = evk + ((size_t)((j * 2 + 1) * nfull + tf) << S::LOGN) + rowoff;
#pragma unroll
        for (int i = 0; i < S::REGB; ++i) {
            const int c = i * S::TB + tau;
            accb[i] = mac_redc(accb[i], x[i], __ldg(eb + c), q, mc.mont);
            acca[i] = mac_redc(acca[i], x[i], __ldg(ea + c), q, mc.mont);
        }
    }
    const TwRow itw{T.itw + ((size_t)tf << S::LOGN), (1 << S::LA) + h};
    row_inv_core<S>(accb, itw, srow, tau, q, q2);
    u64 *ob = cp + ((size_t)t << S::LOGN) + rowoff;
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) ob[i * S::TB + tau] = accb[i];
    row_inv_core<S>(acca, itw, srow, tau, q, q2);
    u64 *oa = cp + ((size_t)(nt + t) << S::LOGN) + rowoff;
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) oa[i * S::TB + tau] = acca[i];
}

// Q section, fused row kernel.  grid (2^LA/ROWS, nact).  tmp2 holds
// [nd + 2][nact] limbs: rows j < nd the ModUp limbs of digit j (slot of the
// own digit unused), rows nd, nd+1 the ModDown limbs of the two polynomials.
template <class S>
__global__ void __launch_bounds__(S::THREADS_B) k_oc_rowQ(Tables T, int nact, int nd, const u64 *tmp2, const u64 *d,
                                                          const u64 *evk, u64 *out0, u64 *out1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sm = reinterpret_cast<u64 *>(smem_raw);
    const int t = blockIdx.y;
    const int j0 = t / T.alpha;
    const int nfull = T.nq + T.kp;
    const ModC mc = T.modc[t];
    const u64 q = mc.q, q2 = 2 * q;
    const int rr = threadIdx.x / S::TB, tau = threadIdx.x % S::TB;
    const int h = blockIdx.x * S::ROWS + rr;
    u64 *srow = sm + rr * S::ROWPAD;
    const TwRow tw{T.tw + ((size_t)t << S::LOGN), (1 << S::LA) + h};
    const size_t rowoff = (size_t)h << S::LB;
    u64 accb[S::REGB], acca[S::REGB];
#pragma unroll
    for (int i = 0; i < S::REGB; ++i) accb[i] = acca[i] = 0;
    for (int j = 0; j < nd; ++j) {
        u64 x[S::REGB];
        if (j == j0) {
            const u64 *gin = d + ((size_t)t << S::LOGN) + rowoff;
#pragma unroll
            for (int i = 0; i < S::REGB; ++i) x[i] = gin[i * S::TB + tau];
        } else {
            const u64 *gin = tmp2 + ((size_t)(j * nact + t) << S::LOGN) + rowoff;
#pragma unroll
            for (int i = 0; i < S::REGB; ++i) x[i] = gin[i * S::TB + tau];
            row_fwd_core<S>(x, tw, srow, tau, q, q2);
        }
        const u64 *eb = evk + ((size_t)((j * 2 + 0) * nfull + t) << S::LOGN) + rowoff;
        const u64 *ea = evk + ((size_t)((j * 2 + 1) * nfull + t) << S::LOGN) + rowoff;
#pragma unroll
        for (int i = 0; i < S::REGB; ++i) {
            const int c = i * S::TB + tau;
            accb[i] = mac_redc(accb[i], x[i], __ldg(eb + c), q, mc.mont);
            acca[i] = mac_redc(acca[i], x[i], __ldg(ea + c), q, mc.mont);
        }
    }
    const u64 q4 = 2 * q2;
#pragma unroll
    for (int xp = 0; xp < 2; ++xp) {
        u64 v[S::REGB];
        const u64 *gin = tmp2 + ((size_t)((nd + xp) * nact + t) << S::LOGN) + rowoff;
#pragma unroll
        for (int i = 0; i < S::REGB; ++i) v[i] = gin[i * S::TB + tau];
        row_fwd_core<S>(v, tw, srow, tau, q, q2);
        u64 *o = (xp == 0 ? out0 : out1) + ((size_t)t << S::LOGN) + rowoff;
#pragma unroll
        for (int i = 0; i < S::REGB; ++i) {
            u64 r = (xp == 0 ? accb[i] : acca[i]) + q4 - v[i];
            r = r >= q4 ? r - q4 : r;
            o[i * S::TB + tau] = reduce4(r, q, q2);
        }
    }
}

template <class S>
static void oc_rows_S(const Tables &T, int nact, int nd, const u64 *tmp1, const u64 *tmp2, const u64 *d,
                      const u64 *evk, u64 *cp, u64 *out0, u64 *out1, bool p_section, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_oc_rowP<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_B);
        cudaFuncSetAttribute(k_oc_rowQ<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_B);
        attr = true;
    }
    if (p_section)
        KS_LAUNCH(st, "oc_row_p",
                  k_oc_rowP<S><<<dim3((1 << S::LA) / S::ROWS, T.kp), S::THREADS_B, S::SMEM_B, st>>>(T, nact, nd, tmp1,
                                                                                                  evk, cp));
    else
        KS_LAUNCH(st, "oc_row_q",
                  k_oc_rowQ<S><<<dim3((1 << S::LA) / S::ROWS, nact), S::THREADS_B, S::SMEM_B, st>>>(
                      T, nact, nd, tmp2, d, evk, out0, out1));
}

static int oc_rows(const Tables &T, int nact, int nd, const u64 *tmp1, const u64 *tmp2, const u64 *d,
                   const u64 *evk, u64 *cp, u64 *out0, u64 *out1, bool p_section, cudaStream_t st)
{
    switch (T.logN) {
    case 10: oc_rows_S<ShapeOf<10>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 11: oc_rows_S<ShapeOf<11>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 12: oc_rows_S<ShapeOf<12>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 13: oc_rows_S<ShapeOf<13>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 14: oc_rows_S<ShapeOf<14>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 15: oc_rows_S<ShapeOf<15>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 16: oc_rows_S<ShapeOf<16>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    case 17: oc_rows_S<ShapeOf<17>::T>(T, nact, nd, tmp1, tmp2, d, evk, cp, out0, out1, p_section, st); break;
    default: return fail(KS_EUNSUPPORTED, "logN outside 10..17");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string("OC row kernel launch: ") + cudaGetErrorString(e));
    return KS_OK;
}

int launch_oc(const Tables &T, int nact, const u64 *d, const u64 *evk, u64 *out0, u64 *out1, u64 *y, u64 *tmp,
              u64 *cp, const ulonglong2 *prescale, cudaStream_t st)
{
    const size_t N = (size_t)1 << T.logN;
    const int K = T.kp;
    const int nt = nact + K;
    const int nd = (nact + T.alpha - 1) / T.alpha;
    int rc;
    // 1. prep (ModUp P1)
    LimbMap m1{d, y, nact, 0, 0, 0, nact, -1};
    if ((rc = launch_ntt_inv(T, m1, nact, prescale, false, st)) != KS_OK) return rc;
    // 2. P section: BConv to the special towers, column pass, fused rows, inverse column pass
    u64 *tmp1 = tmp;
    if ((rc = launch_bconv_up_range(T, nact, nact, nt, nact, y, tmp1, (size_t)K * N, st)) != KS_OK) return rc;
    LimbMap mp{tmp1, tmp1, K, K, 0, nact, nact, -1};
    if ((rc = launch_fwd_col(T, mp, nd * K, st)) != KS_OK) return rc;
    if ((rc = oc_rows(T, nact, nd, tmp1, nullptr, nullptr, evk, cp, nullptr, nullptr, true, st)) != KS_OK) return rc;
    LimbMap mw{cp, cp, K, nt, nact, nact, nact, -1};
    if ((rc = launch_inv_col(T, mw, 2 * K, nullptr, false, st)) != KS_OK) return rc;
    // 3. Q section: BConv of the other digits and of w to each output tower,
    //    column passes, fused rows with ModDown
    u64 *tmp2 = tmp;
    if ((rc = launch_bconv_up_range(T, nact, 0, nact, 0, y, tmp2, (size_t)nact * N, st)) != KS_OK) return rc;
    if ((rc = launch_bconv_down(T, nact, 2, cp, (size_t)nt * N, tmp2 + (size_t)nd * nact * N, (size_t)nact * N, st)) !=
        KS_OK)
        return rc;
    LimbMap mq{tmp2, tmp2, nact, nact, 0, 0, nact, 0};
    if ((rc = launch_fwd_col(T, mq, (nd + 2) * nact, st)) != KS_OK) return rc;
    return oc_rows(T, nact, nd, nullptr, tmp2, d, evk, nullptr, out0, out1, false, st);
}

}  // namespace ks
