// ks_ntt_core.cuh -- limb addressing and the row/column NTT pass bodies shared
// by the stage kernels (ks_kernels.cu) and the Output-Centric fused kernels
// (ks_oc.cu).  See ks_device.cuh for the decomposition.
#pragma once
#include "ks_device.cuh"
#include "ks_launch.h"

namespace ks {

struct LimbRef {
    const u64 *src;
    u64 *dst;
    const ulonglong2 *scale;
    int t, tf, b;
    bool skip;
};

__device__ __forceinline__ LimbRef limb_ref(const LimbMaps &ms, int lg, int nq, int alpha, int logN)
{
    const int jb = find_slot(ms.pre, ms.n, lg);
    const LimbMap &m = ms.m[jb];
    const int l = lg - ms.pre[jb];
    const int a = l / m.per, b = l % m.per;
    const int t = m.toff + b;
    const size_t o = ((size_t)a * m.row_stride + m.aoff + b) << logN;
    LimbRef r;
    r.src = m.src ? m.src + o : nullptr;
    r.dst = m.dst ? m.dst + o : nullptr;
    r.scale = m.scale;
    r.t = t;
    r.b = b;
    r.tf = full_tower(t, m.nact, nq);
    r.skip = m.skip_base >= 0 && t < m.nact && (t / alpha) == a + m.skip_base;
    return r;
}

// Padded index inside a shared-memory row: one spare word after every group
// of MB words keeps the second-round reads of a row free of bank conflicts.
template <class S>
__device__ __forceinline__ int rpad(int c)
{
    return c + c / S::MB;
}

// First-round twiddles of one row (local stages s < RB, group g < 2^s),
// copied by the row's own TB threads into sh[2^s - 1 + g]: one load each,
// issued together with the row's data loads, so the first round's
// butterflies read shared memory instead of waiting on dependent L2 loads
// (the first round's twiddles are common to the whole row; the second
// round's differ per thread and stay in the table).
template <class S>
__device__ __forceinline__ void stage_row_round1(ulonglong2 *sh, const ulonglong2 *t, int G, int tau)
{
    for (int f = tau; f < S::REGB - 1; f += S::TB) {
        const int st = 31 - __clz(f + 1);
        sh[f] = __ldg(t + (G << st) + f + 1 - (1 << st));
    }
}

// Twiddle fetcher of the forward row pass: first round from the staged row
// block, second round from the tower table.
template <class S>
struct TwStaged {
    const ulonglong2 *sh;
    const ulonglong2 *t;
    int G;
    __device__ __forceinline__ ulonglong2 operator()(int s, int i) const
    {
        if (s < S::RB) return sh[(1 << s) - 1 + i];
        return __ldg(t + (G << s) + i);
    }
};

// Row pass of the forward NTT on one row held by TB threads: x enters and
// leaves in the first-round layout (x[k] is element k*TB + tau of the row),
// srow is the row's padded shared-memory buffer.  Contains block barriers:
// every thread of the block must call it.
template <class S, bool SP = false, class TW>
__device__ __forceinline__ void row_fwd_core(u64 (&x)[S::REGB], const TW &tw, u64 *srow, int tau, u64 q, u64 q2)
{
    constexpr int M = S::MB, NG = S::REGB / S::MB;
    fwd_round1<S::RB, SP>(x, tw, q, q2);
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) srow[rpad<S>(k * S::TB + tau)] = x[k];
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) x[gg * M + k2] = srow[rpad<S>((tau * NG + gg) * M + k2)];
    fwd_round2<S::LB, S::RB, SP>(x, tau * NG, tw, q, q2);
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) srow[rpad<S>((tau * NG + gg) * M + k2)] = x[gg * M + k2];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) x[k] = srow[rpad<S>(k * S::TB + tau)];
    __syncthreads();
}

// Row pass of the inverse NTT (stages logN-1 .. LA), same layout contract.
template <class S, bool SP = false, class TW>
__device__ __forceinline__ void row_inv_core(u64 (&x)[S::REGB], const TW &tw, u64 *srow, int tau, u64 q, u64 q2)
{
    constexpr int M = S::MB, NG = S::REGB / S::MB;
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) srow[rpad<S>(k * S::TB + tau)] = x[k];
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) x[gg * M + k2] = srow[rpad<S>((tau * NG + gg) * M + k2)];
    inv_round2<S::LB, S::RB, SP>(x, tau * NG, tw, q, q2);
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < NG; ++gg)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) srow[rpad<S>((tau * NG + gg) * M + k2)] = x[gg * M + k2];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::REGB; ++k) x[k] = srow[rpad<S>(k * S::TB + tau)];
    __syncthreads();
    inv_round1<S::RB, SP>(x, tw, q, q2);
}

}  // namespace ks
