// ks_cluster.cuh -- thread-block-cluster helpers shared by the one-launch
// cluster NTT (ks_ntt_cluster.cu) and the per-output-tower Output-Centric
// kernel (ks_oc_tower.cu): the cluster geometry of a two-pass NTT shape,
// the cluster barrier, and loads from another CTA's shared memory
// (distributed shared memory, mapa + ld.shared::cluster).
#pragma once
#include <algorithm>
#include <atomic>

#include "ks_ntt_core.cuh"

namespace ks {

// Cluster geometry of a two-pass shape: CTAs of MUL column groups of the
// column pass (COLS columns), C CTAs per limb, each then running the row
// pass on ROWS = 2^LA / C rows.  Supported when both passes fit the same
// block size and C is at most 16 (the non-portable cluster limit).
template <class S, int MUL>
struct NttClusterShape {
    static constexpr int COLS = S::COLS * MUL;
    static constexpr int C = (1 << S::LB) / COLS;
    static constexpr int ROWS = C > 0 ? (1 << S::LA) / C : 1;
    static constexpr int THREADS = COLS * S::TA;
    static constexpr bool OK = C >= 1 && C * COLS == (1 << S::LB) && C * ROWS == (1 << S::LA) &&
                               ROWS * S::TB == THREADS && C <= 16;
    static constexpr int BLOCKW = S::N / (C > 0 ? C : 1);  // words of a CTA's block of the limb
    static constexpr int BUFW = BLOCKW > ROWS * S::ROWPAD ? BLOCKW : ROWS * S::ROWPAD;
    static constexpr int SMEM = BUFW * 8 + (1 << S::LA) * 16 + ROWS * S::REGB * 16;
    static constexpr int MINB = S::LA <= 8 ? (4 / MUL > 0 ? 4 / MUL : 1) : 1;
};

template <class S, int MUL>
using Cl = NttClusterShape<S, MUL>;

__device__ __forceinline__ int cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// Full cluster barrier: shared-memory writes before it are visible to every
// CTA of the cluster after it.
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}

// Address in CTA `rank`'s shared memory of the word at local address p.
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, int rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ u64 ld_dsmem(uint32_t addr)
{
    u64 v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// Kernel attributes (dynamic shared memory, cluster sizes above 8) and
// whether the device can run a cluster of the kernel at all.
template <class KERN>
inline bool cluster_prepare(KERN kern, int C, int threads, int smem)
{
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();  // a refused query leaves no sticky error
    return ok;
}

}  // namespace ks
