// ks_launch.h -- host-side launchers of the key-switching kernels.
//
// Every stage launcher takes a small table of per-job descriptors passed to
// the kernel by value (kernel parameters, up to kMaxBatch jobs), so one launch
// covers the limbs of every job of a batch; a single key switch is a batch of
// one.  Blocks find their job by a search over per-launch prefix counts.
#pragma once
#include <vector>

#include "ks_internal.h"

namespace ks {

constexpr int kMaxBatch = 64;

// A set of limbs addressed arithmetically.  Limb l of the set is entry
// b = l % per of limb-row a = l / per; it lives at (a*row_stride + aoff + b)*N
// words from src/dst and belongs to compact tower t = toff + b of the level
// basis D_l (Q towers 0..nact-1, then the K special towers).  With
// skip_base >= 0, limbs whose tower lies inside digit a + skip_base are
// skipped (the ModUp bypass); -1 skips nothing.  scale (optional) holds one
// Shoup pair per entry b for the inverse column pass.
struct LimbMap {
    const u64 *src;
    u64 *dst;
    const ulonglong2 *scale;
    int per;
    int row_stride;
    int aoff;
    int toff;
    int nact;
    int skip_base;
};

// One LimbMap per job; job j owns launch limbs [pre[j], pre[j+1]).
struct LimbMaps {
    int n;
    int pre[kMaxBatch + 1];
    LimbMap m[kMaxBatch];
};

__host__ __device__ inline int full_tower(int t, int nact, int nq) { return t < nact ? t : nq + (t - nact); }

// Job of launch item x given prefix counts pre[0..n] (binary search).
__host__ __device__ inline int find_slot(const int *pre, int n, int x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Host helpers to build launch tables.
LimbMaps one_map(const LimbMap &m, int nlimbs);
void add_map(LimbMaps &ms, const LimbMap &m, int nlimbs);

// Forward NTT (column pass src->dst, row pass in place on dst).  Input below
// 4q.  canonical: output in [0, q); otherwise lazy, below kFwdLazy*q = 72q (every
// consumer of lazy output reduces it).
int launch_ntt_fwd(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st);
// Inverse NTT without the N^-1 factor (row pass src->dst, column pass in
// place); the column pass multiplies by the per-entry scale when the job's
// map has one, or by N^-1 when scale_by_ninv; output canonical.  Input below 4q.
int launch_ntt_inv(const Tables &T, const LimbMaps &m, bool scale_by_ninv, cudaStream_t st);
// One-launch forms over thread-block clusters (ks_ntt_cluster.cu): the same
// contracts and bit-identical outputs; sc of the inverse: 0 none, 1 the
// job's per-entry scale, 2 N^-1.  They return KS_EUNSUPPORTED, launching
// nothing, when the ring degree's shape or the device has no cluster form;
// launch_ntt_fwd/inv use them when T.ntt_cluster is set and fall back.
bool ntt_cluster_shape(int logN);
int launch_ntt_fwd_cluster(const Tables &T, const LimbMaps &m, bool canonical, cudaStream_t st);
int launch_ntt_inv_cluster(const Tables &T, const LimbMaps &m, int sc, cudaStream_t st);
// Single passes.
int launch_fwd_col(const Tables &T, const LimbMaps &m, cudaStream_t st);
int launch_inv_col(const Tables &T, const LimbMaps &m, bool scale_by_ninv, cudaStream_t st);

// ModUp P2.  Job: digit j (all active digits, or only jsel >= 0) converts its
// canonical coefficient-form towers y[lo..hi) to the towers of D_l with
// compact index in [t_begin, t_end) outside the digit; output lazy in
// [0, 2r) at D + j'*dstride + (t - t_base)*N, j' = j (or 0 with jsel).
struct BUpJob {
    const u64 *y;
    u64 *D;
    size_t dstride;
    int nact, t_begin, t_end, t_base, jsel;
};
struct BUpJobs {
    int n;
    int zpre[kMaxBatch + 1];  // digit blocks of job j: [zpre[j], zpre[j+1])
    BUpJob job[kMaxBatch];
};
void add_bup(BUpJobs &b, const Tables &T, const BUpJob &j);
int launch_bconv_up(const Tables &T, const BUpJobs &b, cudaStream_t st);

// ModDown P2: w = cp rows [nact, nact+K) of each polynomial (canonical,
// coefficient form) -> v[x][i] = sum_k w_k * p_k^-1 mod q_i, lazy [0, 2q).
struct BDnJob {
    const u64 *cp;
    size_t cp_stride;
    u64 *v;
    size_t v_stride;
    int nact, npoly;
    // Optional (CUDA-core kernel only; jobs using them skip the tensor
    // cores): targets [i_begin, i_end) only, written at v + (i - i_begin)*N
    // (i_end < 0: all nact); w, when set, holds the sources of polynomial x
    // at w + x*w_stride instead of cp's rows nact..nact+K-1.
    int i_begin = 0, i_end = -1;
    const u64 *w = nullptr;
    size_t w_stride = 0;
};
struct BDnJobs {
    int n;
    int zpre[kMaxBatch + 1];
    BDnJob job[kMaxBatch];
};
void add_bdn(BDnJobs &b, const BDnJob &j);
int launch_bconv_down(const Tables &T, const BDnJobs &b, cudaStream_t st);

// Tensor-core base conversion (ks_bconv_tc.cu): same jobs and outputs as the
// CUDA-core kernels; used by launch_bconv_up/down when the tables are present
// and the shape is supported (at most 18 sources, N a multiple of 128).
bool bconv_tc_supported(const Tables &T, int nsrc);
int launch_bconv_up_tc(const Tables &T, const BUpJobs &b, const uint4 *slabs, const int *slab_lvl, cudaStream_t st);
int launch_bconv_down_tc(const Tables &T, const BDnJobs &b, const uint4 *slabs, cudaStream_t st);
// K blocks of 64 slice columns for nsrc sources: one up to 9, two up to 18.
inline int tc_kblocks(int nsrc) { return nsrc <= 9 ? 1 : 2; }
// Bits of the constants' slices: 9 (6 slices, partial sums below 9*7*255*511
// < 2^23) with one K block when every modulus is below 2^54, else 8 (7).
inline int tc_slice_bits(int kblocks, int below54) { return kblocks == 1 && below54 ? 9 : 8; }
// Host: one B slab of kblocks KB (8 slice rows x 64*kblocks slice columns,
// f16, canonical layout) for the constants c[0..nsrc) (carrying 2^64) of one
// target of modulus r: row b, column 7i + a holds bit slice b (of `bits`
// bits) of c_i * 2^(8a) * 2^-32 mod r.
constexpr int kTcSlabHalves = 8 * 64;  // f16 words of a slab per K block
void tc_slab(const std::vector<u64> &c, u64 r, int kblocks, int bits, uint16_t *slab);
// Device flag set by a tensor-core kernel whose MMA wait gave up (-1: unreadable).
int tc_error_flag(bool clear);
// Device flag set by a staged row pass whose bulk-copy wait gave up (-1: unreadable).
int ntt_error_flag(bool clear);

// ModUp P4+P5 (single job): cp[x][t] = sum_j D_{j,t} * evk_{j,x,t}, D_{j,t} = d_t
// inside digit j; D holds lazy NTT output.  accumulate: add to cp.  galois
// g != 1: every D_{j,t} (and d_t) is read through X -> X^g (hoisted rotation).
int launch_apply_key(const Tables &T, int nact, int j_begin, int j_end, const u64 *d, const u64 *D,
                     size_t D_digit_stride, const KeyView &key, u64 *cp, bool accumulate, cudaStream_t st,
                     uint64_t galois = 1);
// Automorphism X -> X^g of the evaluation slots of ntowers limbs (full
// towers t0..t0+ntowers-1): out = phi_g(in), or out + phi_g(in) mod q with
// accumulate.  in and out must not overlap.
int launch_automorph(const Tables &T, int t0, int ntowers, const u64 *in, u64 *out, uint64_t galois, bool accumulate,
                     cudaStream_t st);
// ModDown P4 (single job; P^-1 folded): out_x[i] = cp[x][i] - v[x][i] mod q_i,
// v lazy NTT output.
int launch_down_final(const Tables &T, int nact, int npoly, const u64 *cp, size_t cp_stride, const u64 *v,
                      size_t v_stride, u64 *const *outs, cudaStream_t st);
// Multiply limbs by per-tower factors (plain, Shoup; indexed by full tower).
int launch_scale(const Tables &T, const LimbMaps &m, const ulonglong2 *factors_full, cudaStream_t st);
// Copy the input towers of every digit into D (ModUp bypass, stage entry).
int launch_bypass_copy(const Tables &T, int nact, const u64 *d, u64 *D, cudaStream_t st);

// Key preparation: canonical evk [ndig][2][nq+kp][N] -> stored form
// (times key_sc[t], Montgomery factor included), in place.
int launch_key_convert(const Tables &T, u64 *evk, cudaStream_t st);
// Key generation combine: b_j = -a_j*s + e_j + g_j*s' per tower.
int launch_keygen_combine(const Tables &T, const u64 *s_hat, const u64 *sp_hat, const u64 *e_hat,
                          const u64 *pmod, u64 *evk, cudaStream_t st);
// Signed coefficients -> residues per tower: out[v][t][n] = in[v][n] mod r_t.
int launch_signed_to_towers(const Tables &T, const int64_t *v, int nvec, u64 *out, cudaStream_t st);

// Output-Centric key switch of a batch of jobs.
struct OcJob {
    const u64 *d;
    u64 *out0, *out1;
    KeyView key;  // the fused variant reads full keys only (launch_oc)
    u64 *y;    // [nact][N]
    u64 *tmp;  // [nd*(nact+K) + 2*nact][N]
    u64 *cp;   // [2][nact+K][N]
    const ulonglong2 *pre;  // ModUp P1 factors of the level
    int nact, nd;
};
// The jobs of one Output-Centric launch group, with prefix counts of their Q
// towers: job j owns Q-section items [pre[j], pre[j+1]).
struct OcJobs {
    int n;
    int pre[kMaxBatch + 1];
    OcJob job[kMaxBatch];
};
// Scratch words one job needs at level nact.
size_t oc_scratch_words(const Tables &T, int nact);
// The job of one key switch with its scratch (oc_scratch_words words) at
// `scratch`: y, then the section temporaries, then c' (ks_api.cu).
OcJob oc_job(const ks_params *P, const ks_key *K, int nact, const u64 *d, u64 *out0, u64 *out1, u64 *scratch);
// Host-side checks of one job's arguments (key of this parameter set, level
// in 1..n_q, non-NULL, 16-byte aligned, non-overlapping buffers); KS_OK or
// KS_EINVAL with the message set (ks_api.cu).
int check_job(const ks_params *P, const ks_key *K, uint32_t nact, const uint64_t *d, const uint64_t *o0,
              const uint64_t *o1);
// The parameter set's tables with a schedule's implementation choices
// (base-conversion engine, NTT form) applied (ks_api.cu).
Tables call_tables(const ks_params *P, const ks_schedule &sc);
// Output-Centric variants: FUSED runs each section's row pass, key product
// and ModDown step in one kernel per row block; SPLIT runs the row passes
// with the plain row-pass kernel and the key product / subtraction in a
// streaming combine kernel; WHOLE raises every digit to every tower in one
// base-conversion launch and one NTT launch, then runs the same per-tower
// combine kernels (special towers, ModDown, Q towers).
enum { KS_OC_FUSED = 0, KS_OC_SPLIT = 1, KS_OC_WHOLE = 2, KS_OC_TOWER = 3 };
// TOWER: the split variant's prep and special-tower section, then one
// thread-block-cluster kernel per (job, Q output tower) that keeps the
// tower's limbs on chip from ModUp base conversion to the ModDown
// subtraction (ks_oc_tower.cu).  KS_EUNSUPPORTED (nothing launched) where
// the ring degree has no cluster geometry, the device cannot run it, or a
// job's key is compressed.
bool oc_tower_supported(const Tables &T);
int launch_oc_tower(const Tables &T, const OcJobs &oj, cudaStream_t st);
// share_keys: jobs of a launch that share a key run through the key-grouped
// combine kernels (each key word read once per group of jobs); otherwise
// every job streams its own key limbs.
int launch_oc(const Tables &T, int njobs, const OcJob *jobs, int variant, cudaStream_t st, bool share_keys = false);

}  // namespace ks
