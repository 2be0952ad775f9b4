// ks_shard.cu -- one key switch split over G devices by tower.
//
// The output towers of a key switch are independent (CiFlow Sec. IV-C: the
// Output-Centric dataflow computes them one at a time), so one key switch
// can be spread over G devices by tower.  Rank g owns a contiguous range of
// Q towers and a contiguous range of special (P) towers, holds the input
// towers and the key limbs of those towers only (the key is sharded, never
// replicated), and produces the output towers of its Q range.  Two
// exchanges are needed:
//   1. prep      ModUp P1 of the rank's input towers (iNTT, (Q_j/q_i)^-1)
//                -> y_own;                    all-gather y (every digit's
//                sources are needed by every target tower);
//   2. keyprod   ModUp P2/P3 of every digit to the rank's towers (Q and P),
//                the key product summed over digits (P4+P5) -> c'_own; for
//                the rank's special towers also ModDown P1 (iNTT, the
//                (P/p_k)^-1 factor folded into the key) -> w_own;
//                                             all-gather w (every Q tower's
//                ModDown needs all K special towers);
//   3. moddown   ModDown P2-P4 of the rank's Q towers from the gathered w
//                -> out0_own, out1_own.
// The exchanges are the caller's (NCCL all-gather, or copies between
// devices); this file holds the per-rank device work.  Every step uses the
// same kernels and arithmetic as the single-device key switch, so the
// gathered outputs are bit-identical to ks_switch's.
#include <algorithm>

#include "ks_device.cuh"
#include "ks_launch.h"

namespace ks {

namespace {

// The rank's towers at level nact: active Q towers [q0, q1) (possibly
// none), special towers [p0, p1); slot s < nq is Q tower q0+s, slot nq + k'
// special tower p0+k'.
struct ShardLv {
    int q0, q1, p0, p1;
    int nq, np, nown;
    int kq;  // Q limbs per digit and polynomial in the shard key (full level)
};

ShardLv shard_level(const ks_shard &sh, int nact)
{
    ShardLv L;
    L.q0 = std::min<int>((int)sh.q_begin, nact);
    L.q1 = std::min<int>((int)sh.q_end, nact);
    L.p0 = (int)sh.p_begin;
    L.p1 = (int)sh.p_end;
    L.nq = L.q1 - L.q0;
    L.np = L.p1 - L.p0;
    L.nown = L.nq + L.np;
    L.kq = (int)(sh.q_end - sh.q_begin);
    return L;
}

int check_shard(const ks_params *P, const ks_shard *sh)
{
    if (!sh) return fail(KS_EINVAL, "shard is NULL");
    if (sh->q_begin > sh->q_end || sh->q_end > (uint32_t)P->nq || sh->p_begin > sh->p_end ||
        sh->p_end > (uint32_t)P->kp)
        return fail(KS_EINVAL, "shard ranges must satisfy q_begin <= q_end <= n_q and p_begin <= p_end <= k_p");
    return KS_OK;
}

ks_shard key_shard_of(const ks_key *K) { return ks_shard{K->q0, K->q1, K->p0, K->p1}; }

// Key product of the rank's towers: grid (N/256, nown).  D holds, per
// active digit j, the rank's raised limbs [j][slot][N] (lazy NTT output);
// the bypassed digit of a Q tower reads the input tower d_own[slot].  The
// shard key's limb of (digit j, polynomial x, slot) is at
// key[((2j+x)*kown + kslot)*N], kslot = slot for Q towers and kq + (k - p_begin)
// for special tower k.
__global__ void __launch_bounds__(256) k_shard_keyprod(Tables T, int nact, int nd, ShardLv L, int kown, const u64 *d_own,
                                                       const u64 *D, const u64 *key, u64 *cp_own)
{
    const int s = blockIdx.y;
    const bool isq = s < L.nq;
    const int t = isq ? L.q0 + s : nact + L.p0 + (s - L.nq);  // compact tower at the level
    const int tf = full_tower(t, nact, T.nq);
    // the rank's active Q towers start at q_begin (q0 == q_begin whenever
    // nq > 0), its special towers at p_begin: key slots s and kq + (s - nq)
    const int kslot = isq ? s : L.kq + (s - L.nq);
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ModC &mc = T.modc[tf];
    U128 sb = {0, 0}, sa = {0, 0};
    for (int j = 0; j < nd; ++j) {
        const bool own = isq && t / T.alpha == j;
        const u64 dv = own ? d_own[(size_t)s * N + n] : D[((size_t)j * L.nown + s) * N + n];
        mac128(sb, dv, key[((size_t)(2 * j) * kown + kslot) * N + n]);
        mac128(sa, dv, key[((size_t)(2 * j + 1) * kown + kslot) * N + n]);
    }
    cp_own[(size_t)s * N + n] = reduce_any(redc(sb, mc.q, mc.mont), mc.q, mc.one_sh);
    cp_own[((size_t)L.nown + s) * N + n] = reduce_any(redc(sa, mc.q, mc.mont), mc.q, mc.one_sh);
}

// ModDown P4 of the rank's Q towers: out_x[s] = c'_x[s] - v_x[s] mod q (P^-1
// folded into the key), v lazy NTT output below kFwdLazy*q.  grid (N/256, nq, 2).
__global__ void __launch_bounds__(256) k_shard_final(Tables T, ShardLv L, const u64 *cp_own, const u64 *v, u64 *out0,
                                                     u64 *out1)
{
    const int s = blockIdx.y, x = blockIdx.z;
    const size_t N = (size_t)1 << T.logN;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ModC &mc = T.modc[L.q0 + s];
    const u64 r = cp_own[((size_t)x * L.nown + s) * N + n] + kFwdLazy * mc.q - v[((size_t)x * L.nq + s) * N + n];
    (x == 0 ? out0 : out1)[(size_t)s * N + n] = reduce_any(r, mc.q, mc.one_sh);
}

int cuda_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(KS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return KS_OK;
}

int set_dev(const ks_params *P)
{
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    return KS_OK;
}

int check_level(const ks_params *P, uint32_t nact)
{
    if (nact < 1 || nact > (uint32_t)P->nq) return fail(KS_EINVAL, "level_towers must be in 1..n_q");
    return KS_OK;
}

int check_shard_key(const ks_params *P, const ks_key *K)
{
    if (!K || K->params != P || !K->shard) return fail(KS_EINVAL, "key must be a tower shard of this params object");
    return KS_OK;
}

}  // namespace

}  // namespace ks

using namespace ks;

extern "C" {

int ks_key_shard(const ks_key *full, const ks_shard *sh, ks_stream_t stream, ks_key **out)
{
    if (!full || !out) return fail(KS_EINVAL, "NULL argument");
    *out = nullptr;
    const ks_params *P = full->params;
    int rc = check_shard(P, sh);
    if (rc) return rc;
    if (full->shard || full->compressed) return fail(KS_EINVAL, "ks_key_shard needs a full (uncompressed) key");
    if ((rc = set_dev(P)) != KS_OK) return rc;
    const size_t N = P->N;
    const int nfull = P->nq + P->kp;
    const int kq = (int)(sh->q_end - sh->q_begin), kp = (int)(sh->p_end - sh->p_begin);
    const int kown = kq + kp;
    ks_key *K = new ks_key();
    K->params = P;
    K->shard = 1;
    K->q0 = sh->q_begin;
    K->q1 = sh->q_end;
    K->p0 = sh->p_begin;
    K->p1 = sh->p_end;
    K->bytes = (size_t)P->ndig * 2 * kown * N * sizeof(u64);
    cudaStream_t st = (cudaStream_t)stream;
    if (K->bytes > 0 && cudaMalloc((void **)&K->d_evk, K->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete K;
        return fail(KS_ENOMEM, "shard key allocation failed");
    }
    // per (digit, polynomial): the Q range and the special range are each
    // one contiguous run of limbs in the full key
    for (int jx = 0; jx < 2 * P->ndig && rc == KS_OK; ++jx) {
        const u64 *src = full->d_evk + (size_t)jx * nfull * N;
        u64 *dst = K->d_evk + (size_t)jx * kown * N;
        if (kq > 0 &&
            cudaMemcpyAsync(dst, src + (size_t)sh->q_begin * N, (size_t)kq * N * 8, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            rc = fail(KS_ECUDA, "shard key copy");
        if (rc == KS_OK && kp > 0 &&
            cudaMemcpyAsync(dst + (size_t)kq * N, src + ((size_t)P->nq + sh->p_begin) * N, (size_t)kp * N * 8,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = fail(KS_ECUDA, "shard key copy");
    }
    if (rc == KS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(KS_ECUDA, "shard key copy");
    if (rc != KS_OK) {
        cudaGetLastError();
        if (K->d_evk) cudaFree(K->d_evk);
        delete K;
        return rc;
    }
    *out = K;
    return KS_OK;
}

size_t ks_shard_scratch_words(const ks_params *P, const ks_shard *sh, uint32_t nact)
{
    if (!P || !sh || check_shard(P, sh) != KS_OK || check_level(P, nact) != KS_OK) return 0;
    const ShardLv L = shard_level(*sh, (int)nact);
    const size_t nd = ((size_t)nact + P->alpha - 1) / P->alpha;
    return (nd * L.nown + 2 * (size_t)L.nq) * P->N;
}

int ks_shard_prep(const ks_params *P, const ks_shard *sh, uint32_t nact, const uint64_t *d_own, uint64_t *y_own,
                  ks_stream_t stream)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    int rc = check_shard(P, sh);
    if (rc || (rc = check_level(P, nact)) != KS_OK) return rc;
    const ShardLv L = shard_level(*sh, (int)nact);
    if (L.nq == 0) return KS_OK;
    if (!d_own || !y_own) return fail(KS_EINVAL, "NULL data pointer");
    if ((rc = set_dev(P)) != KS_OK) return rc;
    // iNTT with the ModUp P1 factor of each tower at this level
    const ulonglong2 *pre = P->d_up_pre_lvl + (size_t)(nact - 1) * P->nq + L.q0;
    LimbMap m{d_own, y_own, pre, L.nq, L.nq, 0, L.q0, (int)nact, -1};
    return launch_ntt_inv(P->tables, one_map(m, L.nq), false, (cudaStream_t)stream);
}

int ks_shard_keyprod(const ks_params *P, const ks_key *K, uint32_t nact, const uint64_t *y_all, const uint64_t *d_own,
                     uint64_t *cp_own, uint64_t *scratch, ks_stream_t stream)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    int rc = check_shard_key(P, K);
    if (rc || (rc = check_level(P, nact)) != KS_OK) return rc;
    const ks_shard sh = key_shard_of(K);
    const ShardLv L = shard_level(sh, (int)nact);
    if (L.nown == 0) return KS_OK;
    if (!y_all || !cp_own || !scratch || (L.nq > 0 && !d_own)) return fail(KS_EINVAL, "NULL data pointer");
    if ((rc = set_dev(P)) != KS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const Tables &T = P->tables;
    const size_t N = P->N;
    const int na = (int)nact;
    const int nd = (na + P->alpha - 1) / P->alpha;
    u64 *D = scratch;  // [nd][nown][N]
    // ModUp P2: every digit to the rank's Q towers and special towers
    BUpJobs bu;
    bu.n = 0;
    if (L.nq > 0) add_bup(bu, T, BUpJob{y_all, D, (size_t)L.nown * N, na, L.q0, L.q1, L.q0, -1});
    if (L.np > 0)
        add_bup(bu, T, BUpJob{y_all, D + (size_t)L.nq * N, (size_t)L.nown * N, na, na + L.p0, na + L.p1, na + L.p0, -1});
    if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;
    // ModUp P3: their NTTs (the Q towers' own digit is bypassed)
    LimbMaps mf;
    mf.n = 0;
    if (L.nq > 0) add_map(mf, LimbMap{D, D, nullptr, L.nq, L.nown, 0, L.q0, na, 0}, nd * L.nq);
    if (L.np > 0) add_map(mf, LimbMap{D, D, nullptr, L.np, L.nown, L.nq, na + L.p0, na, -1}, nd * L.np);
    if ((rc = launch_ntt_fwd(T, mf, false, st)) != KS_OK) return rc;
    // ModUp P4+P5: key product summed over the digits
    KS_LAUNCH(st, "shard_keyprod",
              k_shard_keyprod<<<dim3((unsigned)(N / 256), (unsigned)L.nown), 256, 0, st>>>(
                  T, na, nd, L, L.kq + (int)(sh.p_end - sh.p_begin), d_own, D, K->d_evk, cp_own));
    if ((rc = cuda_status("shard key product launch")) != KS_OK) return rc;
    // ModDown P1 of the special towers, in place (factor folded into the key)
    if (L.np > 0) {
        LimbMap mw{cp_own, cp_own, nullptr, L.np, L.nown, L.nq, na + L.p0, na, -1};
        if ((rc = launch_ntt_inv(T, one_map(mw, 2 * L.np), false, st)) != KS_OK) return rc;
    }
    return KS_OK;
}

int ks_shard_moddown(const ks_params *P, const ks_key *K, uint32_t nact, const uint64_t *w_all, const uint64_t *cp_own,
                     uint64_t *out0_own, uint64_t *out1_own, uint64_t *scratch, ks_stream_t stream)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    int rc = check_shard_key(P, K);
    if (rc || (rc = check_level(P, nact)) != KS_OK) return rc;
    const ks_shard sh = key_shard_of(K);
    const ShardLv L = shard_level(sh, (int)nact);
    if (L.nq == 0) return KS_OK;
    if (!w_all || !cp_own || !out0_own || !out1_own || !scratch) return fail(KS_EINVAL, "NULL data pointer");
    if ((rc = set_dev(P)) != KS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const Tables &T = P->tables;
    const size_t N = P->N;
    const int na = (int)nact;
    const int nd = (na + P->alpha - 1) / P->alpha;
    u64 *v = scratch + (size_t)nd * L.nown * N;  // [2][nq][N]
    // ModDown P2: the gathered w (both polynomials) to the rank's Q towers
    BDnJobs bd;
    bd.n = 0;
    BDnJob j{nullptr, 0, v, (size_t)L.nq * N, na, 2};
    j.i_begin = L.q0;
    j.i_end = L.q1;
    j.w = w_all;
    j.w_stride = (size_t)P->kp * N;
    add_bdn(bd, j);
    if ((rc = launch_bconv_down(T, bd, st)) != KS_OK) return rc;
    // ModDown P3, then P4
    LimbMap mv{v, v, nullptr, L.nq, L.nq, 0, L.q0, na, -1};
    if ((rc = launch_ntt_fwd(T, one_map(mv, 2 * L.nq), false, st)) != KS_OK) return rc;
    KS_LAUNCH(st, "shard_final",
              k_shard_final<<<dim3((unsigned)(N / 256), (unsigned)L.nq, 2), 256, 0, st>>>(T, L, cp_own, v, out0_own,
                                                                                         out1_own));
    return cuda_status("shard final launch");
}

}  // extern "C"
