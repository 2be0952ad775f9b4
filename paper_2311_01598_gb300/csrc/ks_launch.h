// ks_launch.h -- host-side launchers of the key-switching kernels.
#pragma once
#include "ks_internal.h"

namespace ks {

// A set of limbs addressed arithmetically.  Limb l of the set is entry
// b = l % per of limb-row a = l / per; it lives at (a*row_stride + aoff + b)*N
// words from src/dst and belongs to compact tower t = toff + b of the level
// basis D_l (Q towers 0..nact-1, then the K special towers).  With
// skip_base >= 0, limbs whose tower lies inside digit a + skip_base are
// skipped (the ModUp bypass); -1 skips nothing.
struct LimbMap {
    const u64 *src;
    u64 *dst;
    int per;
    int row_stride;
    int aoff;
    int toff;
    int nact;
    int skip_base;
};

__host__ __device__ inline int full_tower(int t, int nact, int nq) { return t < nact ? t : nq + (t - nact); }

// Single passes (column pass of the forward NTT, column pass of the inverse
// NTT with the same scale options as launch_ntt_inv).
int launch_fwd_col(const Tables &T, const LimbMap &m, int nlimbs, cudaStream_t st);
int launch_inv_col(const Tables &T, const LimbMap &m, int nlimbs, const ulonglong2 *scale, bool scale_by_ninv,
                   cudaStream_t st);
// ModUp P2 for digits [0, nd) restricted to targets of compact tower index
// in [t_begin, t_end) (outside the digit); output row t goes to
// D + j*dstride + (t - t_base)*N.
int launch_bconv_up_range(const Tables &T, int nact, int t_begin, int t_end, int t_base, const u64 *y, u64 *D,
                          size_t dstride, cudaStream_t st);

// Forward NTT (column pass src->dst, row pass in place on dst).  Input in
// [0, 4q); output canonical or lazy in [0, 4q).
int launch_ntt_fwd(const Tables &T, const LimbMap &m, int nlimbs, bool canonical, cudaStream_t st);
// Inverse NTT without the N^-1 factor (row pass src->dst, column pass in
// place); the column pass multiplies limb b by scale[b] when scale is set
// (the Shoup pair of the wanted factor), and the output is canonical.
int launch_ntt_inv(const Tables &T, const LimbMap &m, int nlimbs, const ulonglong2 *scale, bool scale_by_ninv,
                   cudaStream_t st);

// ModUp P2 over all active digits: y [nact][N] canonical coefficient form ->
// D [nd][nact+K][N] (entries outside each digit), lazy [0, 2r).
int launch_bconv_up(const Tables &T, int nact, const u64 *y, u64 *D, cudaStream_t st);
// Same for one digit j only (Digit-Centric).
int launch_bconv_up_digit(const Tables &T, int nact, int j, const u64 *y, u64 *Dj, cudaStream_t st);
// ModUp P4+P5: cp[x][t] = sum_j D_{j,t} * evk_{j,x,t}, D_{j,t} = d_t inside digit j.
// accumulate: add to the existing cp (Digit-Centric partial sums).
int launch_apply_key(const Tables &T, int nact, int j_begin, int j_end, const u64 *d, const u64 *D,
                     size_t D_digit_stride, const u64 *evk, u64 *cp, bool accumulate, cudaStream_t st);
// ModDown P2: w = cp[x][nact..nact+K) canonical coefficient form ->
// v[x][i] = sum_k w_k * p_k^-1 mod q_i, lazy [0, 2q).  npoly polynomials,
// cp rows strided by cp_stride words, v rows by v_stride words.
int launch_bconv_down(const Tables &T, int nact, int npoly, const u64 *cp, size_t cp_stride, u64 *v,
                      size_t v_stride, cudaStream_t st);
// ModDown P4 (P^-1 already folded): out_x[i] = cp[x][i] - v[x][i] mod q_i.
int launch_down_final(const Tables &T, int nact, int npoly, const u64 *cp, size_t cp_stride, const u64 *v,
                      size_t v_stride, u64 *const *outs, cudaStream_t st);
// Multiply limbs by per-tower factors (plain, Shoup) and canonicalise:
// used by the stage entry points that take unscaled inputs.
int launch_scale(const Tables &T, const LimbMap &m, int nlimbs, const ulonglong2 *factors_full, cudaStream_t st);
// Copy the input towers of every digit into D (ModUp bypass, stage entry).
int launch_bypass_copy(const Tables &T, int nact, const u64 *d, u64 *D, cudaStream_t st);
// Canonicalise limbs in [0, 4q).
int launch_canon(const Tables &T, const LimbMap &m, int nlimbs, cudaStream_t st);

// Key preparation: canonical evk [ndig][2][nq+kp][N] -> stored form
// (times key_sc[t], Montgomery factor included), in place.
int launch_key_convert(const Tables &T, u64 *evk, cudaStream_t st);
// Key generation combine on the device: inputs are residues already in
// evaluation form; b_j = -a_j*s + e_j + g_j*s' per tower (g_j = [P]_{q_i} on
// the digit's towers).  a is read from the a-slots of evk, e_hat [ndig][nt][N].
int launch_keygen_combine(const Tables &T, const u64 *s_hat, const u64 *sp_hat, const u64 *e_hat,
                          const u64 *pmod, u64 *evk, cudaStream_t st);
// Signed coefficients -> residues per tower: out[t][n] = v[n] mod r_t.
int launch_signed_to_towers(const Tables &T, const int64_t *v, int nvec, u64 *out, cudaStream_t st);

// Output-Centric fused kernels.
// prescale: ModUp P1 factors of the level (nact Shoup pairs).
int launch_oc(const Tables &T, int nact, const u64 *d, const u64 *evk, u64 *out0, u64 *out1, u64 *y, u64 *tmp,
              u64 *cp, const ulonglong2 *prescale, cudaStream_t st);

}  // namespace ks
