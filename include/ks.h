/*
 * ks.h -- C ABI of the GB300 (sm_103a) RNS hybrid key-switching library.
 *
 * The operation is hybrid key switching (HKS) of CKKS as laid out in CiFlow
 * (arxiv 2311.01598), Sec. III: ModUp (P1 iNTT, P2 BConv, P3 NTT, P4 apply
 * key, P5 reduce over digits) followed by ModDown (P1 iNTT of the K special
 * towers, P2 BConv to the Q towers, P3 NTT, P4 subtract and scale by P^-1),
 * scheduled under the Max-Parallel, Digit-Centric or Output-Centric
 * dataflow of Sec. IV.  All dataflows return bit-identical results: the
 * paper notes that the operation count of HKS does not depend on the
 * dataflow (Sec. IV, arithmetic-intensity comparison with Table II), and
 * every step here is exact integer arithmetic.
 *
 * Conventions shared by every entry point:
 *   - A polynomial over a set of primes is stored limb-major: tower t
 *     occupies words [t*N, (t+1)*N), one uint64 residue per coefficient or
 *     slot, canonical in [0, prime).  Q towers come first (q_0..q_l), then
 *     the K special towers (p_0..p_{K-1}) where those appear.
 *   - Evaluation form (Sec. II, NTT domain): slot k holds the value at
 *     psi^(2*brv(k)+1), brv the logN-bit reversal, psi the primitive 2N-th
 *     root fixed by the prime rule of ks_params_create.
 *   - Pointers named d_* are device pointers owned by the caller; pointers
 *     named h_* are host pointers owned by the caller.  Handles (ks_params,
 *     ks_key) are owned by the library and freed by their destroy call.
 *   - Every call returns KS_OK (0) or a negative ks_status.  Argument errors
 *     are detected on the host before any launch; ks_last_error() then
 *     returns a message for the calling thread.  Device work is queued
 *     asynchronously on the given stream (0 = legacy default stream);
 *     errors raised by already-queued device work surface on a later call
 *     or on the caller's synchronisation.
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ks_params ks_params; /* library-owned parameter set          */
typedef struct ks_key ks_key;       /* library-owned device-resident evk    */
typedef void *ks_stream_t;          /* a cudaStream_t                       */

typedef enum {
    KS_OK = 0,
    KS_EINVAL = -1,       /* bad argument (caught before any launch)         */
    KS_ENOMEM = -2,       /* device or host allocation failed                */
    KS_ECUDA = -3,        /* a CUDA runtime call failed                      */
    KS_ETIMEOUT = -4,     /* a bounded device wait ran out                   */
    KS_EUNSUPPORTED = -5  /* valid request outside what this build supports  */
} ks_status;

/* Dataflows of CiFlow Sec. IV. */
typedef enum {
    KS_MP = 0,  /* Max-Parallel (Sec. IV-A): one stage at a time over all
                   towers, every intermediate materialised in device memory */
    KS_DC = 1,  /* Digit-Centric (Sec. IV-B): ModUp P1-P5 one digit at a
                   time, partial sums accumulated, then ModDown            */
    KS_OC = 2,  /* Output-Centric (Sec. IV-C): BConv only to the towers of
                   the section being produced, the key product and P5
                   reduce fused into the NTT row pass; the special towers
                   first, then the Q towers with ModDown fused in           */
    KS_AUTO = 3 /* let the library choose (autotuned schedule cache)         */
} ks_dataflow;

/* Message for the last failed call on this thread ("" if none). */
const char *ks_last_error(void);

/* Create a parameter set (Table I of the paper: N, Q = q_0..q_L, P =
 * p_0..p_{K-1}, dnum digits of alpha = ceil((L+1)/dnum) towers).
 *   logN      : ring degree N = 2^logN, 10 <= logN <= 17
 *   n_q       : L+1 Q primes, 1 <= n_q <= 64
 *   k_p       : K special primes, 1 <= k_p <= 32
 *   dnum      : number of digits, 1 <= dnum <= n_q
 *   h_q, h_p  : optional explicit primes (both or neither; each must be a
 *               prime = 1 mod 2N below 2^56, all distinct).  With NULL the
 *               prime rule applies: the n_q+k_p largest primes below
 *               2^prime_bits that are 1 mod 2N, descending; the first k_p
 *               become p_0.., the rest q_0, q_1, ...
 *   prime_bits: 30..56, used only when h_q/h_p are NULL.
 * Uploads twiddle and base-conversion tables to the current device.
 * On success *out receives the handle. */
int ks_params_create(uint32_t logN, uint32_t n_q, uint32_t k_p, uint32_t dnum,
                     const uint64_t *h_q, const uint64_t *h_p, uint32_t prime_bits,
                     ks_params **out);
void ks_params_destroy(ks_params *params);

/* The count largest primes below 2^bits of the special form k*2^32 + 1
 * (descending; each is 1 mod 2N for every supported N), for explicit prime
 * lists (h_q/h_p of ks_params_create).  The paper fixes no primes; the
 * default rule of ks_params_create (largest primes = 1 mod 2N) does not
 * produce this form.  When every prime of a parameter set has it, the
 * two-pass NTT kernels use a cheaper butterfly product (q*E mod 2^64 is
 * E + ((E mod 2^32)*k mod 2^32)*2^32), with identical results.  Host only
 * (no device work).  bits in 33..56; KS_EINVAL when fewer than count exist. */
int ks_special_primes(uint32_t bits, uint32_t count, uint64_t *h_out);

/* Read back the primes (h_q: n_q words, h_p: k_p words; either may be NULL)
 * and the digit geometry. */
int ks_params_info(const ks_params *params, uint64_t *h_q, uint64_t *h_p,
                   uint32_t *alpha, uint32_t *n_digits);

/* Implementation options of a parameter set (none changes any result).
 *   KS_OPT_BCONV_TENSOR (default 1): run the fast base conversions (ModUp P2,
 *     ModDown P2) on the tensor cores (tcgen05, exact f16 slices)
 *     wherever at most 18 source towers meet N >= 2^7; 0 selects the CUDA-core
 *     kernels everywhere.
 *   KS_OPT_BATCH_LANES (default 2, 1..4): an Output-Centric batch of at least
 *     4 jobs per lane is split over that many library streams, forked from
 *     and joined back to the caller's stream (the memory-bound combine
 *     kernels of one part then overlap the integer-bound passes of another);
 *     1 keeps every launch on the caller's stream.
 *   KS_OPT_NTT_CLUSTER (default 0): run each NTT (forward and inverse) as
 *     one launch in which a thread-block cluster transforms a limb, its
 *     column and row passes exchanging the limb through distributed shared
 *     memory, instead of two launches through device memory.  Ring degrees
 *     without a cluster form (2^13, 2^17) keep the two launches.
 *   KS_OPT_NTT_ROW_STAGE (0 or 1): run the forward row passes as persistent
 *     blocks whose row blocks are staged in shared memory by bulk copies
 *     (the next block's copy in flight while the current one is
 *     transformed).  Row-pass inputs that are not 16-byte aligned keep the
 *     plain pass.  Same results.
 * Returns KS_EINVAL for an unknown option or value.  Not thread-safe with
 * concurrent calls on the same params object. */
enum { KS_OPT_BCONV_TENSOR = 1, KS_OPT_BATCH_LANES = 2, KS_OPT_NTT_CLUSTER = 3, KS_OPT_NTT_ROW_STAGE = 4 };
int ks_params_set_option(ks_params *params, int option, int value);

/* Device-side status of the library on the params object's GPU: bit 0 is set
 * when a tensor-core kernel gave up waiting for its MMAs, bit 1 when a staged
 * row pass gave up waiting for a bulk copy (bounded waits), since the last
 * call with clear = 1; the outputs of that work are then not valid.  Returns
 * KS_OK, or KS_ECUDA if the flags cannot be read. */
int ks_device_status(const ks_params *params, int clear, uint32_t *flags);

/* Generate and upload an evaluation key switching s' -> s (hybrid key):
 *   b_j = -a_j*s + e_j + [P*g_j]*s',  a_j uniform, e_j rounded Gaussian
 *   (sigma 3.2, |e| <= 19), g_j the CRT idempotent of digit j.
 * Sampling is on the host from SplitMix64 streams seed^0 (a_j: digit, then
 * tower q_0..q_L,p_0..p_{K-1}, then coefficient) and seed^1 (e_j: digit,
 * then coefficient); NTTs and the key combination run on the device.
 *   h_s       : N coefficients of s in {-1,0,1}
 *   h_s_prime : N signed coefficients of s' (|s'_i| < 2^62)
 * The key stays resident in device memory until ks_key_destroy. */
int ks_keygen_upload(const ks_params *params, const int8_t *h_s, const int64_t *h_s_prime,
                     uint64_t seed, ks_stream_t stream, ks_key **out);

/* Compressed key (Sec. IV-D: regenerating a key's uniform half from a seed
 * halves the key's data movement).  Same relation and e_j stream as
 * ks_keygen_upload, but a_j is defined by counter-addressed SplitMix64 so it
 * can be regenerated anywhere:  a-word (j, t, n) (t the full tower index
 * q_0..q_L, p_0..p_{K-1}) is the first draw
 *   SM(seed^2, ((j*(n_q+k_p) + t)*N + n)*64 + m) & mask(bitlen(r_t)),
 * m = 0..63, below r_t (if all 64 reject, the last one mod r_t), where
 * SM(x, c) is output c (from 0) of the SplitMix64 stream seeded with x.
 * Only b_j is stored (half the device memory of a full key); the kernels
 * regenerate a_j while they form the key product.  A compressed key works
 * with every entry point; Output-Centric schedules asking for the fused
 * variant run the split variant for batches that contain one. */
int ks_keygen_upload_compressed(const ks_params *params, const int8_t *h_s, const int64_t *h_s_prime,
                                uint64_t seed, ks_stream_t stream, ks_key **out);

/* Upload a key given in the canonical layout
 *   evk[digit j < n_digits][b=0 / a=1][tower q_0..q_L, p_0..p_{K-1}][N]
 * (evaluation form, canonical).  h_evk is host memory. */
int ks_key_upload_raw(const ks_params *params, const uint64_t *h_evk, ks_stream_t stream,
                      ks_key **out);
void ks_key_destroy(ks_key *key);
/* Bytes of device memory the key occupies. */
size_t ks_key_bytes(const ks_key *key);

/* Key switch one polynomial (Sec. III; Fig. 1 of the paper).
 *   level_towers : l+1 active Q towers, 1 <= l+1 <= n_q.  Digit j covers
 *                  towers [j*alpha, min((j+1)*alpha, l+1)); the key's towers
 *                  outside D_l = {q_0..q_l} u P are not read.
 *   d_in         : device [l+1][N], evaluation form, canonical; not written.
 *   d_out0/out1  : device [l+1][N]; receive (out0, out1) with
 *                  out0 + out1*s = d*s' + small noise (mod Q_l), canonical.
 *                  Must not overlap d_in or each other.
 * d_in, d_out0 and d_out1 must be 16-byte aligned (every cudaMalloc and
 * torch allocation is; an offset view may not be): KS_EINVAL otherwise.
 * The same holds for the jobs of every batched, hoisted and host-staged
 * call.  Device scratch is owned by the params object, one set per stream;
 * calls on different streams may overlap. */
int ks_switch(const ks_params *params, const ks_key *key, uint32_t level_towers,
              const uint64_t *d_in, uint64_t *d_out0, uint64_t *d_out1, ks_dataflow dataflow,
              ks_stream_t stream);

/* Hoisted rotations (Sec. II: a rotation needs the key switch of a Galois
 * automorphism X -> X^g; hoisting shares one ModUp among several).
 * For r < n_rot, with g_r = galois[r] (odd, < 2N) and keys[r] a key from
 * s(X^g_r) to s:
 *   (out0[r], out1[r]) = ModDown( sum_j phi_r(ModUp_j(d)) * evk_r,j )
 * where phi_r permutes the evaluation slots as X -> X^g_r (slot k takes slot
 * k' with 2brv(k')+1 = (2brv(k)+1) g_r mod 2N).  So out0[r] + out1[r]*s =
 * phi_r(d)*s(X^g_r) + small noise: the key-switched second component of a
 * ciphertext rotated by g_r (the caller applies phi_r to the first).  The
 * digits of d are raised once for all rotations, so the result differs
 * (within the same noise bound) from ks_switch of phi_r(d).  g_r = 1 gives
 * ks_switch exactly.
 *   level_towers, d_in : as ks_switch (device, evaluation form).
 *   d_out0, d_out1     : host arrays of n_rot device pointers to [l+1][N];
 *                        none may overlap d_in or one another.
 * Scratch: the params object's per-stream workspace plus 2*(2l+2+K)*N words
 * per rotation in flight (up to 64 at a time).  n_rot = 0 is a no-op. */
int ks_switch_hoisted(const ks_params *params, uint32_t n_rot, const ks_key *const *keys, const uint64_t *galois,
                      uint32_t level_towers, const uint64_t *d_in, uint64_t *const *d_out0, uint64_t *const *d_out1,
                      ks_stream_t stream);

/* The automorphism X -> X^g of a polynomial in evaluation form (Sec. II:
 * the slot permutation of a rotation): slot k of the output takes slot k' of
 * the input with 2brv(k')+1 = (2brv(k)+1) g mod 2N, tower by tower.  With
 * accumulate = 1 the result is added to d_out mod q (so a rotation by g is
 * (phi_g(c0) + out0, out1) with out0, out1 from ks_switch_hoisted of c1).
 *   first_tower, n_towers : towers of the full basis (Q towers 0..n_q-1, then
 *                           the K special towers) held by d_in and d_out;
 *   galois                : odd, below 2N;
 *   d_in, d_out           : device [n_towers][N], canonical; must not overlap.
 * n_towers = 0 is a no-op. */
int ks_automorph(const ks_params *params, uint32_t first_tower, uint32_t n_towers, uint64_t galois,
                 const uint64_t *d_in, uint64_t *d_out, int accumulate, ks_stream_t stream);

/* One job of a batched key switch. */
typedef struct {
    const ks_key *key;
    uint32_t level_towers;
    const uint64_t *d_in;
    uint64_t *d_out0;
    uint64_t *d_out1;
} ks_job;

/* Key switch n independent jobs (uneven levels, each with its own key) in
 * one batched launch sequence on `stream`.  Each output equals what
 * ks_switch gives for the same job.  h_jobs is host memory. */
int ks_switch_batch(const ks_params *params, uint32_t n, const ks_job *h_jobs,
                    ks_dataflow dataflow, ks_stream_t stream);

/* Key switch without allocating (the paper has no counterpart; this is a
 * deployment aid).  For callers that cannot allocate device memory while
 * running -- e.g. a server whose device memory is wholly owned by its own
 * pool allocator, or a loop that cannot afford cudaMalloc's device-wide
 * synchronisation.  Same inputs, outputs and result as ks_switch with
 * KS_OC, but the scratch is one static device array of
 * ks_switch_noalloc_max_words() words (32 MiB), reserved on every GPU that
 * loads the library until the process exits.
 *   - Argument errors are refused as ks_switch refuses them (KS_EINVAL
 *     before any launch): level outside 1..n_q, NULL, overlapping, or not
 *     16-byte aligned d_in/d_out0/d_out1.
 *   - The scratch needed is (nact + nd*(nact+K) + 2*nact + 2*(nact+K)) * N
 *     words at level nact (nd = active digits); e.g. N=2^16, 24+8 primes,
 *     dnum 3 at the top level needs 232 limbs, 15.2 million words.
 *     Requests needing more than the array holds fail with KS_EINVAL and a
 *     message giving both sizes; nothing runs.
 *   - Runs with the parameter set's current schedule and engines (as
 *     ks_switch with KS_OC does, including after ks_set_default_schedule).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 *   - All calls share the one array: calls that may overlap on the GPU (on
 *     different streams without ordering between them) race and must not be
 *     issued.  Nothing in the array needs to start at zero.
 *   - The array's address is kept for the life of the process:
 *     cudaDeviceReset while the library is in use is not supported (it also
 *     frees every params object's and key's device memory). */
int ks_switch_noalloc(const ks_params *params, const ks_key *key, uint32_t level_towers,
                      const uint64_t *d_in, uint64_t *d_out0, uint64_t *d_out1, ks_stream_t stream);
/* Words of the static scratch array of ks_switch_noalloc. */
size_t ks_switch_noalloc_max_words(void);

/* ---------------------------------------------------------------------
 * Stage entry points (the individual steps of Sec. III; used by the
 * parity tests and available to callers composing their own schedules).
 * ------------------------------------------------------------------- */

/* Forward (inverse = 0) or inverse (inverse = 1) negacyclic NTT of
 * n_towers limbs stored contiguously at d_data, in place.  Limb i uses
 * tower (first_tower + i) of the full-level basis q_0..q_L, p_0..p_{K-1}.
 * Input canonical; output canonical.  The inverse includes the N^-1
 * factor. */
int ks_ntt(const ks_params *params, uint32_t first_tower, uint32_t n_towers, uint64_t *d_data,
           int inverse, ks_stream_t stream);

/* ModUp (Sec. III-B, P1-P3) at level l+1 = level_towers: d_in [l+1][N]
 * -> d_ext [n_active_digits][l+1+K][N] in evaluation form over D_l (Q
 * towers then P towers); row j holds digit j raised to D_l, its own towers
 * being the input towers.  Values canonical. */
int ks_modup(const ks_params *params, uint32_t level_towers, const uint64_t *d_in,
             uint64_t *d_ext, ks_stream_t stream);

/* ModDown (Sec. III-C, P1-P4) of one polynomial c' over D_l:
 * d_cp [l+1+K][N] evaluation form -> d_out [l+1][N] = (c' - NTT(BConv(
 * iNTT(c'_P)))) * P^-1 (mod q_i).  Values canonical. */
int ks_moddown(const ks_params *params, uint32_t level_towers, const uint64_t *d_cp,
               uint64_t *d_out, ks_stream_t stream);

/* A schedule: how a batch is executed.  All schedules give identical
 * results; they differ in speed only. */
typedef struct {
    int32_t dataflow;    /* KS_MP, KS_DC or KS_OC                                  */
    int32_t oc_variant;  /* KS_OC: 0 = fused row kernels (row pass, key product,
                            ModDown step in one kernel per row block), 1 = split
                            (plain row pass, then a streaming combine kernel),
                            2 = whole basis (one base conversion and one NTT
                            launch over every raised limb, then the combines),
                            3 = one thread-block-cluster kernel per output
                            tower (ModUp base conversion, NTTs, key product,
                            ModDown, subtraction with the tower's limbs on
                            chip; ring degrees with a cluster geometry and
                            full keys, else run as 1)                          */
    int32_t chunk;       /* KS_OC: jobs per batched launch group, 1..64           */
    int32_t order;       /* 0 = jobs in the given order, 1 = grouped by level
                            (descending), 2 = grouped by key (KS_OC: jobs of a
                            launch sharing a key also share each read of its
                            limbs in the combine kernels)                        */
    int32_t ntt;         /* NTT form: 0 = two launches (column pass, row pass),
                            1 = one cluster launch per NTT (KS_OPT_NTT_CLUSTER),
                            2 = the same with CTAs twice as wide; -1 = the
                            parameter set's option                               */
    int32_t bconv;       /* base conversion engine: 0 = CUDA cores, 1 = tensor
                            cores where supported; -1 = the parameter set's
                            option (KS_OPT_BCONV_TENSOR)                         */
} ks_schedule;

/* Batched key switch with an explicit schedule (see ks_schedule). */
int ks_switch_batch_sched(const ks_params *params, uint32_t n, const ks_job *h_jobs,
                          const ks_schedule *schedule, ks_stream_t stream);

/* The schedule KS_OC and KS_AUTO use when no tuned entry applies
 * (initially: Output-Centric, split variant, chunk 64, given order). */
int ks_get_default_schedule(const ks_params *params, ks_schedule *out);
int ks_set_default_schedule(ks_params *params, const ks_schedule *schedule);

/* ---------------------------------------------------------------------
 * Autotuning (schedule search by measurement) and its cache.
 * ------------------------------------------------------------------- */

/* The structural candidate schedules the autotuner measures first, in a
 * fixed order (the order the learned cost model predicts): dataflow, OC
 * variant, launch group and job order, each with ntt = bconv = -1 (the
 * parameter set's options).  *n_out = count; up to max are written. */
int ks_tune_candidates(const ks_params *params, uint32_t max, ks_schedule *out, uint32_t *n_out);

/* Autotune a batch in two stages (each timing: one untimed run, then the
 * best of `reps` timed runs with CUDA events on `stream`; the jobs' outputs
 * are overwritten -- every schedule writes the same values):
 *   1. every structural candidate (ks_tune_candidates); ms_out[i] gets
 *      candidate i's time in ms (max entries); of the candidates within
 *      0.3% of the fastest, the one with the largest launch group wins;
 *   2. the fastest structure under each implementation pair (ntt, bconv) in
 *      {(0,1), (1,1), (0,0), (1,0)} (ks_autotune_impl); when max leaves room
 *      for them, ms_out[n_candidates + k] gets pair k's time.
 * The fastest schedule, with explicit ntt and bconv, is written to *best and
 * stored in the params' tuning cache under this batch's signature (job count
 * rounded up to a power of two, mean level rounded to a multiple of 4),
 * where KS_AUTO finds it.  Synchronises `stream`. */
int ks_autotune(ks_params *params, uint32_t n, const ks_job *h_jobs, uint32_t reps, ks_stream_t stream,
                uint32_t max, float *ms_out, ks_schedule *best);

/* Stage 2 alone: time `base` under the four implementation pairs above
 * (ms_out[4] in that order, may be NULL) and write the fastest to *best.
 * Does not touch the tuning cache.  Synchronises `stream`. */
int ks_autotune_impl(ks_params *params, uint32_t n, const ks_job *h_jobs, uint32_t reps, ks_stream_t stream,
                     const ks_schedule *base, float *ms_out, ks_schedule *best);

/* Tuning cache: store / look up the schedule of a signature (n jobs, mean
 * level); lookup returns KS_OK and fills *out, or KS_EINVAL if absent. */
int ks_tune_cache_put(ks_params *params, uint32_t n_jobs, uint32_t mean_level, const ks_schedule *s);
int ks_tune_cache_get(const ks_params *params, uint32_t n_jobs, uint32_t mean_level, ks_schedule *out);
/* Persist / restore the cache as text (one entry per line, with the
 * parameter set and device name it was measured on; entries for another
 * parameter set or device are skipped on load). */
int ks_tune_cache_save(const ks_params *params, const char *path);
int ks_tune_cache_load(ks_params *params, const char *path);

/* ---------------------------------------------------------------------
 * Learned schedule cost model: an FP32 multilayer perceptron trained and
 * evaluated on the device by the library's own kernels (dense layers with
 * ReLU between them, linear output, mean-squared error with an optional
 * 0/1 mask, backpropagation, Adam).  Parameters are laid out per layer as
 * W [out][in] then b [out].  Device pointers d_*: row-major [batch][width].
 * ------------------------------------------------------------------- */
typedef struct ks_mlp ks_mlp;
/* dims[0..n_layers]: input width, hidden widths, output width (each 1..256);
 * weights He-normal from a SplitMix64 stream of `seed`, biases zero. */
int ks_mlp_create(uint32_t n_layers, const uint32_t *dims, uint64_t seed, ks_mlp **out);
void ks_mlp_destroy(ks_mlp *mlp);
size_t ks_mlp_num_params(const ks_mlp *mlp);
int ks_mlp_get_params(const ks_mlp *mlp, float *h_params);
/* Replaces the parameters and resets the optimiser state. */
int ks_mlp_set_params(ks_mlp *mlp, const float *h_params);
int ks_mlp_forward(ks_mlp *mlp, uint32_t batch, const float *d_x, float *d_y, ks_stream_t stream);
/* Loss sum(mask*(y-t)^2)/sum(mask) of the batch and its gradient with
 * respect to every parameter (h_grad, same layout; may be NULL).
 * Synchronises `stream` when h_loss or h_grad is given. */
int ks_mlp_gradients(ks_mlp *mlp, uint32_t batch, const float *d_x, const float *d_t, const float *d_mask,
                     float *h_grad, float *h_loss, ks_stream_t stream);
/* One Adam step (beta 0.9/0.999, eps 1e-8) on the batch's gradient. */
int ks_mlp_train_step(ks_mlp *mlp, uint32_t batch, const float *d_x, const float *d_t, const float *d_mask,
                      float lr, float *h_loss, ks_stream_t stream);

/* Learned schedule choice (the cost model in place of exhaustive search;
 * the paper's dataflows are Sec. IV, the model is this library's).
 * Attach a trained MLP to a parameter set: 10 inputs (ks_cost_features) and
 * one output per structural candidate (ks_tune_candidates order) followed by
 * one per implementation pair (ntt, bconv) in the order {(0,1), (1,1),
 * (0,0), (1,0)}; outputs are normalised log ms per key switch, de-normalised
 * as y * t_scale + t_mean.  The model is not owned and must outlive its use;
 * NULL detaches.  Allocates the model's one-row buffers (so later
 * predictions allocate nothing).  KS_EINVAL when the widths do not match.
 * Once attached, ks_switch_batch (and each chunk of ks_switch_batch_host)
 * with KS_AUTO on a batch whose signature is not in the tuning cache runs
 * the model on `stream` (its forward kernel),
 * reads the prediction back (this synchronises `stream`: make the first
 * such call before any stream capture), stores the predicted schedule in
 * the cache and runs it; ks_autotune remains the exhaustive search whose
 * timings the model is trained on and judged against. */
int ks_params_set_cost_model(ks_params *params, ks_mlp *model, float t_mean, float t_scale);
/* The schedule the attached model predicts fastest for a batch (the fastest
 * structural candidate with the fastest implementation pair).  h_pred
 * (nullable) receives every de-normalised output (log ms per key switch).
 * Synchronises `stream`.  KS_EINVAL when no model is attached. */
int ks_predict_schedule(ks_params *params, uint32_t n, const ks_job *h_jobs, ks_stream_t stream,
                        ks_schedule *out, float *h_pred);
/* The model's 10 inputs for a batch (host): logN, L+1 (the batch's mean
 * level, rounded), dnum (the parameter set's at the top level, else the
 * active digits), K, log2 batch, alpha = ceil((L+1)/dnum), log2 input words,
 * each scaled by fixed constants, then +-1 flags: tensor-core ModUp base
 * conversion available (the parameter set's alpha <= 18), tensor-core ModDown
 * (K <= 18), cluster NTT (logN not 13 or 17). */
int ks_cost_features(const ks_params *params, uint32_t n, const ks_job *h_jobs, float *h_x);

/* A key with pseudo-random residues generated on the device (for timing
 * and tuning; it switches to no particular secret). */
int ks_key_synthetic(const ks_params *params, uint64_t seed, ks_stream_t stream, ks_key **out);

/* One job of a batched key switch whose data live in HOST memory. */
typedef struct {
    const ks_key *key;
    uint32_t level_towers;
    const uint64_t *h_in;  /* host [l+1][N] evaluation form                    */
    uint64_t *h_out0;      /* host [l+1][N]                                    */
    uint64_t *h_out1;      /* host [l+1][N]                                    */
} ks_host_job;

/* End-to-end batched key switch from host memory: copy the inputs to the
 * device, key switch (results as ks_switch gives them), copy both outputs
 * back.  Jobs run in equal chunks of at most 8, each chunk one device batch
 * (ks_switch_batch with the same dataflow; KS_AUTO uses the tuned schedule of
 * the chunk's shape, else the one tuned for the whole call's shape, else the
 * attached cost model's pick).  Copies in, compute and copies out run on three
 * library-owned streams over double-buffered device staging owned by the
 * params object, so chunk c computes while chunk c+1 is copied in and chunk
 * c-1 is copied out, and consecutive calls overlap the same way.  The call's
 * device work does NOT wait for work queued earlier on `stream` (the jobs read
 * only host memory and keys, which are complete when created); `stream` is
 * made to wait for every copy-out.  Host buffers should be page-locked for
 * the copies to overlap.  Calls on one params object are serialised on the
 * host.  Returns after queueing; synchronise `stream` before reading or
 * reusing the host buffers. */
int ks_switch_batch_host(const ks_params *params, uint32_t n, const ks_host_job *h_jobs,
                         ks_dataflow dataflow, ks_stream_t stream);

/* ---------------------------------------------------------------------
 * Tower-sharded key switching: one key switch split over G devices by tower
 * (the output towers are independent, Sec. IV-C).  Rank g owns full Q towers
 * [q_begin, q_end) and special towers [p_begin, p_end) (the ranks' ranges
 * partition [0, n_q) and [0, k_p)), holds the input towers and the key limbs
 * of those towers only, and produces its Q range of the outputs.  Per key
 * switch at level l+1 (= level_towers), with the rank's active Q towers
 * [min(q_begin, l+1), min(q_end, l+1)) = nq_own of them and np_own =
 * p_end - p_begin special towers, nown = nq_own + np_own:
 *   ks_shard_prep      d_own [nq_own][N] -> y_own [nq_own][N] (ModUp P1);
 *   (caller)           all-gather y: y_all [l+1][N], towers in order;
 *   ks_shard_keyprod   y_all, d_own -> cp_own [2][nown][N]: c' of the
 *                      rank's towers (ModUp P2-P5); rows nq_own.. of each
 *                      polynomial then hold w_own, the special towers after
 *                      ModDown P1 (coefficient form);
 *   (caller)           all-gather w: w_all [2][K][N], towers in order;
 *   ks_shard_moddown   w_all, cp_own -> out0_own, out1_own [nq_own][N]
 *                      (ModDown P2-P4).
 * The gathered outputs equal ks_switch's bit for bit.  All data are device
 * memory owned by the caller; scratch holds ks_shard_scratch_words() words
 * (the same buffer for keyprod and moddown of one key switch).  Calls queue
 * work on `stream` and return KS_EINVAL for bad ranges, levels or keys.  A
 * rank with no active Q towers at a level skips prep and moddown. */
typedef struct {
    uint32_t q_begin, q_end; /* full Q towers of the rank */
    uint32_t p_begin, p_end; /* special towers of the rank */
} ks_shard;
/* A key holding only the shard's towers ([ndig][2][own towers][N]), copied
 * from a full key on `stream` (synchronised before returning).  Free it
 * with ks_key_destroy; it serves the ks_shard_* calls only. */
int ks_key_shard(const ks_key *full_key, const ks_shard *shard, ks_stream_t stream, ks_key **out);
size_t ks_shard_scratch_words(const ks_params *params, const ks_shard *shard, uint32_t level_towers);
int ks_shard_prep(const ks_params *params, const ks_shard *shard, uint32_t level_towers, const uint64_t *d_own,
                  uint64_t *y_own, ks_stream_t stream);
int ks_shard_keyprod(const ks_params *params, const ks_key *shard_key, uint32_t level_towers,
                     const uint64_t *y_all, const uint64_t *d_own, uint64_t *cp_own, uint64_t *scratch,
                     ks_stream_t stream);
int ks_shard_moddown(const ks_params *params, const ks_key *shard_key, uint32_t level_towers,
                     const uint64_t *w_all, const uint64_t *cp_own, uint64_t *out0_own, uint64_t *out1_own,
                     uint64_t *scratch, ks_stream_t stream);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of key-switch requests.
 *
 * A server owns one scheduler thread, n_streams device lanes and a scratch
 * pool of hbm_budget_bytes allocated at creation.  Requests are admitted in
 * arrival order while fewer than max_inflight_jobs are on the device and
 * their scratch fits in the pool (HBM-budget admission); admitted requests
 * that share a parameter set are launched together (up to max_batch) as one
 * Output-Centric batch on the next lane, so batches overlap on the device
 * and requests that arrive meanwhile join the next batch.  Results equal
 * ks_switch's.  Params, keys and data buffers stay owned by the caller and
 * must outlive their requests.
 * ------------------------------------------------------------------- */
typedef struct ks_server ks_server;
typedef struct {
    uint32_t max_inflight_jobs;  /* slots: requests on the device at once (>= 1)     */
    uint32_t max_batch;          /* requests per batched launch, 1..64               */
    uint32_t n_streams;          /* device lanes, 1..16                              */
    uint32_t reserved;           /* set to 0                                         */
    uint64_t hbm_budget_bytes;   /* scratch pool, >= 1 MiB                           */
} ks_server_config;
typedef struct {
    const ks_params *params;
    const ks_key *key;
    uint32_t level_towers;
    const uint64_t *d_in;  /* device [l+1][N] */
    uint64_t *d_out0;      /* device [l+1][N] */
    uint64_t *d_out1;      /* device [l+1][N] */
} ks_request;

/* Create on the current device; starts the scheduler thread. */
int ks_server_create(const ks_server_config *cfg, ks_server **out);
/* Finish every queued and running request, then stop and free. */
void ks_server_destroy(ks_server *server);
/* Queue a request (thread-safe, non-blocking); *ticket identifies it.
 * Buffers as for ks_switch (16-byte aligned, not overlapping); requests
 * that break this, or whose scratch exceeds the whole budget, fail with
 * KS_EINVAL. */
int ks_server_submit(ks_server *server, const ks_request *req, uint64_t *ticket);
/* Wait for a request: its status, or KS_ETIMEOUT if still unfinished after
 * timeout_ms (the request keeps running). */
int ks_server_wait(ks_server *server, uint64_t ticket, uint32_t timeout_ms);
/* Arrival, admission and completion times (seconds since the server was
 * created) of a finished request. */
int ks_server_times(ks_server *server, uint64_t ticket, double *t_arrive, double *t_admit, double *t_done);
/* Requests finished, batches launched, largest batch so far. */
int ks_server_stats(ks_server *server, uint64_t *n_done, uint64_t *n_batches, uint64_t *max_batch);
/* Replay a trace: submit request i at arrival_s[i] seconds after the call
 * (precise host timing), wait for all, write each request's latency
 * (completion minus arrival, seconds) to latency_s. */
int ks_server_run_trace(ks_server *server, uint32_t n, const ks_request *reqs, const double *arrival_s,
                        double *latency_s, uint32_t timeout_ms);

/* ---------------------------------------------------------------------
 * Measurement hooks (used by the benchmark; cheap when disabled).
 * ------------------------------------------------------------------- */

/* Arithmetic ceilings of the current GPU for the two inner loops of key
 * switching, measured with register-only loops of the same device code:
 * forward NTT butterflies per second and base-conversion multiply-
 * accumulates per second.  iters: loop trips per thread (e.g. 4096). */
int ks_probe_alu(int iters, double *bfly_per_s, double *mac_per_s);

/* The same ceiling for the inverse (Harvey) NTT butterfly, inverse
 * butterflies per second (the ceiling of the inverse NTT passes). */
int ks_probe_inv_bfly(int iters, double *inv_bfly_per_s);

/* Issue rates of single integer instructions on this GPU, in lanes per SM
 * per clock (all SMs, 8 independent chains per thread, the device's clock
 * attribute): out[0] mad.lo.u32, [1] mad.wide.u32 (64-bit accumulate),
 * [2] mul.lo.u64, [3] mul.hi.u64, [4] add.u32.  n >= 5.  The multiply-pipe
 * cost of the kernels' modular products follows from these (a Shoup product
 * is two mul.lo.u64 and one mul.hi.u64). */
int ks_probe_int_pipes(double *lanes_per_clk_sm, int n);

/* Number of kernels this library has launched since it was loaded. */
uint64_t ks_kernel_launches(void);

/* When on, every kernel launch is bracketed by CUDA events on its stream. */
void ks_profile_enable(int on);

/* Synchronise the recorded events and return, per kernel name, the number of
 * launches and their summed device time (ms) since the last collect; then
 * clear.  names: max x 48 chars.  *n_out receives the number of names. */
int ks_profile_collect(uint32_t max, char *names, double *total_ms, uint32_t *counts, uint32_t *n_out);

#ifdef __cplusplus
}
#endif
#endif /* KS_H */
