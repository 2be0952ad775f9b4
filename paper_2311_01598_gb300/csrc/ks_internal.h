// ks_internal.h -- internal types of the key-switching library (host + device).
//
// Layout of everything the library keeps on the device (one parameter set):
//   modc[t]          per-tower constants, t over the full basis q_0..q_L, p_0..p_{K-1}
//   tw[t][N]         forward twiddles (w, floor(w*2^64/q)) in bit-reversed order:
//                    tw[t][i] = psi^brv(i) for the Cooley-Tukey NTT
//   itw[t][N]        inverse twiddles psi^-brv(i) for the Gentleman-Sande iNTT
//   up_pre[...]      ModUp P1 scale N^-1 * (Q_j/q_i)^-1 mod q_i per (digit, active
//                    towers, source tower)
//   up_mat[...]      ModUp P2 matrix (Q_j/q_i) mod r per (digit, active towers,
//                    source tower, target tower), split in two 28-bit halves
//   dn_mat[k][i]     ModDown P2 matrix (P/p_k) * P^-1 mod q_i (P^-1 of P4 folded in)
//   key_sc[t]        per-tower factor folded into the stored key: P^-1 on Q towers
//                    (ModDown P4), N^-1 * (P/p_k)^-1 on P towers (ModDown P1 + P2
//                    prescale), times 2^64 for the Montgomery product of P4
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ks.h"

namespace ks {

typedef uint64_t u64;
typedef uint32_t u32;

constexpr int kMaxQ = 64;
constexpr int kMaxP = 32;
constexpr int kMaxT = kMaxQ + kMaxP;
constexpr int kMinLogN = 10;
constexpr int kMaxLogN = 17;
constexpr int kMaxPrimeBits = 56;  // 28-bit split products in BConv; 4q < 2^58 in the NTT
constexpr int kSplit = 28;

// Per-tower constants.
struct ModC {
    u64 q;       // modulus
    u64 q2;      // 2q
    u64 mont;    // -q^-1 mod 2^64 (Montgomery reduction)
    u64 one_sh;  // floor(2^64 / q): Shoup companion of 1
    u64 r28, r28_sh;  // 2^28 mod q and its Shoup companion
    u64 r56, r56_sh;  // 2^56 mod q and its Shoup companion
    u64 ninv, ninv_sh;  // N^-1 mod q and its Shoup companion
    u64 r2;             // 2^128 mod q (into Montgomery form)
    u64 pad;
};

// Device tables of one parameter set, passed to kernels by value.
// A key as the kernels read it: a full key, or a compressed one (b stored,
// a regenerated from a_seed; see key_a_word in ks_device.cuh).
struct KeyView {
    const u64 *evk;
    u64 a_seed;
    int comp;
};

struct Tables {
    const ModC *modc;
    const ulonglong2 *tw;
    const ulonglong2 *itw;
    const ulonglong2 *up_pre;
    const u64 *up_mat;
    const u64 *dn_mat;
    const ulonglong2 *key_sc;   // Montgomery-form fold factors (see header)
    const ulonglong2 *plain_sc; // the same factors without 2^64
    const int *up_mat_lvl;    // ModUp matrix offset of digit j at level nact: [(nact-1)*ndig + j]
    // tensor-core base conversion: per-target B slabs (null when unsupported
    // or switched off) and the ModUp slab base of digit j at level nact
    const uint4 *up_tc;
    const int *up_tc_lvl;
    const uint4 *dn_tc;
    int ntt_cluster;  // host side: NTTs as one cluster launch where supported
    int row_stage;    // host side: forward row passes staged by bulk copies (k_fwd_row_st)
    int spq;          // every modulus is q1*2^32 + 1: two-pass NTTs use shoup_est_sp
    int tc_below54;   // every modulus is below 2^54: 9-bit constant slices (tensor-core BConv)
    int logN;
    int nq, kp, alpha, ndig;
};

// Offsets of the ModUp tables for digit j with `a` active towers.
struct UpOffsets {
    std::vector<int> pre;  // [j * (alpha + 1) + a]
    std::vector<int> mat;
};

struct Workspace;
struct HostStage;

}  // namespace ks

struct ks_params {
    int logN = 0;
    uint32_t N = 0;
    int nq = 0, kp = 0, dnum = 0, alpha = 0, ndig = 0;
    int device = 0;
    std::vector<uint64_t> q, p, psi;  // psi over the full basis
    ks::UpOffsets up_off;
    // device allocations
    ks::ModC *d_modc = nullptr;
    ulonglong2 *d_tw = nullptr, *d_itw = nullptr;
    ulonglong2 *d_up_pre = nullptr;
    ulonglong2 *d_up_pre_lvl = nullptr;  // [nq levels][nq]: ModUp P1 factor per level
    int *d_up_mat_lvl = nullptr;         // [nq levels][ndig]: ModUp matrix offsets per level
    uint4 *d_up_tc = nullptr, *d_dn_tc = nullptr;  // tensor-core BConv slabs
    int *d_up_tc_lvl = nullptr;
    int bconv_tensor = 1;                // use the tensor-core BConv where supported
    int ntt_cluster = 0;                 // NTTs as one cluster launch where supported
    int row_stage = 0;                   // forward row passes staged by bulk copies
    int batch_lanes = 2;                 // internal streams a large Output-Centric batch is split over
    cudaStream_t lane_st[4] = {};        // created on first use
    cudaEvent_t lane_ev[5] = {};
    std::mutex lane_mu;                  // one batch at a time enqueues on the lanes
    uint64_t *d_up_mat = nullptr;
    uint64_t *d_dn_mat = nullptr;
    ulonglong2 *d_key_sc = nullptr, *d_plain_sc = nullptr;
    ks::Tables tables{};
    // per-stream scratch
    std::mutex mu;
    std::map<void *, ks::Workspace *> ws;
    // default schedule (KS_OC / KS_AUTO without a tuned entry)
    ks_schedule sched{KS_OC, 1, 64, 0, -1, -1};
    // tuning cache: (job-count bucket, mean-level bucket) -> schedule;
    // every access holds tune_mu (KS_AUTO calls on several threads share it)
    std::map<std::pair<uint32_t, uint32_t>, ks_schedule> tune;
    mutable std::mutex tune_mu;
    // learned cost model consulted by KS_AUTO on a tuning-cache miss (not
    // owned), its target normalisation and its one-row input/output buffers
    ks_mlp *cost_model = nullptr;
    float cm_mean = 0.f, cm_scale = 1.f;
    float *d_cm_x = nullptr, *d_cm_y = nullptr;
    // double-buffered device staging of ks_switch_batch_host
    std::mutex host_mu;
    ks::HostStage *stage = nullptr;
};

struct ks_key {
    const ks_params *params = nullptr;
    // full key: [ndig][2][nq+kp][N]; compressed: [ndig][nq+kp][N] (b only);
    // Montgomery form with key_sc folded in
    uint64_t *d_evk = nullptr;
    size_t bytes = 0;
    int compressed = 0;
    uint64_t a_seed = 0;  // compressed: seed of the regenerated a half
    // tower shard (ks_key_shard): the limbs of full Q towers [q0, q1) and
    // special towers [p0, p1) only, [ndig][2][(q1-q0)+(p1-p0)][N]; used by
    // the ks_shard_* calls only
    int shard = 0;
    uint32_t q0 = 0, q1 = 0, p0 = 0, p1 = 0;
};

namespace ks {
inline KeyView key_view(const ks_key *K) { return KeyView{K->d_evk, K->a_seed, K->compressed}; }
}  // namespace ks

namespace ks {

// Every kernel launch of the library runs inside a LaunchScope: the scope
// counts the launch and, while profiling is on, brackets it with CUDA events
// recorded on the launch stream (ks_profile_collect sums them per name).
class LaunchScope {
  public:
    LaunchScope(cudaStream_t st, const char *name);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

  private:
    cudaStream_t st_;
    long rec_ = -1;
};
#define KS_LAUNCH(st, name, ...)              \
    do {                                      \
        ::ks::LaunchScope ks_scope_(st, name); \
        __VA_ARGS__;                          \
    } while (0)

// Per-device one-time setup (kernel attributes are per device context):
// runs setup() once for the current device; callers on other threads wait
// for it to finish.  done is the caller's static bit set of devices.
inline std::mutex &setup_mutex()
{
    static std::mutex m;
    return m;
}
template <class F>
inline void once_per_device(std::atomic<uint64_t> &done, F &&setup)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    std::lock_guard<std::mutex> g(setup_mutex());
    if (done.load(std::memory_order_relaxed) & bit) return;
    setup();
    done.fetch_or(bit, std::memory_order_release);
}

// Thread-local error message (ks_last_error).
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

// Host number theory (ks_host.cpp).
bool is_prime_u64(u64 n);
int gen_primes(int logN, int bits, int count, std::vector<u64> &out);
int gen_special_primes(int bits, int count, std::vector<u64> &out);
u64 find_psi(u64 q, int logN);
u64 mulmod_h(u64 a, u64 b, u64 m);
u64 powmod_h(u64 b, u64 e, u64 m);
u64 invmod_h(u64 a, u64 m);
u64 shoup_h(u64 w, u64 q);  // floor(w * 2^64 / q)

// Batch execution under a schedule (ks_api.cu), used by the autotuner.
int run_batch(ks_params *P, uint32_t n, const ks_job *jobs, const ks_schedule &sc, cudaStream_t st);
int check_batch(const ks_params *P, uint32_t n, const ks_job *jobs);
int check_schedule(const ks_schedule *sc);
// Tuning-cache signature of a batch.
std::pair<uint32_t, uint32_t> tune_signature(uint32_t n, uint32_t mean_level);
// The schedule the parameter set's cost model predicts fastest for a batch
// (ks_tune.cu): runs the model's forward kernel on st and reads the
// predictions back (synchronises st).  h_pred (nullable) receives the raw
// outputs (predicted log ms per key switch).
int predict_schedule(ks_params *P, uint32_t n, const ks_job *jobs, cudaStream_t st, ks_schedule *out, float *h_pred);
// MLP internals used by the schedule predictor (ks_mlp.cu).
int mlp_io_dims(const ks_mlp *M, int *in, int *out);
int mlp_reserve(ks_mlp *M, int batch);
// Fill a key buffer with pseudo-random canonical residues (ks_kernels.cu).
int launch_key_random(const Tables &T, u64 *evk, uint64_t seed, cudaStream_t st);

// Build every host table and upload it (ks_host.cpp).
int build_tables(ks_params *P);
void free_tables(ks_params *P);

}  // namespace ks
