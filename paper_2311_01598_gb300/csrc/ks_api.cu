// ks_api.cu -- C ABI entry points, parameter/key objects, per-stream scratch
// and the Max-Parallel / Digit-Centric executors (CiFlow Sec. IV-A, IV-B).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ks_internal.h"
#include "ks_launch.h"

namespace ks {

static thread_local std::string tl_err;

void set_error(const std::string &msg) { tl_err = msg; }
int fail(int code, const std::string &msg)
{
    tl_err = msg;
    return code;
}

// ------------------------------------------------------------------ launches
static std::atomic<uint64_t> g_launches{0};
static std::atomic<bool> g_prof{false};
struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
};
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_ev_pool;

static cudaEvent_t pool_event()
{
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

LaunchScope::LaunchScope(cudaStream_t st, const char *name) : st_(st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    ProfRec r{name, pool_event(), pool_event()};
    cudaEventRecord(r.e0, st);
    rec_ = (long)g_recs.size();
    g_recs.push_back(r);
}

LaunchScope::~LaunchScope()
{
    if (rec_ < 0) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    cudaEventRecord(g_recs[rec_].e1, st_);
}

static int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return KS_OK;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? KS_ENOMEM : KS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Scratch of one stream: sized for the top level of the parameter set.
struct Workspace {
    u64 *y = nullptr;    // [nq][N]          ModUp P1 output (coefficient form)
    u64 *D = nullptr;    // [ndig][nq+kp][N] ModUp P2/P3 output (MP); digit 0 slot (DC)
    u64 *cp = nullptr;   // [2][nq+kp][N]    ModUp P5 output c'
    u64 *v = nullptr;    // [2][nq][N]       ModDown P2/P3 output
    u64 *oc = nullptr;   // Output-Centric scratch of one job at the top level
    u64 *batch = nullptr;  // Output-Centric scratch of a batch
    size_t batch_words = 0;
    u64 *rot = nullptr;    // c' and v of each hoisted rotation
    size_t rot_words = 0;
};

static int ws_alloc(u64 **p, size_t words)
{
    return cuda_check(cudaMalloc((void **)p, words * sizeof(u64)), "workspace allocation");
}

static int get_ws(ks_params *P, cudaStream_t st, bool need_D, Workspace **out)
{
    std::lock_guard<std::mutex> g(P->mu);
    Workspace *&w = P->ws[(void *)st];
    if (!w) w = new Workspace();
    const size_t N = P->N;
    const size_t nt = (size_t)P->nq + P->kp;
    int rc = KS_OK;
    if (!w->y && (rc = ws_alloc(&w->y, (size_t)P->nq * N)) != KS_OK) return rc;
    if (!w->cp && (rc = ws_alloc(&w->cp, 2 * nt * N)) != KS_OK) return rc;
    if (!w->v && (rc = ws_alloc(&w->v, 2 * (size_t)P->nq * N)) != KS_OK) return rc;
    if (need_D && !w->D && (rc = ws_alloc(&w->D, (size_t)P->ndig * nt * N)) != KS_OK) return rc;
    if (!w->oc && (rc = ws_alloc(&w->oc, oc_scratch_words(P->tables, P->nq))) != KS_OK) return rc;
    *out = w;
    return KS_OK;
}

// Double-buffered device staging of the host-memory batch path: jobs run in
// chunks of at most kHostChunk; chunk c computes while chunk c+1 is copied in
// and chunk c-1 is copied out.
constexpr int kHostChunk = 8;
struct HostStage {
    u64 *din[2] = {nullptr, nullptr}, *dout0[2] = {nullptr, nullptr}, *dout1[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_out = nullptr, s_comp = nullptr;
    cudaEvent_t h2d[2] = {}, comp[2] = {}, d2h[2] = {};
    int next = 0;  // slot of the next chunk (alternation continues across calls)
};

static int get_stage(ks_params *P, HostStage **out)
{
    if (!P->stage) {
        HostStage *h = new HostStage();
        P->stage = h;  // partially built stages are released by free_ws
        const size_t words = (size_t)kHostChunk * P->nq * P->N;
        int rc = KS_OK;
        for (int i = 0; i < 2 && rc == KS_OK; ++i) {
            if ((rc = ws_alloc(&h->din[i], words)) != KS_OK) break;
            if ((rc = ws_alloc(&h->dout0[i], words)) != KS_OK) break;
            if ((rc = ws_alloc(&h->dout1[i], words)) != KS_OK) break;
            rc = cuda_check(cudaEventCreateWithFlags(&h->h2d[i], cudaEventDisableTiming), "event");
            if (rc == KS_OK) rc = cuda_check(cudaEventCreateWithFlags(&h->comp[i], cudaEventDisableTiming), "event");
            if (rc == KS_OK) rc = cuda_check(cudaEventCreateWithFlags(&h->d2h[i], cudaEventDisableTiming), "event");
        }

        if (rc == KS_OK) rc = cuda_check(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking), "stream");
        if (rc == KS_OK) rc = cuda_check(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking), "stream");
        if (rc == KS_OK) rc = cuda_check(cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking), "stream");
        if (rc != KS_OK) return rc;
    }
    *out = P->stage;
    return KS_OK;
}

static void free_ws(ks_params *P)
{
    for (int l = 0; l < 4; ++l)
        if (P->lane_st[l]) {
            cudaStreamDestroy(P->lane_st[l]);
            P->lane_st[l] = nullptr;
        }
    for (int e = 0; e < 5; ++e)
        if (P->lane_ev[e]) {
            cudaEventDestroy(P->lane_ev[e]);
            P->lane_ev[e] = nullptr;
        }
    if (P->stage) {
        HostStage *h = P->stage;
        for (int i = 0; i < 2; ++i) {
            u64 *bufs[] = {h->din[i], h->dout0[i], h->dout1[i]};
            for (u64 *b : bufs)
                if (b) cudaFree(b);
            cudaEvent_t evs[] = {h->h2d[i], h->comp[i], h->d2h[i]};
            for (cudaEvent_t e : evs)
                if (e) cudaEventDestroy(e);
        }
        if (h->s_in) cudaStreamDestroy(h->s_in);
        if (h->s_out) cudaStreamDestroy(h->s_out);
        if (h->s_comp) cudaStreamDestroy(h->s_comp);
        delete h;
        P->stage = nullptr;
    }
    for (auto &kv : P->ws) {
        Workspace *w = kv.second;
        u64 *bufs[] = {w->y, w->D, w->cp, w->v, w->oc, w->batch, w->rot};
        for (u64 *b : bufs)
            if (b) cudaFree(b);
        delete w;
    }
    P->ws.clear();
}

static int active_digits(const ks_params *P, int nact) { return (nact + P->alpha - 1) / P->alpha; }

// ModUp P1 scale of tower i at level nact: N^-1 * (Q_j/q_i)^-1 mod q_i,
// one contiguous row of nact pairs per level.
static const ulonglong2 *pre_level(const ks_params *P, int nact) { return P->d_up_pre_lvl + (size_t)(nact - 1) * P->nq; }

// ------------------------------------------------------------------ ModDown
static int run_moddown(const ks_params *P, const Tables &T, Workspace *w, int nact, int npoly, u64 *out0, u64 *out1,
                       cudaStream_t st)
{
    const size_t N = P->N;
    const int nt = nact + P->kp;
    int rc;
    // P1: iNTT of the special towers of each polynomial (N^-1 (P/p_k)^-1 is
    // folded into the key), canonical.
    LimbMap mP{w->cp, w->cp, nullptr, P->kp, nt, nact, nact, nact, -1};
    if ((rc = launch_ntt_inv(T, one_map(mP, npoly * P->kp), false, st)) != KS_OK) return rc;
    // P2: fast base conversion P -> q_0..q_l (P^-1 folded into the matrix).
    BDnJobs bd;
    bd.n = 0;
    add_bdn(bd, BDnJob{w->cp, (size_t)nt * N, w->v, (size_t)nact * N, nact, npoly});
    if ((rc = launch_bconv_down(T, bd, st)) != KS_OK) return rc;
    // P3: NTT of the converted towers.
    LimbMap mV{w->v, w->v, nullptr, nact, nact, 0, 0, nact, -1};
    if ((rc = launch_ntt_fwd(T, one_map(mV, npoly * nact), false, st)) != KS_OK) return rc;
    // P4: subtract.
    u64 *outs[2] = {out0, out1};
    return launch_down_final(T, nact, npoly, w->cp, (size_t)nt * N, w->v, (size_t)nact * N, outs, st);
}

// ------------------------------------------------------------------ MP
// Max-Parallel: each stage over all towers, intermediates in device memory.
static int run_mp(const ks_params *P, const Tables &T, const ks_key *K, int nact, const u64 *d, u64 *out0, u64 *out1,
                  Workspace *w, cudaStream_t st)
{
    const size_t N = P->N;
    const int nt = nact + P->kp;
    const int nd = active_digits(P, nact);
    int rc;
    // ModUp P1: iNTT and the (Q_j/q_i)^-1 prescale of every input tower.
    LimbMap m1{d, w->y, pre_level(P, nact), nact, 0, 0, 0, nact, -1};
    if ((rc = launch_ntt_inv(T, one_map(m1, nact), false, st)) != KS_OK) return rc;
    // P2: every digit to every other tower of D_l.
    BUpJobs bu;
    bu.n = 0;
    add_bup(bu, T, BUpJob{w->y, w->D, (size_t)nt * N, nact, 0, nt, 0, -1});
    if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;
    // P3: NTT of the converted towers (digit towers are bypassed).
    LimbMap mD{w->D, w->D, nullptr, nt, nt, 0, 0, nact, 0};
    if ((rc = launch_ntt_fwd(T, one_map(mD, nd * nt), false, st)) != KS_OK) return rc;
    // P4 + P5: key product summed over digits.
    if ((rc = launch_apply_key(T, nact, 0, nd, d, w->D, (size_t)nt * N, key_view(K), w->cp, false, st)) != KS_OK) return rc;
    return run_moddown(P, T, w, nact, 2, out0, out1, st);
}

// ------------------------------------------------------------------ hoisted rotations
// One ModUp of d (as MP) shared by R rotations: rotation r's key product reads
// the raised digits through X -> X^g_r, then the ModDowns of all rotations
// run as batched launches (groups of kMaxBatch rotations).
static int run_hoisted(ks_params *P, uint32_t R, const ks_key *const *keys, const uint64_t *gal, int nact,
                       const u64 *d, u64 *const *out0, u64 *const *out1, cudaStream_t st)
{
    const Tables &T = P->tables;
    const size_t N = P->N;
    const int nt = nact + P->kp;
    const int nd = active_digits(P, nact);
    const int K = P->kp;
    Workspace *w = nullptr;
    int rc = get_ws(P, st, true, &w);
    if (rc) return rc;
    const uint32_t G = std::min<uint32_t>(R, kMaxBatch);
    const size_t cp_words = 2 * (size_t)nt * N, v_words = 2 * (size_t)nact * N;
    {
        std::lock_guard<std::mutex> g(P->mu);
        const size_t words = (size_t)G * (cp_words + v_words);
        if (w->rot_words < words) {
            if (w->rot) {
                cudaStreamSynchronize(st);  // queued work may still use the old buffer
                cudaFree(w->rot);
                w->rot = nullptr;
                w->rot_words = 0;
            }
            if ((rc = ws_alloc(&w->rot, words)) != KS_OK) return rc;
            w->rot_words = words;
        }
    }
    // ModUp P1-P3 once (digit towers are read from d by the key product).
    LimbMap m1{d, w->y, pre_level(P, nact), nact, 0, 0, 0, nact, -1};
    if ((rc = launch_ntt_inv(T, one_map(m1, nact), false, st)) != KS_OK) return rc;
    BUpJobs bu;
    bu.n = 0;
    add_bup(bu, T, BUpJob{w->y, w->D, (size_t)nt * N, nact, 0, nt, 0, -1});
    if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;
    LimbMap mD{w->D, w->D, nullptr, nt, nt, 0, 0, nact, 0};
    if ((rc = launch_ntt_fwd(T, one_map(mD, nd * nt), false, st)) != KS_OK) return rc;
    for (uint32_t r0 = 0; r0 < R; r0 += G) {
        const uint32_t g = std::min(G, R - r0);
        u64 *cpr = w->rot, *vr = w->rot + (size_t)G * cp_words;
        for (uint32_t i = 0; i < g; ++i)
            if ((rc = launch_apply_key(T, nact, 0, nd, d, w->D, (size_t)nt * N, key_view(keys[r0 + i]),
                                       cpr + i * cp_words, false, st, gal[r0 + i])) != KS_OK)
                return rc;
        // ModDown of the g rotations: P1 iNTT, P2 BConv, P3 NTT, P4.
        LimbMaps mP, mV;
        mP.n = mV.n = 0;
        BDnJobs bd;
        bd.n = 0;
        for (uint32_t i = 0; i < g; ++i) {
            u64 *c = cpr + i * cp_words, *v = vr + i * v_words;
            add_map(mP, LimbMap{c, c, nullptr, K, nt, nact, nact, nact, -1}, 2 * K);
            add_bdn(bd, BDnJob{c, (size_t)nt * N, v, (size_t)nact * N, nact, 2});
            add_map(mV, LimbMap{v, v, nullptr, nact, nact, 0, 0, nact, -1}, 2 * nact);
        }
        if ((rc = launch_ntt_inv(T, mP, false, st)) != KS_OK) return rc;
        if ((rc = launch_bconv_down(T, bd, st)) != KS_OK) return rc;
        if ((rc = launch_ntt_fwd(T, mV, false, st)) != KS_OK) return rc;
        for (uint32_t i = 0; i < g; ++i) {
            u64 *outs[2] = {out0[r0 + i], out1[r0 + i]};
            if ((rc = launch_down_final(T, nact, 2, cpr + i * cp_words, (size_t)nt * N, vr + i * v_words,
                                        (size_t)nact * N, outs, st)) != KS_OK)
                return rc;
        }
    }
    return KS_OK;
}

// ------------------------------------------------------------------ DC
// Digit-Centric: ModUp P1..P5 for one digit at a time, partial sums of c'
// accumulated in device memory, then ModDown.
static int run_dc(const ks_params *P, const Tables &T, const ks_key *K, int nact, const u64 *d, u64 *out0, u64 *out1,
                  Workspace *w, cudaStream_t st)
{
    const int nt = nact + P->kp;
    const int nd = active_digits(P, nact);
    int rc;
    for (int j = 0; j < nd; ++j) {
        const int lo = j * P->alpha;
        const int a = std::min(P->alpha, nact - lo);
        LimbMap m1{d, w->y, pre_level(P, nact) + lo, a, 0, lo, lo, nact, -1};
        if ((rc = launch_ntt_inv(T, one_map(m1, a), false, st)) != KS_OK) return rc;
        BUpJobs bu;
        bu.n = 0;
        add_bup(bu, T, BUpJob{w->y, w->D, 0, nact, 0, nt, 0, j});
        if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;
        LimbMap mD{w->D, w->D, nullptr, nt, nt, 0, 0, nact, j};
        if ((rc = launch_ntt_fwd(T, one_map(mD, nt), false, st)) != KS_OK) return rc;
        if ((rc = launch_apply_key(T, nact, j, j + 1, d, w->D, 0, key_view(K), w->cp, j > 0, st)) != KS_OK) return rc;
    }
    return run_moddown(P, T, w, nact, 2, out0, out1, st);
}

// ------------------------------------------------------------------ OC
OcJob oc_job(const ks_params *P, const ks_key *K, int nact, const u64 *d, u64 *out0, u64 *out1, u64 *scratch)
{
    const size_t N = P->N;
    const int nd = active_digits(P, nact);
    OcJob J;
    J.d = d;
    J.out0 = out0;
    J.out1 = out1;
    J.key = key_view(K);
    J.y = scratch;
    J.tmp = J.y + (size_t)nact * N;
    J.cp = J.tmp + ((size_t)nd * (nact + P->kp) + 2 * (size_t)nact) * N;
    J.pre = pre_level(P, nact);
    J.nact = nact;
    J.nd = nd;
    return J;
}

static int run_oc(const ks_params *P, const Tables &T, int oc_variant, const ks_key *K, int nact, const u64 *d, u64 *out0,
                  u64 *out1, Workspace *w, cudaStream_t st)
{
    OcJob J = oc_job(P, K, nact, d, out0, out1, w->oc);
    return launch_oc(T, 1, &J, oc_variant, st);
}

// Tables of one call: the parameter set's tables with the schedule's
// implementation choices applied (-1 keeps the parameter set's option).
Tables call_tables(const ks_params *P, const ks_schedule &sc)
{
    Tables T = P->tables;
    if (sc.bconv == 0) {
        T.up_tc = nullptr;
        T.dn_tc = nullptr;
    } else if (sc.bconv == 1) {
        T.up_tc = P->d_up_tc;  // null where the parameter set has no tensor-core form
        T.dn_tc = P->d_dn_tc;
    }
    if (sc.ntt >= 0) T.ntt_cluster = sc.ntt;
    return T;
}

int check_job(const ks_params *P, const ks_key *K, uint32_t nact, const uint64_t *d, const uint64_t *o0,
              const uint64_t *o1)
{
    if (!K || K->params != P) return fail(KS_EINVAL, "key is NULL or belongs to another params object");
    if (K->shard) return fail(KS_EINVAL, "key is a tower shard: it serves the ks_shard_* calls only");
    if (nact < 1 || nact > (uint32_t)P->nq) return fail(KS_EINVAL, "level_towers must be in 1..n_q");
    if (!d || !o0 || !o1) return fail(KS_EINVAL, "NULL data pointer");
    // the combine kernels move two words at a time
    if (((uintptr_t)d | (uintptr_t)o0 | (uintptr_t)o1) & 15)
        return fail(KS_EINVAL, "d_in, d_out0 and d_out1 must be 16-byte aligned");
    const size_t bytes = (size_t)nact * P->N * sizeof(u64);
    auto overlap = [bytes](const void *a, const void *b) {
        const char *x = (const char *)a, *y = (const char *)b;
        return x < y + bytes && y < x + bytes;
    };
    if (overlap(d, o0) || overlap(d, o1) || overlap(o0, o1)) return fail(KS_EINVAL, "d_in, d_out0, d_out1 overlap");
    return KS_OK;
}

static int check_params(const ks_params *P)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    return KS_OK;
}

static int set_device(const ks_params *P)
{
    return cuda_check(cudaSetDevice(P->device), "cudaSetDevice");
}

}  // namespace ks

using namespace ks;

extern "C" {

const char *ks_last_error(void) { return tl_err.c_str(); }

int ks_params_create(uint32_t logN, uint32_t n_q, uint32_t k_p, uint32_t dnum, const uint64_t *h_q,
                     const uint64_t *h_p, uint32_t prime_bits, ks_params **out)
{
    if (!out) return fail(KS_EINVAL, "out is NULL");
    *out = nullptr;
    if (logN < (uint32_t)kMinLogN || logN > (uint32_t)kMaxLogN) return fail(KS_EUNSUPPORTED, "logN must be in 10..17");
    if (n_q < 1 || n_q > (uint32_t)kMaxQ) return fail(KS_EINVAL, "n_q must be in 1..64");
    if (k_p < 1 || k_p > (uint32_t)kMaxP) return fail(KS_EINVAL, "k_p must be in 1..32");
    if (dnum < 1 || dnum > n_q) return fail(KS_EINVAL, "dnum must be in 1..n_q");
    if ((h_q == nullptr) != (h_p == nullptr)) return fail(KS_EINVAL, "give both prime lists or neither");
    const uint64_t N = 1ull << logN;
    std::vector<u64> q(n_q), p(k_p);
    if (h_q) {
        std::vector<u64> all;
        for (uint32_t i = 0; i < n_q; ++i) all.push_back(h_q[i]);
        for (uint32_t i = 0; i < k_p; ++i) all.push_back(h_p[i]);
        for (size_t i = 0; i < all.size(); ++i) {
            if (all[i] >= (1ull << kMaxPrimeBits) || all[i] % (2 * N) != 1 || !is_prime_u64(all[i]))
                return fail(KS_EINVAL, "explicit primes must be primes = 1 mod 2N below 2^56");
            for (size_t k = 0; k < i; ++k)
                if (all[k] == all[i]) return fail(KS_EINVAL, "explicit primes must be distinct");
        }
        for (uint32_t i = 0; i < n_q; ++i) q[i] = h_q[i];
        for (uint32_t i = 0; i < k_p; ++i) p[i] = h_p[i];
    } else {
        if (prime_bits < 30 || prime_bits > (uint32_t)kMaxPrimeBits)
            return fail(KS_EUNSUPPORTED, "prime_bits must be in 30..56");
        std::vector<u64> all;
        if (gen_primes((int)logN, (int)prime_bits, (int)(n_q + k_p), all) != 0)
            return fail(KS_EINVAL, "not enough primes = 1 mod 2N below 2^prime_bits");
        for (uint32_t k = 0; k < k_p; ++k) p[k] = all[k];
        for (uint32_t i = 0; i < n_q; ++i) q[i] = all[k_p + i];
    }
    ks_params *P = new ks_params();
    P->logN = (int)logN;
    P->N = (uint32_t)N;
    P->nq = (int)n_q;
    P->kp = (int)k_p;
    P->dnum = (int)dnum;
    P->alpha = (int)((n_q + dnum - 1) / dnum);
    P->ndig = (P->nq + P->alpha - 1) / P->alpha;
    P->q = q;
    P->p = p;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return fail(KS_ECUDA, "no CUDA device");
    }
    int rc = build_tables(P);
    if (rc != KS_OK) {
        free_tables(P);
        delete P;
        return rc;
    }
    *out = P;
    return KS_OK;
}

void ks_params_destroy(ks_params *P)
{
    if (!P) return;
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    free_ws(P);
    free_tables(P);
    if (P->d_cm_x) cudaFree(P->d_cm_x);
    if (P->d_cm_y) cudaFree(P->d_cm_y);
    delete P;
}

int ks_params_info(const ks_params *P, uint64_t *h_q, uint64_t *h_p, uint32_t *alpha, uint32_t *n_digits)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (h_q) std::memcpy(h_q, P->q.data(), sizeof(uint64_t) * P->nq);
    if (h_p) std::memcpy(h_p, P->p.data(), sizeof(uint64_t) * P->kp);
    if (alpha) *alpha = (uint32_t)P->alpha;
    if (n_digits) *n_digits = (uint32_t)P->ndig;
    return KS_OK;
}

static size_t evk_words(const ks_params *P) { return (size_t)P->ndig * 2 * (P->nq + P->kp) * P->N; }

int ks_key_upload_raw(const ks_params *P, const uint64_t *h_evk, ks_stream_t stream, ks_key **out)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!h_evk || !out) return fail(KS_EINVAL, "NULL argument");
    *out = nullptr;
    if ((rc = set_device(P)) != KS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    ks_key *K = new ks_key();
    K->params = P;
    K->bytes = evk_words(P) * sizeof(u64);
    if ((rc = cuda_check(cudaMalloc((void **)&K->d_evk, K->bytes), "key allocation")) != KS_OK) {
        delete K;
        return rc;
    }
    rc = cuda_check(cudaMemcpyAsync(K->d_evk, h_evk, K->bytes, cudaMemcpyHostToDevice, st), "key upload");
    if (rc == KS_OK) rc = launch_key_convert(P->tables, K->d_evk, st);
    if (rc == KS_OK) rc = cuda_check(cudaStreamSynchronize(st), "key upload sync");
    if (rc != KS_OK) {
        cudaFree(K->d_evk);
        delete K;
        return rc;
    }
    *out = K;
    return KS_OK;
}

void ks_key_destroy(ks_key *K)
{
    if (!K) return;
    cudaSetDevice(K->params->device);
    cudaDeviceSynchronize();
    cudaFree(K->d_evk);
    delete K;
}

size_t ks_key_bytes(const ks_key *K) { return K ? K->bytes : 0; }

// SplitMix64 (Steele, Lea & Flood 2014).
namespace {
struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
};
uint64_t uniform_mod(SplitMix &g, uint64_t m)
{
    int b = 64 - __builtin_clzll(m);
    uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1);
    for (;;) {
        uint64_t v = g.next() & mask;
        if (v < m) return v;
    }
}
int64_t gauss(SplitMix &g)
{
    const double sigma = 3.2;
    for (;;) {
        double u1 = (double)((g.next() >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(g.next() >> 11) * 0x1.0p-53;
        double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
        int64_t e = (int64_t)std::llround(sigma * z);
        if (e >= -19 && e <= 19) return e;
    }
}
// a-word (j, t, n) of a compressed key: the first SplitMix64 draw of stream
// seed^2 at counters ((j*nfull + t)*N + n)*64 + m, masked to bitlen(r), that
// is below r (output c of a stream is reached by starting its state at
// seed^2 + c*gamma); the same definition the kernels regenerate.
uint64_t key_a_word_host(uint64_t seed, int j, int t, size_t n, int logN, int nfull, uint64_t r)
{
    const int b = 64 - __builtin_clzll(r);
    const uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1);
    const uint64_t base = ((((uint64_t)j * nfull + t) << logN) + n) * 64;
    uint64_t v = 0;
    for (int m = 0; m < 64; ++m) {
        SplitMix g{(seed ^ 2) + (base + m) * 0x9E3779B97F4A7C15ULL};
        v = g.next() & mask;
        if (v < r) return v;
    }
    return v % r;
}
}  // namespace

static int keygen_impl(const ks_params *P, const int8_t *h_s, const int64_t *h_s_prime, uint64_t seed,
                       bool compressed, ks_stream_t stream, ks_key **out);

int ks_keygen_upload(const ks_params *P, const int8_t *h_s, const int64_t *h_s_prime, uint64_t seed,
                     ks_stream_t stream, ks_key **out)
{
    return keygen_impl(P, h_s, h_s_prime, seed, false, stream, out);
}

int ks_keygen_upload_compressed(const ks_params *P, const int8_t *h_s, const int64_t *h_s_prime, uint64_t seed,
                                ks_stream_t stream, ks_key **out)
{
    return keygen_impl(P, h_s, h_s_prime, seed, true, stream, out);
}

static int keygen_impl(const ks_params *P, const int8_t *h_s, const int64_t *h_s_prime, uint64_t seed,
                       bool compressed, ks_stream_t stream, ks_key **out)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!h_s || !h_s_prime || !out) return fail(KS_EINVAL, "NULL argument");
    *out = nullptr;
    const size_t N = P->N;
    const int nfull = P->nq + P->kp;
    for (size_t n = 0; n < N; ++n) {
        if (h_s[n] < -1 || h_s[n] > 1) return fail(KS_EINVAL, "s must be ternary");
        if (h_s_prime[n] > (1ll << 62) || h_s_prime[n] < -(1ll << 62)) return fail(KS_EINVAL, "|s'| must be < 2^62");
    }
    if ((rc = set_device(P)) != KS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // host sampling, in the documented draw order
    std::vector<u64> evk_h(evk_words(P), 0);
    SplitMix ga{seed ^ 0}, ge{seed ^ 1};
    for (int j = 0; j < P->ndig; ++j)
        for (int t = 0; t < nfull; ++t) {
            const u64 r = t < P->nq ? P->q[t] : P->p[t - P->nq];
            u64 *dst = evk_h.data() + (((size_t)j * 2 + 1) * nfull + t) * N;
            if (compressed)
                for (size_t n = 0; n < N; ++n) dst[n] = key_a_word_host(seed, j, t, n, P->logN, nfull, r);
            else
                for (size_t n = 0; n < N; ++n) dst[n] = uniform_mod(ga, r);
        }
    std::vector<int64_t> vecs((2 + (size_t)P->ndig) * N);
    for (size_t n = 0; n < N; ++n) {
        vecs[n] = h_s[n];
        vecs[N + n] = h_s_prime[n];
    }
    for (int j = 0; j < P->ndig; ++j)
        for (size_t n = 0; n < N; ++n) vecs[(2 + (size_t)j) * N + n] = gauss(ge);
    std::vector<u64> pmod(nfull, 0);
    for (int t = 0; t < P->nq; ++t) {
        u64 pm = 1;
        for (int k = 0; k < P->kp; ++k) pm = mulmod_h(pm, P->p[k] % P->q[t], P->q[t]);
        pmod[t] = pm;
    }
    ks_key *K = new ks_key();
    K->params = P;
    K->bytes = evk_words(P) * sizeof(u64);
    int64_t *d_vecs = nullptr;
    u64 *d_res = nullptr, *d_pmod = nullptr;
    const int nvec = 2 + P->ndig;
    rc = cuda_check(cudaMalloc((void **)&K->d_evk, K->bytes), "key allocation");
    if (rc == KS_OK) rc = cuda_check(cudaMalloc((void **)&d_vecs, vecs.size() * 8), "keygen scratch");
    if (rc == KS_OK) rc = cuda_check(cudaMalloc((void **)&d_res, (size_t)nvec * nfull * N * 8), "keygen scratch");
    if (rc == KS_OK) rc = cuda_check(cudaMalloc((void **)&d_pmod, nfull * 8), "keygen scratch");
    if (rc == KS_OK)
        rc = cuda_check(cudaMemcpyAsync(K->d_evk, evk_h.data(), K->bytes, cudaMemcpyHostToDevice, st), "key upload");
    if (rc == KS_OK)
        rc = cuda_check(cudaMemcpyAsync(d_vecs, vecs.data(), vecs.size() * 8, cudaMemcpyHostToDevice, st), "upload");
    if (rc == KS_OK) rc = cuda_check(cudaMemcpyAsync(d_pmod, pmod.data(), nfull * 8, cudaMemcpyHostToDevice, st), "upload");
    if (rc == KS_OK) rc = launch_signed_to_towers(P->tables, d_vecs, nvec, d_res, st);
    if (rc == KS_OK) {
        LimbMap m{d_res, d_res, nullptr, nfull, nfull, 0, 0, P->nq, -1};
        rc = launch_ntt_fwd(P->tables, one_map(m, nvec * nfull), true, st);
    }
    if (rc == KS_OK)
        rc = launch_keygen_combine(P->tables, d_res, d_res + (size_t)nfull * N, d_res + 2 * (size_t)nfull * N, d_pmod,
                                   K->d_evk, st);
    if (rc == KS_OK) rc = launch_key_convert(P->tables, K->d_evk, st);
    if (rc == KS_OK && compressed) {
        // keep the b halves only; the a halves are regenerated by the kernels
        u64 *b_only = nullptr;
        const size_t half = (size_t)nfull * N;
        rc = cuda_check(cudaMalloc((void **)&b_only, (size_t)P->ndig * half * 8), "key allocation");
        for (int j = 0; j < P->ndig && rc == KS_OK; ++j)
            rc = cuda_check(cudaMemcpyAsync(b_only + (size_t)j * half, K->d_evk + (size_t)2 * j * half, half * 8,
                                            cudaMemcpyDeviceToDevice, st),
                            "key compaction");
        if (rc == KS_OK) rc = cuda_check(cudaStreamSynchronize(st), "keygen sync");
        if (rc == KS_OK) {
            cudaFree(K->d_evk);
            K->d_evk = b_only;
            K->bytes = (size_t)P->ndig * half * 8;
            K->compressed = 1;
            K->a_seed = seed;
        } else if (b_only) {
            cudaFree(b_only);
        }
    }
    if (rc == KS_OK) rc = cuda_check(cudaStreamSynchronize(st), "keygen sync");
    cudaFree(d_vecs);
    cudaFree(d_res);
    cudaFree(d_pmod);
    if (rc != KS_OK) {
        cudaFree(K->d_evk);
        delete K;
        return rc;
    }
    *out = K;
    return KS_OK;
}

static int switch_one(ks_params *P, const Tables &T, int oc_variant, const ks_key *K, uint32_t nact, const uint64_t *d,
                      uint64_t *o0, uint64_t *o1, ks_dataflow df, cudaStream_t st)
{
    Workspace *w = nullptr;
    const ks_dataflow eff = df == KS_AUTO ? (ks_dataflow)P->sched.dataflow : df;
    int rc = get_ws(P, st, eff == KS_MP || eff == KS_DC, &w);
    if (rc) return rc;
    if (df == KS_AUTO) df = (ks_dataflow)P->sched.dataflow;
    switch (df) {
    case KS_MP: return run_mp(P, T, K, (int)nact, d, o0, o1, w, st);
    case KS_DC: return run_dc(P, T, K, (int)nact, d, o0, o1, w, st);
    case KS_OC:
    case KS_AUTO: return run_oc(P, T, oc_variant, K, (int)nact, d, o0, o1, w, st);
    }
    return fail(KS_EINVAL, "unknown dataflow");
}

int ks_switch(const ks_params *P, const ks_key *K, uint32_t level_towers, const uint64_t *d_in, uint64_t *d_out0,
              uint64_t *d_out1, ks_dataflow dataflow, ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if ((rc = check_job(P, K, level_towers, d_in, d_out0, d_out1)) != KS_OK) return rc;
    if ((int)dataflow < 0 || (int)dataflow > 3) return fail(KS_EINVAL, "unknown dataflow");
    if ((rc = set_device(P)) != KS_OK) return rc;
    return switch_one(const_cast<ks_params *>(P), call_tables(P, P->sched), P->sched.oc_variant, K, level_towers, d_in,
                      d_out0, d_out1, dataflow, (cudaStream_t)stream);
}

int ks_params_set_option(ks_params *P, int option, int value)
{
    int rc = check_params(P);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(P->mu);
    if (option == KS_OPT_BCONV_TENSOR && (value == 0 || value == 1)) {
        P->bconv_tensor = value;
        P->tables.up_tc = value ? P->d_up_tc : nullptr;
        P->tables.dn_tc = value ? P->d_dn_tc : nullptr;
        return KS_OK;
    }
    if (option == KS_OPT_NTT_CLUSTER && value >= 0 && value <= 2) {
        P->ntt_cluster = value;
        P->tables.ntt_cluster = value;
        return KS_OK;
    }
    if (option == KS_OPT_NTT_ROW_STAGE && (value == 0 || value == 1)) {
        P->row_stage = value;
        P->tables.row_stage = value;
        return KS_OK;
    }
    if (option == KS_OPT_BATCH_LANES && value >= 1 && value <= 4) {
        P->batch_lanes = value;
        return KS_OK;
    }
    return fail(KS_EINVAL, "unknown option or value");
}

int ks_device_status(const ks_params *P, int clear, uint32_t *flags)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!flags) return fail(KS_EINVAL, "flags is NULL");
    if ((rc = set_device(P)) != KS_OK) return rc;
    const int v = tc_error_flag(clear != 0);
    const int w = ntt_error_flag(clear != 0);
    if (v < 0 || w < 0) return fail(KS_ECUDA, "device status unreadable");
    *flags = (v ? 1u : 0u) | (w ? 2u : 0u);
    return KS_OK;
}

int ks_switch_hoisted(const ks_params *P, uint32_t n_rot, const ks_key *const *keys, const uint64_t *galois,
                      uint32_t level_towers, const uint64_t *d_in, uint64_t *const *d_out0, uint64_t *const *d_out1,
                      ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (n_rot == 0) return KS_OK;
    if (!keys || !galois || !d_out0 || !d_out1) return fail(KS_EINVAL, "ks_switch_hoisted: NULL array");
    const uint64_t two_n = 2ull * P->N;
    for (uint32_t r = 0; r < n_rot; ++r) {
        if ((rc = check_job(P, keys[r], level_towers, d_in, d_out0[r], d_out1[r])) != KS_OK) return rc;
        if (galois[r] % 2 == 0 || galois[r] >= two_n)
            return fail(KS_EINVAL, "galois elements must be odd and below 2N");
    }
    if ((rc = set_device(P)) != KS_OK) return rc;
    return run_hoisted(const_cast<ks_params *>(P), n_rot, keys, galois, (int)level_towers, d_in, d_out0, d_out1,
                       (cudaStream_t)stream);
}

int ks_automorph(const ks_params *P, uint32_t first_tower, uint32_t n_towers, uint64_t galois, const uint64_t *d_in,
                 uint64_t *d_out, int accumulate, ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (n_towers == 0) return KS_OK;
    if (!d_in || !d_out) return fail(KS_EINVAL, "ks_automorph: NULL data pointer");
    if ((uint64_t)first_tower + n_towers > (uint64_t)(P->nq + P->kp))
        return fail(KS_EINVAL, "ks_automorph: towers beyond the basis");
    if (galois % 2 == 0 || galois >= 2ull * P->N) return fail(KS_EINVAL, "galois element must be odd and below 2N");
    const size_t bytes = (size_t)n_towers * P->N * sizeof(u64);
    const char *a = (const char *)d_in, *b = (const char *)d_out;
    if (a < b + bytes && b < a + bytes) return fail(KS_EINVAL, "ks_automorph: d_in and d_out overlap");
    if ((rc = set_device(P)) != KS_OK) return rc;
    return launch_automorph(P->tables, (int)first_tower, (int)n_towers, d_in, d_out, galois, accumulate != 0,
                            (cudaStream_t)stream);
}

}  // extern "C"

namespace ks {

int check_schedule(const ks_schedule *sc)
{
    if (!sc) return fail(KS_EINVAL, "schedule is NULL");
    if (sc->dataflow < KS_MP || sc->dataflow > KS_OC) return fail(KS_EINVAL, "schedule dataflow must be MP, DC or OC");
    if (sc->oc_variant < 0 || sc->oc_variant > 3) return fail(KS_EINVAL, "schedule oc_variant must be 0, 1, 2 or 3");
    if (sc->chunk < 1 || sc->chunk > kMaxBatch) return fail(KS_EINVAL, "schedule chunk must be in 1..64");
    if (sc->order < 0 || sc->order > 2) return fail(KS_EINVAL, "schedule order must be 0, 1 or 2");
    if (sc->ntt < -1 || sc->ntt > 2) return fail(KS_EINVAL, "schedule ntt must be -1, 0, 1 or 2");
    if (sc->bconv < -1 || sc->bconv > 1) return fail(KS_EINVAL, "schedule bconv must be -1, 0 or 1");
    return KS_OK;
}

static int run_oc_batch(ks_params *P, const Tables &T, uint32_t n, const ks_job *jobs, const ks_schedule &sc,
                        cudaStream_t st);
constexpr uint32_t kLaneJobs = 4;  // fewest jobs worth a lane of their own

static int lane_streams(ks_params *P)
{
    std::lock_guard<std::mutex> g(P->mu);
    if (P->lane_st[0]) return KS_OK;
    for (int l = 0; l < 4; ++l)
        if (cudaStreamCreateWithFlags(&P->lane_st[l], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "lane stream creation failed");
        }
    for (int e = 0; e < 5; ++e)
        if (cudaEventCreateWithFlags(&P->lane_ev[e], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "lane event creation failed");
        }
    return KS_OK;
}

// Run a validated batch under a schedule.
int run_batch(ks_params *P, uint32_t n, const ks_job *jobs, const ks_schedule &sc, cudaStream_t st)
{
    int rc;
    std::vector<uint32_t> idx(n);
    for (uint32_t i = 0; i < n; ++i) idx[i] = i;
    if (sc.order == 1)
        std::stable_sort(idx.begin(), idx.end(),
                         [&](uint32_t a, uint32_t b) { return jobs[a].level_towers > jobs[b].level_towers; });
    else if (sc.order == 2)
        std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return jobs[a].key < jobs[b].key; });
    const Tables T = call_tables(P, sc);
    if (sc.dataflow == KS_MP || sc.dataflow == KS_DC) {
        for (uint32_t i : idx) {
            const ks_job &j = jobs[i];
            rc = switch_one(P, T, sc.oc_variant, j.key, j.level_towers, j.d_in, j.d_out0, j.d_out1,
                            (ks_dataflow)sc.dataflow, st);
            if (rc) return rc;
        }
        return KS_OK;
    }
    // Output-Centric: every stage launch covers a group of sc.chunk jobs, each
    // with its own scratch.  A large batch is split over internal streams
    // (at least kLaneJobs jobs each) forked from and joined back to st, so the
    // memory-bound combine kernels of one part overlap the integer-bound
    // passes of another.
    const int lanes = std::min<int>(P->batch_lanes, (int)(n / kLaneJobs));
    if (lanes > 1) {
        std::vector<ks_job> sorted(n);
        for (uint32_t i = 0; i < n; ++i) sorted[i] = jobs[idx[i]];
        if ((rc = lane_streams(P)) != KS_OK) return rc;
        std::lock_guard<std::mutex> lg(P->lane_mu);  // the fork event and lanes are shared
        if ((rc = cuda_check(cudaEventRecord(P->lane_ev[4], st), "lane fork")) != KS_OK) return rc;
        ks_schedule one = sc;
        one.order = 0;  // already ordered
        uint32_t at = 0;
        for (int l = 0; l < lanes; ++l) {
            const uint32_t cnt = n / lanes + ((uint32_t)l < n % lanes ? 1 : 0);
            if ((rc = cuda_check(cudaStreamWaitEvent(P->lane_st[l], P->lane_ev[4], 0), "lane fork")) != KS_OK) return rc;
            if ((rc = run_oc_batch(P, T, cnt, sorted.data() + at, one, P->lane_st[l])) != KS_OK) return rc;
            if ((rc = cuda_check(cudaEventRecord(P->lane_ev[l], P->lane_st[l]), "lane join")) != KS_OK) return rc;
            if ((rc = cuda_check(cudaStreamWaitEvent(st, P->lane_ev[l], 0), "lane join")) != KS_OK) return rc;
            at += cnt;
        }
        return KS_OK;
    }
    std::vector<ks_job> sorted(n);
    for (uint32_t i = 0; i < n; ++i) sorted[i] = jobs[idx[i]];
    return run_oc_batch(P, T, n, sorted.data(), sc, st);
}

// Output-Centric batch in the given order on one stream.
static int run_oc_batch(ks_params *P, const Tables &T, uint32_t n, const ks_job *jobs, const ks_schedule &sc,
                        cudaStream_t st)
{
    int rc;
    Workspace *w = nullptr;
    if ((rc = get_ws(P, st, false, &w)) != KS_OK) return rc;
    size_t words = 0;
    for (uint32_t i = 0; i < n; ++i) words += oc_scratch_words(P->tables, (int)jobs[i].level_towers);
    {
        std::lock_guard<std::mutex> g(P->mu);
        if (w->batch_words < words) {
            if (w->batch) {
                // the old buffer may still be in use by queued work on this stream
                cudaStreamSynchronize(st);
                cudaFree(w->batch);
                w->batch = nullptr;
                w->batch_words = 0;
            }
            if ((rc = ws_alloc(&w->batch, words)) != KS_OK) return rc;
            w->batch_words = words;
        }
    }
    std::vector<OcJob> oj(n);
    size_t off = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const ks_job &j = jobs[k];
        const int nact = (int)j.level_towers;
        oj[k] = oc_job(P, j.key, nact, j.d_in, j.d_out0, j.d_out1, w->batch + off);
        off += oc_scratch_words(P->tables, nact);
    }
    for (uint32_t i0 = 0; i0 < n; i0 += (uint32_t)sc.chunk) {
        const int m = (int)std::min<uint32_t>((uint32_t)sc.chunk, n - i0);
        if ((rc = launch_oc(T, m, oj.data() + i0, sc.oc_variant, st, sc.order == 2)) != KS_OK) return rc;
    }
    return KS_OK;
}

int check_batch(const ks_params *P, uint32_t n, const ks_job *jobs)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (n > 0 && !jobs) return fail(KS_EINVAL, "jobs is NULL");
    for (uint32_t i = 0; i < n; ++i)
        if ((rc = check_job(P, jobs[i].key, jobs[i].level_towers, jobs[i].d_in, jobs[i].d_out0, jobs[i].d_out1)) != KS_OK)
            return rc;
    return KS_OK;
}

}  // namespace ks

extern "C" {

int ks_switch_batch(const ks_params *P, uint32_t n, const ks_job *jobs, ks_dataflow dataflow, ks_stream_t stream)
{
    int rc = check_batch(P, n, jobs);
    if (rc) return rc;
    if ((int)dataflow < 0 || (int)dataflow > 3) return fail(KS_EINVAL, "unknown dataflow");
    if ((rc = set_device(P)) != KS_OK) return rc;
    ks_schedule sc = P->sched;
    if (dataflow == KS_MP || dataflow == KS_DC) sc.dataflow = dataflow;
    if (dataflow == KS_OC) sc.dataflow = KS_OC;
    if (dataflow == KS_AUTO && n > 0) {
        uint64_t lv = 0;
        for (uint32_t i = 0; i < n; ++i) lv += jobs[i].level_towers;
        const auto sig = tune_signature(n, (uint32_t)(lv / n));
        bool hit = false;
        {
            std::lock_guard<std::mutex> g(P->tune_mu);
            auto it = P->tune.find(sig);
            if (it != P->tune.end()) {
                sc = it->second;
                hit = true;
            }
        }
        if (!hit && P->cost_model) {
            // learned schedule: the cost model's pick, cached for the signature
            ks_schedule pick;
            if ((rc = predict_schedule(const_cast<ks_params *>(P), n, jobs, (cudaStream_t)stream, &pick, nullptr)) !=
                KS_OK)
                return rc;
            std::lock_guard<std::mutex> g(P->tune_mu);
            const_cast<ks_params *>(P)->tune[sig] = pick;
            sc = pick;
        }
    }
    return run_batch(const_cast<ks_params *>(P), n, jobs, sc, (cudaStream_t)stream);
}

int ks_switch_batch_sched(const ks_params *P, uint32_t n, const ks_job *jobs, const ks_schedule *schedule,
                          ks_stream_t stream)
{
    int rc = check_batch(P, n, jobs);
    if (rc) return rc;
    if ((rc = check_schedule(schedule)) != KS_OK) return rc;
    if ((rc = set_device(P)) != KS_OK) return rc;
    return run_batch(const_cast<ks_params *>(P), n, jobs, *schedule, (cudaStream_t)stream);
}

int ks_get_default_schedule(const ks_params *P, ks_schedule *out)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!out) return fail(KS_EINVAL, "out is NULL");
    *out = P->sched;
    return KS_OK;
}

int ks_set_default_schedule(ks_params *P, const ks_schedule *schedule)
{
    int rc = check_params(P);
    if (rc) return rc;
    if ((rc = check_schedule(schedule)) != KS_OK) return rc;
    P->sched = *schedule;
    return KS_OK;
}

}  // extern "C"

namespace ks {
// Chunk sizes of a host batch of n jobs.
static std::vector<uint32_t> host_chunks(uint32_t n)
{
    std::vector<uint32_t> out;
    uint32_t left = n;
    while (left > 0) {
        // equal chunks of at most kHostChunk (consecutive calls pipeline, so
        // the copies at a call's ends are hidden behind the neighbours' work)
        const uint32_t k = (left + kHostChunk - 1) / kHostChunk;
        const uint32_t c = (left + k - 1) / k;
        out.push_back(c);
        left -= c;
    }
    return out;
}
}  // namespace ks

extern "C" {

int ks_switch_batch_host(const ks_params *P, uint32_t n, const ks_host_job *jobs, ks_dataflow dataflow,
                         ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (n > 0 && !jobs) return fail(KS_EINVAL, "jobs is NULL");
    if ((int)dataflow < 0 || (int)dataflow > 3) return fail(KS_EINVAL, "unknown dataflow");
    for (uint32_t i = 0; i < n; ++i) {
        const ks_host_job &j = jobs[i];
        if (!j.key || j.key->params != P) return fail(KS_EINVAL, "key is NULL or belongs to another params object");
        if (j.level_towers < 1 || j.level_towers > (uint32_t)P->nq) return fail(KS_EINVAL, "level_towers must be in 1..n_q");
        if (!j.h_in || !j.h_out0 || !j.h_out1) return fail(KS_EINVAL, "NULL host pointer");
    }
    if ((rc = set_device(P)) != KS_OK) return rc;
    ks_params *PP = const_cast<ks_params *>(P);
    std::lock_guard<std::mutex> g(PP->host_mu);
    HostStage *h = nullptr;
    if ((rc = get_stage(PP, &h)) != KS_OK) return rc;
    // The chunks compute on the stage's own stream: host-buffer jobs read no
    // device data of the caller (keys are complete when their constructors
    // return), so they need not wait for earlier work on the caller's stream, and consecutive calls pipeline (the next call's
    // copy-in and compute overlap this call's copy-out).  The caller's stream
    // waits for every copy-out at the end.
    cudaStream_t cs = h->s_comp, caller = (cudaStream_t)stream;
    const size_t N = P->N;
    const size_t slot_words = (size_t)P->nq * N;
    const std::vector<uint32_t> chunks = host_chunks(n);
    uint64_t call_lv = 0;
    for (uint32_t i = 0; i < n; ++i) call_lv += jobs[i].level_towers;
    const uint32_t call_mean = n ? (uint32_t)(call_lv / n) : 0;
    uint32_t i0 = 0;
    for (size_t c = 0; c < chunks.size(); i0 += chunks[c], ++c) {
        const int s = (int)((h->next + c) & 1);
        const uint32_t m = chunks[c];
        // copy the chunk in once the chunk that last used this slot is computed
        rc = cuda_check(cudaStreamWaitEvent(h->s_in, h->comp[s], 0), "wait");
        for (uint32_t k = 0; k < m && rc == KS_OK; ++k) {
            const ks_host_job &j = jobs[i0 + k];
            const size_t bytes = (size_t)j.level_towers * N * sizeof(u64);
            rc = cuda_check(cudaMemcpyAsync(h->din[s] + k * slot_words, j.h_in, bytes, cudaMemcpyHostToDevice, h->s_in),
                            "H2D copy");
        }
        if (rc == KS_OK) rc = cuda_check(cudaEventRecord(h->h2d[s], h->s_in), "record");
        // compute once the inputs are in and the slot's previous outputs are out
        if (rc == KS_OK) rc = cuda_check(cudaStreamWaitEvent(cs, h->h2d[s], 0), "wait");
        if (rc == KS_OK) rc = cuda_check(cudaStreamWaitEvent(cs, h->d2h[s], 0), "wait");
        if (rc == KS_OK) {
            // the chunk as a device batch (its schedule: tuned for KS_AUTO)
            ks_job dj[kHostChunk];
            uint64_t lv = 0;
            for (uint32_t k = 0; k < m; ++k) {
                const ks_host_job &j = jobs[i0 + k];
                dj[k] = ks_job{j.key, j.level_towers, h->din[s] + k * slot_words, h->dout0[s] + k * slot_words,
                               h->dout1[s] + k * slot_words};
                lv += j.level_towers;
            }
            ks_schedule sc = P->sched;
            if (dataflow == KS_MP || dataflow == KS_DC) sc.dataflow = dataflow;
            if (dataflow == KS_OC) sc.dataflow = KS_OC;
            if (dataflow == KS_AUTO) {
                const auto sig = tune_signature(m, (uint32_t)(lv / m));
                bool hit = false;
                {
                    // the chunk's shape, else the whole call's (tuned on the
                    // device batch these jobs form)
                    std::lock_guard<std::mutex> g(P->tune_mu);
                    auto it = P->tune.find(sig);
                    if (it == P->tune.end()) it = P->tune.find(tune_signature(n, call_mean));
                    if (it != P->tune.end()) {
                        sc = it->second;
                        hit = true;
                    }
                }
                // as ks_switch_batch: the cost model's pick on a miss, cached
                ks_schedule pick;
                if (!hit && P->cost_model && (rc = predict_schedule(PP, m, dj, cs, &pick, nullptr)) == KS_OK) {
                    std::lock_guard<std::mutex> g(P->tune_mu);
                    PP->tune[sig] = pick;
                    sc = pick;
                }
            }
            if (rc == KS_OK) rc = run_batch(PP, m, dj, sc, cs);
        }
        if (rc == KS_OK) rc = cuda_check(cudaEventRecord(h->comp[s], cs), "record");
        // copy out
        if (rc == KS_OK) rc = cuda_check(cudaStreamWaitEvent(h->s_out, h->comp[s], 0), "wait");
        for (uint32_t k = 0; k < m && rc == KS_OK; ++k) {
            const ks_host_job &j = jobs[i0 + k];
            const size_t bytes = (size_t)j.level_towers * N * sizeof(u64);
            rc = cuda_check(cudaMemcpyAsync(j.h_out0, h->dout0[s] + k * slot_words, bytes, cudaMemcpyDeviceToHost,
                                            h->s_out), "D2H copy");
            if (rc == KS_OK)
                rc = cuda_check(cudaMemcpyAsync(j.h_out1, h->dout1[s] + k * slot_words, bytes, cudaMemcpyDeviceToHost,
                                                h->s_out), "D2H copy");
        }
        if (rc == KS_OK) rc = cuda_check(cudaEventRecord(h->d2h[s], h->s_out), "record");
        if (rc) return rc;
    }
    h->next = (int)((h->next + chunks.size()) & 1);
    // later work on the caller's stream is ordered after every copy-out
    for (int s = 0; s < 2; ++s)
        if ((rc = cuda_check(cudaStreamWaitEvent(caller, h->d2h[s], 0), "wait")) != KS_OK) return rc;
    return KS_OK;
}

uint64_t ks_kernel_launches(void) { return g_launches.load(); }

void ks_profile_enable(int on) { g_prof.store(on != 0); }

int ks_profile_collect(uint32_t max, char *names, double *total_ms, uint32_t *counts, uint32_t *n_out)
{
    if (!n_out || (max > 0 && (!names || !total_ms || !counts))) return fail(KS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(g_prof_mu);
    std::vector<std::string> keys;
    std::vector<double> ms;
    std::vector<uint32_t> cnt;
    int rc = KS_OK;
    for (ProfRec &r : g_recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(KS_ECUDA, "profiling event query failed");
        }
        size_t k = 0;
        while (k < keys.size() && keys[k] != r.name) ++k;
        if (k == keys.size()) {
            keys.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[k] += t;
        cnt[k] += 1;
        g_ev_pool.push_back(r.e0);
        g_ev_pool.push_back(r.e1);
    }
    g_recs.clear();
    const uint32_t m = (uint32_t)std::min<size_t>(keys.size(), max);
    for (uint32_t i = 0; i < m; ++i) {
        std::strncpy(names + (size_t)i * 48, keys[i].c_str(), 47);
        names[(size_t)i * 48 + 47] = 0;
        total_ms[i] = ms[i];
        counts[i] = cnt[i];
    }
    *n_out = (uint32_t)keys.size();
    return rc;
}

int ks_ntt(const ks_params *P, uint32_t first_tower, uint32_t n_towers, uint64_t *d_data, int inverse,
           ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!d_data) return fail(KS_EINVAL, "NULL data");
    if ((uint64_t)first_tower + n_towers > (uint64_t)(P->nq + P->kp)) return fail(KS_EINVAL, "tower range outside the basis");
    if ((rc = set_device(P)) != KS_OK) return rc;
    LimbMap m{d_data, d_data, nullptr, (int)n_towers, 0, 0, (int)first_tower, P->nq, -1};
    if (inverse) return launch_ntt_inv(P->tables, one_map(m, (int)n_towers), true, (cudaStream_t)stream);
    return launch_ntt_fwd(P->tables, one_map(m, (int)n_towers), true, (cudaStream_t)stream);
}

int ks_modup(const ks_params *P, uint32_t level_towers, const uint64_t *d_in, uint64_t *d_ext, ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!d_in || !d_ext) return fail(KS_EINVAL, "NULL data");
    if (level_towers < 1 || level_towers > (uint32_t)P->nq) return fail(KS_EINVAL, "level_towers must be in 1..n_q");
    if ((rc = set_device(P)) != KS_OK) return rc;
    ks_params *PP = const_cast<ks_params *>(P);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace *w = nullptr;
    if ((rc = get_ws(PP, st, false, &w)) != KS_OK) return rc;
    const int nact = (int)level_towers;
    const int nt = nact + P->kp;
    const int nd = active_digits(P, nact);
    const Tables &T = P->tables;
    LimbMap m1{d_in, w->y, pre_level(P, nact), nact, 0, 0, 0, nact, -1};
    if ((rc = launch_ntt_inv(T, one_map(m1, nact), false, st)) != KS_OK) return rc;
    BUpJobs bu;
    bu.n = 0;
    add_bup(bu, T, BUpJob{w->y, d_ext, (size_t)nt * P->N, nact, 0, nt, 0, -1});
    if ((rc = launch_bconv_up(T, bu, st)) != KS_OK) return rc;
    LimbMap mD{d_ext, d_ext, nullptr, nt, nt, 0, 0, nact, 0};
    if ((rc = launch_ntt_fwd(T, one_map(mD, nd * nt), true, st)) != KS_OK) return rc;
    return launch_bypass_copy(T, nact, d_in, d_ext, st);
}

int ks_moddown(const ks_params *P, uint32_t level_towers, const uint64_t *d_cp, uint64_t *d_out, ks_stream_t stream)
{
    int rc = check_params(P);
    if (rc) return rc;
    if (!d_cp || !d_out) return fail(KS_EINVAL, "NULL data");
    if (level_towers < 1 || level_towers > (uint32_t)P->nq) return fail(KS_EINVAL, "level_towers must be in 1..n_q");
    if ((rc = set_device(P)) != KS_OK) return rc;
    ks_params *PP = const_cast<ks_params *>(P);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace *w = nullptr;
    if ((rc = get_ws(PP, st, false, &w)) != KS_OK) return rc;
    const int nact = (int)level_towers;
    const int nt = nact + P->kp;
    // fold the ModDown factors in (the key normally carries them)
    LimbMap ms{d_cp, w->cp, nullptr, nt, 0, 0, 0, nact, -1};
    if ((rc = launch_scale(P->tables, one_map(ms, nt), P->d_plain_sc, st)) != KS_OK) return rc;
    return run_moddown(P, P->tables, w, nact, 1, d_out, d_out, st);
}

}  // extern "C"
