// ks_tune.cu -- schedule autotuner: exhaustive timing of the candidate
// schedules of a batch with CUDA events, a per-parameter-set cache of the
// winners (used by KS_AUTO), its text persistence, and synthetic keys for
// tuning runs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ks_internal.h"
#include "ks_launch.h"

namespace ks {

// Candidate order is part of the interface: the learned cost model predicts
// one time per structural candidate in this order.
static std::vector<ks_schedule> candidates()
{
    std::vector<ks_schedule> c;
    c.push_back({KS_MP, 0, 1, 0, -1, -1});
    c.push_back({KS_DC, 0, 1, 0, -1, -1});
    c.push_back({KS_OC, 0, 64, 0, -1, -1});
    for (int ch : {1, 8, 64}) c.push_back({KS_OC, 1, ch, 0, -1, -1});
    for (int ch : {1, 8, 16, 64}) c.push_back({KS_OC, 2, ch, 0, -1, -1});
    c.push_back({KS_OC, 1, 64, 1, -1, -1});
    c.push_back({KS_OC, 2, 64, 1, -1, -1});
    c.push_back({KS_OC, 3, 64, 0, -1, -1});
    return c;
}

// Relative timing difference below which stage 1 treats schedules as tied.
constexpr float kTieFrac = 0.003f;

// Implementation pairs (ntt, bconv) of the second stage, in ms_out order.
constexpr int kImplPairs = 4;
static const int kImpl[kImplPairs][2] = {{0, 1}, {1, 1}, {0, 0}, {1, 0}};

// Best of reps timed runs of one schedule (after one untimed run).
static int time_schedule(ks_params *P, uint32_t n, const ks_job *jobs, const ks_schedule &sc, uint32_t reps,
                         cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    int rc = run_batch(P, n, jobs, sc, st);  // untimed: scratch allocation, caches
    float m = 1e30f;
    for (uint32_t r = 0; r < reps && rc == KS_OK; ++r) {
        cudaEventRecord(e0, st);
        rc = run_batch(P, n, jobs, sc, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "ks_autotune: device error while timing");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        m = std::min(m, t);
    }
    *ms = m;
    return rc;
}

static int tune_impl(ks_params *P, uint32_t n, const ks_job *jobs, uint32_t reps, cudaStream_t st, cudaEvent_t e0,
                     cudaEvent_t e1, const ks_schedule &base, float *ms_out, ks_schedule *best)
{
    float best_ms = 1e30f;
    for (int i = 0; i < 4; ++i) {
        ks_schedule sc = base;
        sc.ntt = kImpl[i][0];
        sc.bconv = kImpl[i][1];
        float m = 0.f;
        const int rc = time_schedule(P, n, jobs, sc, reps, st, e0, e1, &m);
        if (rc != KS_OK) return rc;
        if (ms_out) ms_out[i] = m;
        if (m < best_ms) {
            best_ms = m;
            *best = sc;
        }
    }
    return KS_OK;
}

// ------------------------------------------------------------------ cost model
// Inputs of the learned cost model: (logN, L+1, dnum, K, log2 batch, alpha,
// log2 input words), each scaled to roughly unit range by fixed constants,
// then three +-1 flags of which implementations exist for the shape: the
// tensor-core ModUp base conversion (at most 18 sources per digit), the
// tensor-core ModDown one (at most 18 special towers), and the cluster NTT
// (ring degrees other than 2^13 and 2^17); where one is missing, its
// schedule field selects the same kernels as the other value.  The Python
// training code computes the same vector (tune.features).
constexpr int kCostFeatures = 10;

static void cost_features(int logN, int nq, int dnum, int kp, int batch, int alpha_params, float *x)
{
    const int alpha = (nq + dnum - 1) / dnum;
    const double words = (double)batch * nq * std::ldexp(1.0, logN);
    x[0] = (float)((logN - 15) / 2.0);
    x[1] = (float)((nq - 25) / 14.0);
    x[2] = (float)((dnum - 12) / 12.0);
    x[3] = (float)((kp - 6.5) / 3.5);
    x[4] = (float)((std::log2((double)batch) - 4) / 2.5);
    x[5] = (float)((alpha - 12) / 12.0);
    x[6] = (float)((std::log2(words) - 22) / 3.0);
    x[7] = alpha_params <= 18 ? 1.f : -1.f;
    x[8] = kp <= 18 ? 1.f : -1.f;
    x[9] = (logN != 13 && logN != 17) ? 1.f : -1.f;
}

// Features of a batch: its mean level (rounded) stands for L+1; at the top
// level dnum is the parameter set's, below it the number of active digits.
static void batch_features(const ks_params *P, uint32_t n, const ks_job *jobs, float *x)
{
    uint64_t lv = 0;
    for (uint32_t i = 0; i < n; ++i) lv += jobs[i].level_towers;
    const int nact = std::max(1, (int)((lv + n / 2) / n));
    const int dnum = nact == P->nq ? P->dnum : (nact + P->alpha - 1) / P->alpha;
    cost_features(P->logN, nact, dnum, P->kp, (int)n, P->alpha, x);
}

int predict_schedule(ks_params *P, uint32_t n, const ks_job *jobs, cudaStream_t st, ks_schedule *out, float *h_pred)
{
    if (!P->cost_model) return fail(KS_EINVAL, "no cost model attached to this parameter set");
    const std::vector<ks_schedule> c = candidates();
    const int nout = (int)c.size() + kImplPairs;
    float x[kCostFeatures];
    batch_features(P, n, jobs, x);
    std::vector<float> y(nout);
    {
        static std::mutex mu;  // one model may serve several parameter sets
        std::lock_guard<std::mutex> g(mu);
        if (cudaMemcpyAsync(P->d_cm_x, x, sizeof(x), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "cost model: feature upload");
        }
        int rc = ks_mlp_forward(P->cost_model, 1, P->d_cm_x, P->d_cm_y, (ks_stream_t)st);
        if (rc != KS_OK) return rc;
        if (cudaMemcpyAsync(y.data(), P->d_cm_y, sizeof(float) * nout, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "cost model: prediction readback");
        }
    }
    int bs = 0, bi = 0;
    for (int i = 1; i < (int)c.size(); ++i)
        if (y[i] < y[bs]) bs = i;
    for (int i = 1; i < kImplPairs; ++i)
        if (y[c.size() + i] < y[c.size() + bi]) bi = i;
    ks_schedule s = c[bs];
    s.ntt = kImpl[bi][0];
    s.bconv = kImpl[bi][1];
    *out = s;
    if (h_pred)
        for (int i = 0; i < nout; ++i) h_pred[i] = y[i] * P->cm_scale + P->cm_mean;
    return KS_OK;
}

std::pair<uint32_t, uint32_t> tune_signature(uint32_t n, uint32_t mean_level)
{
    uint32_t b = 1;
    while (b < n) b <<= 1;
    return {b, (mean_level + 2) / 4 * 4};
}

static std::string device_name(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s = prop.name;
    for (char &ch : s)
        if (ch == ' ') ch = '_';
    return s;
}

static std::string params_tag(const ks_params *P)
{
    std::ostringstream o;
    o << "logN=" << P->logN << " nq=" << P->nq << " kp=" << P->kp << " dnum=" << P->dnum << " q0=" << P->q[0]
      << " p0=" << P->p[0];
    return o.str();
}

}  // namespace ks

using namespace ks;

extern "C" {

int ks_tune_candidates(const ks_params *P, uint32_t max, ks_schedule *out, uint32_t *n_out)
{
    if (!P || !n_out || (max > 0 && !out)) return fail(KS_EINVAL, "ks_tune_candidates: NULL argument");
    std::vector<ks_schedule> c = candidates();
    *n_out = (uint32_t)c.size();
    for (uint32_t i = 0; i < max && i < c.size(); ++i) out[i] = c[i];
    return KS_OK;
}

static int tune_events(ks_params *P, cudaEvent_t *e0, cudaEvent_t *e1)
{
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    if (cudaEventCreate(e0) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "ks_autotune: event creation failed");
    }
    if (cudaEventCreate(e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(*e0);
        return fail(KS_ECUDA, "ks_autotune: event creation failed");
    }
    return KS_OK;
}

int ks_autotune(ks_params *P, uint32_t n, const ks_job *jobs, uint32_t reps, ks_stream_t stream, uint32_t max,
                float *ms_out, ks_schedule *best)
{
    int rc = check_batch(P, n, jobs);
    if (rc) return rc;
    if (n == 0 || reps < 1 || !best) return fail(KS_EINVAL, "ks_autotune: need n >= 1, reps >= 1 and best");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if ((rc = tune_events(P, &e0, &e1)) != KS_OK) return rc;
    // stage 1: structure
    std::vector<ks_schedule> c = candidates();
    std::vector<float> ms(c.size(), 1e30f);
    float best_ms = 1e30f;
    for (size_t i = 0; i < c.size() && rc == KS_OK; ++i) {
        rc = time_schedule(P, n, jobs, c[i], reps, st, e0, e1, &ms[i]);
        if (rc != KS_OK) break;
        if (i < max && ms_out) ms_out[i] = ms[i];
        best_ms = std::min(best_ms, ms[i]);
    }
    // Among the schedules within kTieFrac of the fastest (timing noise),
    // the one with the largest launch groups: the same time in fewer launches.
    ks_schedule base = c[0];
    int base_chunk = -1;
    for (size_t i = 0; i < c.size(); ++i)
        if (ms[i] <= best_ms * (1.0f + kTieFrac) && c[i].chunk > base_chunk) {
            base = c[i];
            base_chunk = c[i].chunk;
        }
    // stage 2: implementation of the fastest structure (its four timings go
    // to ms_out after the structural ones when the caller has room for them)
    float *impl_out = (ms_out && max >= c.size() + kImplPairs) ? ms_out + c.size() : nullptr;
    if (rc == KS_OK) rc = tune_impl(P, n, jobs, reps, st, e0, e1, base, impl_out, best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KS_OK) return rc;
    uint64_t lv = 0;
    for (uint32_t i = 0; i < n; ++i) lv += jobs[i].level_towers;
    std::lock_guard<std::mutex> g(P->tune_mu);
    P->tune[tune_signature(n, (uint32_t)(lv / n))] = *best;
    return KS_OK;
}

int ks_autotune_impl(ks_params *P, uint32_t n, const ks_job *jobs, uint32_t reps, ks_stream_t stream,
                     const ks_schedule *base, float *ms_out, ks_schedule *best)
{
    int rc = check_batch(P, n, jobs);
    if (rc) return rc;
    if ((rc = check_schedule(base)) != KS_OK) return rc;
    if (n == 0 || reps < 1 || !best) return fail(KS_EINVAL, "ks_autotune_impl: need n >= 1, reps >= 1 and best");
    cudaEvent_t e0, e1;
    if ((rc = tune_events(P, &e0, &e1)) != KS_OK) return rc;
    rc = tune_impl(P, n, jobs, reps, (cudaStream_t)stream, e0, e1, *base, ms_out, best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int ks_params_set_cost_model(ks_params *P, ks_mlp *model, float t_mean, float t_scale)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    std::lock_guard<std::mutex> g(P->mu);
    if (!model) {
        P->cost_model = nullptr;
        return KS_OK;
    }
    int in = 0, out = 0;
    int rc = mlp_io_dims(model, &in, &out);
    if (rc != KS_OK) return rc;
    const int want = (int)candidates().size() + kImplPairs;
    if (in != kCostFeatures || out != want)
        return fail(KS_EINVAL, "cost model must map " + std::to_string(kCostFeatures) + " features to " +
                                   std::to_string(want) + " outputs (structural candidates, then implementation pairs)");
    if (!(t_scale > 0.f)) return fail(KS_EINVAL, "cost model: t_scale must be positive");
    // buffers for one row, and the model's activation buffers for batch 1,
    // allocated here so that KS_AUTO itself allocates nothing
    if (!P->d_cm_x && cudaMalloc((void **)&P->d_cm_x, sizeof(float) * kCostFeatures) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ENOMEM, "cost model buffers");
    }
    if (!P->d_cm_y && cudaMalloc((void **)&P->d_cm_y, sizeof(float) * 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ENOMEM, "cost model buffers");
    }
    if ((rc = mlp_reserve(model, 1)) != KS_OK) return rc;
    P->cost_model = model;
    P->cm_mean = t_mean;
    P->cm_scale = t_scale;
    return KS_OK;
}

int ks_predict_schedule(ks_params *P, uint32_t n, const ks_job *h_jobs, ks_stream_t stream, ks_schedule *out,
                        float *h_pred)
{
    int rc = check_batch(P, n, h_jobs);
    if (rc) return rc;
    if (n == 0 || !out) return fail(KS_EINVAL, "ks_predict_schedule: need n >= 1 and out");
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    return predict_schedule(P, n, h_jobs, (cudaStream_t)stream, out, h_pred);
}

int ks_cost_features(const ks_params *P, uint32_t n, const ks_job *h_jobs, float *h_x)
{
    if (!P || !h_jobs || !h_x || n == 0) return fail(KS_EINVAL, "ks_cost_features: NULL argument or n = 0");
    batch_features(P, n, h_jobs, h_x);
    return KS_OK;
}

int ks_tune_cache_put(ks_params *P, uint32_t n_jobs, uint32_t mean_level, const ks_schedule *s)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    int rc = check_schedule(s);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(P->tune_mu);
    P->tune[tune_signature(n_jobs, mean_level)] = *s;
    return KS_OK;
}

int ks_tune_cache_get(const ks_params *P, uint32_t n_jobs, uint32_t mean_level, ks_schedule *out)
{
    if (!P || !out) return fail(KS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(P->tune_mu);
    auto it = P->tune.find(tune_signature(n_jobs, mean_level));
    if (it == P->tune.end()) return fail(KS_EINVAL, "no tuned schedule for this signature");
    *out = it->second;
    return KS_OK;
}

int ks_tune_cache_save(const ks_params *P, const char *path)
{
    if (!P || !path) return fail(KS_EINVAL, "NULL argument");
    std::ofstream f(path);
    if (!f) return fail(KS_EINVAL, std::string("cannot write ") + path);
    f << "# ks tuning cache v2 (sched=dataflow,oc_variant,chunk,order,ntt,bconv)\n";
    const std::string tag = params_tag(P), dev = device_name(P->device);
    std::lock_guard<std::mutex> g(P->tune_mu);
    for (const auto &kv : P->tune)
        f << dev << " " << tag << " n=" << kv.first.first << " level=" << kv.first.second
          << " sched=" << kv.second.dataflow << "," << kv.second.oc_variant << "," << kv.second.chunk << ","
          << kv.second.order << "," << kv.second.ntt << "," << kv.second.bconv << "\n";
    return f.good() ? KS_OK : fail(KS_EINVAL, std::string("write failed: ") + path);
}

int ks_tune_cache_load(ks_params *P, const char *path)
{
    if (!P || !path) return fail(KS_EINVAL, "NULL argument");
    std::ifstream f(path);
    if (!f) return fail(KS_EINVAL, std::string("cannot read ") + path);
    const std::string prefix = device_name(P->device) + " " + params_tag(P) + " ";
    std::string line;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#' || line.compare(0, prefix.size(), prefix) != 0) continue;
        unsigned n = 0, lvl = 0;
        int d = 0, v = 0, ch = 0, o = 0, nt = -1, bc = -1;
        // v1 lines hold the four structural fields; the implementation fields
        // then take the parameter set's options (-1)
        const int got = std::sscanf(line.c_str() + prefix.size(), "n=%u level=%u sched=%d,%d,%d,%d,%d,%d", &n, &lvl,
                                    &d, &v, &ch, &o, &nt, &bc);
        if (got != 6 && got != 8) continue;
        ks_schedule s{d, v, ch, o, nt, bc};
        if (check_schedule(&s) != KS_OK) continue;
        std::lock_guard<std::mutex> g(P->tune_mu);
        P->tune[{n, lvl}] = s;
    }
    set_error("");
    return KS_OK;
}

int ks_key_synthetic(const ks_params *P, uint64_t seed, ks_stream_t stream, ks_key **out)
{
    if (!P || !out) return fail(KS_EINVAL, "NULL argument");
    *out = nullptr;
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    ks_key *K = new ks_key();
    K->params = P;
    K->bytes = (size_t)P->ndig * 2 * (P->nq + P->kp) * P->N * sizeof(u64);
    if (cudaMalloc((void **)&K->d_evk, K->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete K;
        return fail(KS_ENOMEM, "key allocation failed");
    }
    int rc = launch_key_random(P->tables, K->d_evk, seed, (cudaStream_t)stream);
    if (rc == KS_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(KS_ECUDA, "synthetic key generation failed");
    }
    if (rc != KS_OK) {
        cudaFree(K->d_evk);
        delete K;
        return rc;
    }
    *out = K;
    return KS_OK;
}

}  // extern "C"
