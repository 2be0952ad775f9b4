// ks_mlp.cu -- FP32 multilayer perceptron for the learned schedule cost
// model: dense layers with ReLU between them, a linear output layer,
// mean-squared error (optionally masked), backpropagation and Adam, all in
// hand-written kernels.  Sizes are small (width <= 256, batch <= 65535), so
// every kernel is one thread per output element with a loop over the
// contraction; reductions over the batch run in a fixed order (no atomics),
// so training is deterministic.
//
// Parameter layout (host and device): for each layer l, W_l [out][in] then
// b_l [out], layers in order.
#include <cmath>
#include <cstring>
#include <vector>

#include "ks_internal.h"

namespace ks {

constexpr int kMlpMaxLayers = 8;
constexpr int kMlpMaxWidth = 256;

struct MlpLayer {
    int in, out;
    size_t w_off, b_off;  // offsets into the parameter vector
};

}  // namespace ks

struct ks_mlp {
    int nl = 0;
    ks::MlpLayer layer[ks::kMlpMaxLayers];
    size_t nparams = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;  // params, grads, Adam moments
    float *d_act = nullptr;   // activations of every layer for the batch: [nl+1][batch][width]
    float *d_delta = nullptr;  // two ping-pong delta buffers [2][batch][width]
    float *d_part = nullptr;   // loss partial sums
    size_t cap_batch = 0;
    long step = 0;
    int width_max = 0;
};

namespace ks {

// act_out[b][o] = f(sum_i W[o][i] act_in[b][i] + bias[o]), f = ReLU unless last.
__global__ void k_mlp_dense(const float *p, size_t w_off, size_t b_off, int in, int out, int batch,
                            const float *act_in, float *act_out, int relu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * out) return;
    const int b = idx / out, o = idx % out;
    const float *w = p + w_off + (size_t)o * in;
    const float *x = act_in + (size_t)b * in;
    float acc = p[b_off + o];
    for (int i = 0; i < in; ++i) acc = fmaf(w[i], x[i], acc);
    act_out[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// Output delta of the loss L = sum mask*(y-t)^2 / count, and per-block
// partial sums of the loss (fixed-order reduction later).
__global__ void k_mlp_loss(const float *y, const float *t, const float *mask, int n, float inv_count, float *delta,
                           float *part)
{
    __shared__ float s[256];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (idx < n) {
        const float m = mask ? mask[idx] : 1.f;
        const float d = y[idx] - t[idx];
        delta[idx] = 2.f * m * d * inv_count;
        l = m * d * d * inv_count;
    }
    s[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// dW[o][i] = sum_b delta[b][o] x[b][i]; db[o] = sum_b delta[b][o].
__global__ void k_mlp_wgrad(float *g, size_t w_off, size_t b_off, int in, int out, int batch, const float *x,
                            const float *delta)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= out * (in + 1)) return;
    const int o = idx / (in + 1), i = idx % (in + 1);
    float acc = 0.f;
    if (i < in) {
        for (int b = 0; b < batch; ++b) acc = fmaf(delta[(size_t)b * out + o], x[(size_t)b * in + i], acc);
        g[w_off + (size_t)o * in + i] = acc;
    } else {
        for (int b = 0; b < batch; ++b) acc += delta[(size_t)b * out + o];
        g[b_off + o] = acc;
    }
}

// delta_in[b][i] = (sum_o W[o][i] delta_out[b][o]) * [act_in[b][i] > 0].
__global__ void k_mlp_back(const float *p, size_t w_off, int in, int out, int batch, const float *delta_out,
                           const float *act_in, float *delta_in)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * in) return;
    const int b = idx / in, i = idx % in;
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(p[w_off + (size_t)o * in + i], delta_out[(size_t)b * out + o], acc);
    delta_in[idx] = act_in[idx] > 0.f ? acc : 0.f;
}

// Adam (Kingma & Ba) with bias correction.
__global__ void k_mlp_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                           float eps, float c1, float c2)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const float gi = g[idx];
    const float mi = b1 * m[idx] + (1.f - b1) * gi;
    const float vi = b2 * v[idx] + (1.f - b2) * gi * gi;
    m[idx] = mi;
    v[idx] = vi;
    p[idx] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static int ensure_batch(ks_mlp *M, size_t batch)
{
    if (batch <= M->cap_batch) return KS_OK;
    cudaFree(M->d_act);
    cudaFree(M->d_delta);
    cudaFree(M->d_part);
    M->d_act = M->d_delta = M->d_part = nullptr;
    M->cap_batch = 0;
    const size_t w = (size_t)M->width_max;
    if (cudaMalloc((void **)&M->d_act, sizeof(float) * (M->nl + 1) * batch * w) != cudaSuccess ||
        cudaMalloc((void **)&M->d_delta, sizeof(float) * 2 * batch * w) != cudaSuccess ||
        cudaMalloc((void **)&M->d_part, sizeof(float) * (batch * w / 256 + 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ENOMEM, "MLP activation buffers");
    }
    M->cap_batch = batch;
    return KS_OK;
}

static float *act(ks_mlp *M, int l) { return M->d_act + (size_t)l * M->cap_batch * M->width_max; }

static int forward(ks_mlp *M, int batch, const float *d_x, cudaStream_t st)
{
    cudaMemcpyAsync(act(M, 0), d_x, sizeof(float) * batch * M->layer[0].in, cudaMemcpyDeviceToDevice, st);
    for (int l = 0; l < M->nl; ++l) {
        const MlpLayer &L = M->layer[l];
        const int n = batch * L.out;
        KS_LAUNCH(st, "mlp_dense", k_mlp_dense<<<(n + 255) / 256, 256, 0, st>>>(
                                       M->d_p, L.w_off, L.b_off, L.in, L.out, batch, act(M, l), act(M, l + 1),
                                       l + 1 < M->nl ? 1 : 0));
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KS_OK : fail(KS_ECUDA, std::string("MLP forward: ") + cudaGetErrorString(e));
}

// Loss and gradients of the current batch into d_g; *h_loss gets the loss.
static int backward(ks_mlp *M, int batch, const float *d_t, const float *d_mask, float *h_loss, cudaStream_t st)
{
    const int nout = M->layer[M->nl - 1].out;
    const int n = batch * nout;
    float count = (float)n;
    if (d_mask) {
        std::vector<float> hm(n);
        cudaMemcpyAsync(hm.data(), d_mask, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        count = 0.f;
        for (float v : hm) count += v;
        if (count <= 0.f) count = 1.f;
    }
    const int nb = (n + 255) / 256;
    float *delta = M->d_delta;
    float *delta2 = M->d_delta + M->cap_batch * M->width_max;
    KS_LAUNCH(st, "mlp_loss", k_mlp_loss<<<nb, 256, 0, st>>>(act(M, M->nl), d_t, d_mask, n, 1.f / count, delta,
                                                             M->d_part));
    for (int l = M->nl - 1; l >= 0; --l) {
        const MlpLayer &L = M->layer[l];
        const int nw = L.out * (L.in + 1);
        KS_LAUNCH(st, "mlp_wgrad",
                  k_mlp_wgrad<<<(nw + 255) / 256, 256, 0, st>>>(M->d_g, L.w_off, L.b_off, L.in, L.out, batch,
                                                                act(M, l), delta));
        if (l > 0) {
            const int nx = batch * L.in;
            KS_LAUNCH(st, "mlp_back",
                      k_mlp_back<<<(nx + 255) / 256, 256, 0, st>>>(M->d_p, L.w_off, L.in, L.out, batch, delta,
                                                                   act(M, l), delta2));
            std::swap(delta, delta2);
        }
    }
    if (h_loss) {
        std::vector<float> part(nb);
        cudaMemcpyAsync(part.data(), M->d_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return fail(KS_ECUDA, "MLP loss readback");
        }
        double s = 0.0;
        for (float v : part) s += v;
        *h_loss = (float)s;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KS_OK : fail(KS_ECUDA, std::string("MLP backward: ") + cudaGetErrorString(e));
}

int mlp_io_dims(const ks_mlp *M, int *in, int *out)
{
    if (!M || M->nl < 1) return fail(KS_EINVAL, "MLP is NULL");
    *in = M->layer[0].in;
    *out = M->layer[M->nl - 1].out;
    return KS_OK;
}

int mlp_reserve(ks_mlp *M, int batch) { return ensure_batch(M, batch); }

}  // namespace ks

using namespace ks;

extern "C" {

int ks_mlp_create(uint32_t n_layers, const uint32_t *dims, uint64_t seed, ks_mlp **out)
{
    if (!dims || !out || n_layers < 1 || n_layers > (uint32_t)kMlpMaxLayers) return fail(KS_EINVAL, "MLP: 1..8 layers");
    for (uint32_t l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > (uint32_t)kMlpMaxWidth) return fail(KS_EINVAL, "MLP: widths 1..256");
    ks_mlp *M = new ks_mlp();
    M->nl = (int)n_layers;
    size_t off = 0;
    for (int l = 0; l < M->nl; ++l) {
        M->layer[l] = {(int)dims[l], (int)dims[l + 1], off, off + (size_t)dims[l] * dims[l + 1]};
        off += (size_t)dims[l + 1] * (dims[l] + 1);
        M->width_max = std::max<int>(M->width_max, std::max(dims[l], dims[l + 1]));
    }
    M->nparams = off;
    // He-normal initialisation from a SplitMix64 stream (Box-Muller), zero biases.
    std::vector<float> h(off, 0.f);
    uint64_t s = seed;
    auto next = [&s]() {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    for (int l = 0; l < M->nl; ++l) {
        const MlpLayer &L = M->layer[l];
        const double sd = std::sqrt(2.0 / L.in);
        for (size_t k = 0; k < (size_t)L.in * L.out; ++k) {
            double u1 = ((next() >> 11) + 1) * 0x1.0p-53, u2 = (next() >> 11) * 0x1.0p-53;
            h[L.w_off + k] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    if (cudaMalloc((void **)&M->d_p, sizeof(float) * off) != cudaSuccess ||
        cudaMalloc((void **)&M->d_g, sizeof(float) * off) != cudaSuccess ||
        cudaMalloc((void **)&M->d_m, sizeof(float) * off) != cudaSuccess ||
        cudaMalloc((void **)&M->d_v, sizeof(float) * off) != cudaSuccess) {
        cudaGetLastError();
        ks_mlp_destroy(M);
        return fail(KS_ENOMEM, "MLP parameter buffers");
    }
    cudaMemcpy(M->d_p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    cudaMemset(M->d_m, 0, sizeof(float) * off);
    cudaMemset(M->d_v, 0, sizeof(float) * off);
    cudaMemset(M->d_g, 0, sizeof(float) * off);
    *out = M;
    return KS_OK;
}

void ks_mlp_destroy(ks_mlp *M)
{
    if (!M) return;
    float *bufs[] = {M->d_p, M->d_g, M->d_m, M->d_v, M->d_act, M->d_delta, M->d_part};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete M;
}

size_t ks_mlp_num_params(const ks_mlp *M) { return M ? M->nparams : 0; }

int ks_mlp_get_params(const ks_mlp *M, float *h)
{
    if (!M || !h) return fail(KS_EINVAL, "NULL argument");
    if (cudaMemcpy(h, M->d_p, sizeof(float) * M->nparams, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "MLP parameter readback");
    }
    return KS_OK;
}

int ks_mlp_set_params(ks_mlp *M, const float *h)
{
    if (!M || !h) return fail(KS_EINVAL, "NULL argument");
    if (cudaMemcpy(M->d_p, h, sizeof(float) * M->nparams, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "MLP parameter upload");
    }
    cudaMemset(M->d_m, 0, sizeof(float) * M->nparams);
    cudaMemset(M->d_v, 0, sizeof(float) * M->nparams);
    M->step = 0;
    return KS_OK;
}

int ks_mlp_forward(ks_mlp *M, uint32_t batch, const float *d_x, float *d_y, ks_stream_t stream)
{
    if (!M || !d_x || !d_y || batch < 1 || batch > 65535) return fail(KS_EINVAL, "MLP forward: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_batch(M, batch);
    if (rc == KS_OK) rc = forward(M, (int)batch, d_x, st);
    if (rc == KS_OK)
        cudaMemcpyAsync(d_y, act(M, M->nl), sizeof(float) * batch * M->layer[M->nl - 1].out, cudaMemcpyDeviceToDevice,
                        st);
    return rc;
}

int ks_mlp_gradients(ks_mlp *M, uint32_t batch, const float *d_x, const float *d_t, const float *d_mask, float *h_grad,
                     float *h_loss, ks_stream_t stream)
{
    if (!M || !d_x || !d_t || batch < 1 || batch > 65535) return fail(KS_EINVAL, "MLP gradients: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_batch(M, batch);
    if (rc == KS_OK) rc = forward(M, (int)batch, d_x, st);
    if (rc == KS_OK) rc = backward(M, (int)batch, d_t, d_mask, h_loss, st);
    if (rc == KS_OK && h_grad &&
        cudaMemcpy(h_grad, M->d_g, sizeof(float) * M->nparams, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(KS_ECUDA, "MLP gradient readback");
    }
    return rc;
}

int ks_mlp_train_step(ks_mlp *M, uint32_t batch, const float *d_x, const float *d_t, const float *d_mask, float lr,
                      float *h_loss, ks_stream_t stream)
{
    int rc = ks_mlp_gradients(M, batch, d_x, d_t, d_mask, nullptr, h_loss, stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    const size_t n = M->nparams;
    KS_LAUNCH(st, "mlp_adam", k_mlp_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->d_p, M->d_g, M->d_m, M->d_v,
                                                                                     n, lr, b1, b2, 1e-8f, c1, c2));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KS_OK : fail(KS_ECUDA, std::string("MLP Adam: ") + cudaGetErrorString(e));
}

}  // extern "C"
