// ks_probe.cu -- arithmetic ceilings of this GPU for the two inner loops of
// key switching, measured with the same device functions the kernels use:
//   * the forward NTT butterfly (Shoup product by a twiddle, lazy sums),
//   * the base-conversion multiply-accumulate (three 32x32->64 multiply-adds
//     into three 64-bit column sums, Karatsuba form).
// Each probe runs a register-only loop on every SM (no memory traffic inside
// the timed loop), so its rate is what the integer pipes can sustain; the
// benchmark divides the kernels' achieved rates by these to give a roofline
// fraction for the arithmetic-bound stages.
#include "ks_device.cuh"

namespace ks {

constexpr int kProbeBlocks = 152 * 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_bfly(u64 *out, u64 q, u64 w, u64 wp, int iters)
{
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = (threadIdx.x * 16 + i + blockIdx.x) % q;
    const u64 q2 = 2 * q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) fwd_bfly(x[i], x[i + 8], w + i, wp + i, q, q2);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            fwd_bfly(x[i], x[i + 4], w, wp, q, q2);
            fwd_bfly(x[i + 8], x[i + 12], w + 1, wp + 1, q, q2);
        }
    }
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the loop alive
}

// The inverse (Harvey) butterfly in the same pattern.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ibfly(u64 *out, u64 q, u64 w, u64 wp, int iters)
{
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = (threadIdx.x * 16 + i + blockIdx.x) % q;
    const u64 q2 = 2 * q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) inv_bfly(x[i], x[i + 8], w + i, wp + i, q, q2);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            inv_bfly(x[i], x[i + 4], w, wp, q, q2);
            inv_bfly(x[i + 8], x[i + 12], w + 1, wp + 1, q, q2);
        }
    }
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_bmac(u64 *out, u64 c, int iters)
{
    BAcc acc[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) bacc_zero(acc[g]);
    u64 y = threadIdx.x + 7 * blockIdx.x;
    for (int it = 0; it < iters; ++it) {
        u32 y0, y1;
        split_y(y, y0, y1);
#pragma unroll
        for (int g = 0; g < 8; ++g) bacc_mac(acc[g], y0, y1, c + g);
        y = (y ^ (y >> 7)) + (u64)it;  // a new source value each iteration
    }
    u64 s = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) s += acc[g].a0 ^ acc[g].a1 ^ acc[g].a2;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Throughput of single integer instructions (the building blocks of the
// kernels' modular arithmetic): 8 independent chains per thread.
constexpr int kPipeIters = 2048;
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe_pipe(u64 *out, u64 b0)
{
    u64 acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x + c;
    for (int it = 0; it < kPipeIters; ++it) {
        const u64 b = b0 + it;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (OP == 0) {  // mad.lo.u32
                uint32_t a = (uint32_t)acc[c];
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"((uint32_t)b), "r"((uint32_t)b0));
                acc[c] = a;
            } else if (OP == 1) {  // mad.wide.u32 (64-bit accumulate)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[c]) : "r"((uint32_t)acc[c]), "r"((uint32_t)b));
            } else if (OP == 2) {  // mul.lo.u64
                asm volatile("mul.lo.u64 %0, %0, %1;" : "+l"(acc[c]) : "l"(b));
            } else if (OP == 3) {  // mul.hi.u64
                asm volatile("mul.hi.u64 %0, %0, %1;" : "+l"(acc[c]) : "l"(b | 0x100000000ull));
            } else {  // add.u32
                uint32_t a = (uint32_t)acc[c];
                asm volatile("add.u32 %0, %0, %1;" : "+r"(a) : "r"((uint32_t)b));
                acc[c] = a;
            }
        }
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ks

using namespace ks;

extern "C" int ks_probe_int_pipes(double *lanes_per_clk_sm, int n)
{
    if (!lanes_per_clk_sm || n < 5) return fail(KS_EINVAL, "ks_probe_int_pipes: need room for 5 rates");
    int dev = 0, sms = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "ks_probe_int_pipes: device query failed");
    }
    u64 *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc((void **)&out, sizeof(u64) * kProbeBlocks * kProbeThreads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (out) cudaFree(out);
        return fail(KS_ECUDA, "ks_probe_int_pipes: setup failed");
    }
    const double ops = (double)kProbeBlocks * kProbeThreads * kPipeIters * 8;
    for (int op = 0; op < 5; ++op) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            switch (op) {
            case 0: k_probe_pipe<0><<<kProbeBlocks, kProbeThreads>>>(out, 3); break;
            case 1: k_probe_pipe<1><<<kProbeBlocks, kProbeThreads>>>(out, 3); break;
            case 2: k_probe_pipe<2><<<kProbeBlocks, kProbeThreads>>>(out, 3); break;
            case 3: k_probe_pipe<3><<<kProbeBlocks, kProbeThreads>>>(out, 0x123456789abcdefull); break;
            default: k_probe_pipe<4><<<kProbeBlocks, kProbeThreads>>>(out, 3); break;
            }
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // first repetition warms up
        }
        lanes_per_clk_sm[op] = ops / (best * 1e-3) / ((double)sms * khz * 1e3);
    }
    const bool bad = cudaGetLastError() != cudaSuccess;
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return bad ? fail(KS_ECUDA, "ks_probe_int_pipes: kernel failed") : KS_OK;
}

extern "C" int ks_probe_alu(int iters, double *bfly_per_s, double *mac_per_s)
{
    if (iters < 1 || !bfly_per_s || !mac_per_s) return fail(KS_EINVAL, "ks_probe_alu: bad argument");
    u64 *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = KS_OK;
    if (cudaMalloc((void **)&out, sizeof(u64) * kProbeBlocks * kProbeThreads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(KS_ECUDA, "ks_probe_alu: setup failed");
    }
    const u64 q = 18014398509309953ull;  // a 54-bit odd modulus; the values are irrelevant to the rate
    const u64 w = 1234567890123ull;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == KS_OK; ++rep) {  // first repetition warms up
        cudaEventRecord(e0);
        k_probe_bfly<<<kProbeBlocks, kProbeThreads>>>(out, q, w, wp, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        *bfly_per_s = (double)kProbeBlocks * kProbeThreads * iters * 16 / (ms * 1e-3);
        cudaEventRecord(e0);
        k_probe_bmac<<<kProbeBlocks, kProbeThreads>>>(out, 0x0abcdef01234567ull, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        *mac_per_s = (double)kProbeBlocks * kProbeThreads * iters * 8 / (ms * 1e-3);
    }
    if (rc == KS_OK && cudaGetLastError() != cudaSuccess) rc = fail(KS_ECUDA, "ks_probe_alu: kernel failed");
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

extern "C" int ks_probe_inv_bfly(int iters, double *inv_bfly_per_s)
{
    if (iters < 1 || !inv_bfly_per_s) return fail(KS_EINVAL, "ks_probe_inv_bfly: bad argument");
    u64 *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = KS_OK;
    if (cudaMalloc((void **)&out, sizeof(u64) * kProbeBlocks * kProbeThreads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(KS_ECUDA, "ks_probe_inv_bfly: setup failed");
    }
    const u64 q = 18014398509309953ull;
    const u64 w = 1234567890123ull;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == KS_OK; ++rep) {  // first repetition warms up
        cudaEventRecord(e0);
        k_probe_ibfly<<<kProbeBlocks, kProbeThreads>>>(out, q, w, wp, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        *inv_bfly_per_s = (double)kProbeBlocks * kProbeThreads * iters * 16 / (ms * 1e-3);
    }
    if (rc == KS_OK && cudaGetLastError() != cudaSuccess) rc = fail(KS_ECUDA, "ks_probe_inv_bfly: kernel failed");
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
