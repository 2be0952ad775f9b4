// ks_noalloc.cu -- key switch that allocates nothing.
//
// Some callers cannot allocate device memory once they are running: a
// serving process whose device memory is entirely reserved by its own pool
// allocator (a third-party cudaMalloc would fail or fragment the pool), or a
// latency-critical loop where cudaMalloc/cudaFree would synchronise the
// device and stall every other stream.  ks_switch allocates its scratch on
// first use per stream, so it does not suit them.  ks_switch_noalloc runs
// the same Output-Centric key switch with its scratch in one file-scope
// device array of fixed size, reserved when the library's device code is
// loaded and held by every GPU that loads it until the process exits.
#include <map>
#include <mutex>

#include "ks_internal.h"
#include "ks_launch.h"

namespace ks {

// 4 Mi words = 32 MiB of scratch.
constexpr size_t kNoAllocScratchWords = (size_t)4 << 20;

static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchWords];

// Device address of the scratch array, looked up once per device.  In host
// code the array's name is only a host-side stand-in; its device address
// must come from cudaGetSymbolAddress, called with the device current.
static std::mutex g_noalloc_mu;
static std::map<int, u64 *> g_noalloc_addr;

static int noalloc_scratch(int device, u64 **out)
{
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    auto it = g_noalloc_addr.find(device);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return KS_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return fail(KS_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
                                  cudaGetErrorString(e));
    }
    g_noalloc_addr[device] = (u64 *)p;
    *out = (u64 *)p;
    return KS_OK;
}

// Scratch words the Output-Centric schedule needs at level nact: y (nact
// limbs), the section temporaries (nd*(nact+K) + 2*nact limbs, nd the active
// digits) and c' (2*(nact+K) limbs), each limb N words.  The layout is the
// one oc_job builds for ks_switch, so the check below and the kernels' writes
// agree by construction.
static size_t noalloc_words(const ks_params *P, int nact) { return oc_scratch_words(P->tables, nact); }

}  // namespace ks

using namespace ks;

extern "C" size_t ks_switch_noalloc_max_words(void) { return kNoAllocScratchWords; }

extern "C" int ks_switch_noalloc(const ks_params *P, const ks_key *K, uint32_t level_towers, const uint64_t *d_in,
                                 uint64_t *d_out0, uint64_t *d_out1, ks_stream_t stream)
{
    if (!P) return fail(KS_EINVAL, "params is NULL");
    // the same argument checks as ks_switch: level range, NULL pointers,
    // 16-byte alignment (the combine kernels move two words at a time) and
    // overlapping buffers, all before anything is launched
    int rc = check_job(P, K, level_towers, d_in, d_out0, d_out1);
    if (rc != KS_OK) return rc;
    const int nact = (int)level_towers;
    const size_t need = noalloc_words(P, nact);
    if (need > kNoAllocScratchWords)
        return fail(KS_EINVAL, "ks_switch_noalloc: this parameter set and level need " + std::to_string(need) +
                                   " scratch words, the static buffer holds " +
                                   std::to_string(kNoAllocScratchWords) + " (32 MiB); use ks_switch");
    if (cudaSetDevice(P->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(KS_ECUDA, "cudaSetDevice failed");
    }
    u64 *base = nullptr;
    if ((rc = noalloc_scratch(P->device, &base)) != KS_OK) return rc;
    // Every scratch word the schedule reads is written earlier in the same
    // call, so nothing needs clearing between calls.
    const OcJob J = oc_job(P, K, nact, d_in, d_out0, d_out1, base);
    // the default schedule's variant and engines, as ks_switch applies them
    // with KS_OC (so both calls run the same kernels)
    return launch_oc(call_tables(P, P->sched), 1, &J, P->sched.oc_variant, (cudaStream_t)stream);
}
