// noalloc.cu -- render_score_batch for callers that cannot allocate device memory.
//
// render_score_batch needs a small scratch workspace that its caller
// allocates.  Some callers cannot do that: code running inside a host that owns
// every device allocation (a plugin or an engine with its own memory budget),
// real-time loops whose rules forbid allocating after start-up, and library
// layers with no access to the application's allocator.
// render_score_batch_noalloc serves them: its scratch is a fixed array in this
// library's own device memory, so the caller passes only inputs and outputs.
//
// The array is a file-scope __device__ symbol of HS_NOALLOC_SCRATCH_BYTES
// bytes.  Host code cannot use the symbol's name as a device address, so the
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached.  With lazy module loading (the CUDA default)
// that lookup is also when the driver loads this file's module on the device
// and reserves the array, so the first call on each device is the one that
// can fail for lack of memory (HS_ERR_CUDA): make it at start-up, before any
// stream capture or allocation-free phase.  The device then holds the array
// until the process exits, and later calls allocate nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/handscore.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// device address of the scratch array on the current device (first call: look it up)
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HS_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HS_OK;
}

}  // namespace

extern "C" int render_score_batch_noalloc(const HsModel* model, const HsObs* obs, const HsCamera* cam,
                                          const HsPrim* prims, const float* kc, int P, const HsScoreParams* params,
                                          float* E, HsParts* parts, hs_stream_t stream)
{
    // every argument but P is checked first, by a call that launches nothing
    // (P = 0), so that errors come in the same order as render_score_batch's
    int rc = render_score_batch(model, obs, cam, prims, kc, 0, params, nullptr, 0, E, parts, nullptr, nullptr, stream);
    if (rc != HS_OK) return rc;
    size_t need = 0;
    if ((rc = hs_workspace_size(P, &need)) != HS_OK) return rc;      // P out of range
    if (need > (size_t)HS_NOALLOC_SCRATCH_BYTES) return HS_ERR_SIZE;  // P beyond what the fixed array holds
    if (P == 0) return HS_OK;
    void* scratch = nullptr;
    if ((rc = scratch_address(&scratch)) != HS_OK) return rc;
    // the array keeps whatever the last call left in it: start from zeros
    if (cudaMemsetAsync(scratch, 0, need, (cudaStream_t)stream) != cudaSuccess) return HS_ERR_CUDA;
    return render_score_batch(model, obs, cam, prims, kc, P, params, scratch, need, E, parts, nullptr, nullptr,
                              stream);
}
