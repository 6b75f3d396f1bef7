// hs_device.cuh -- device-side definitions shared by the handscore kernels.
//
// The validated hand model travels to the kernels by value (a launch
// parameter in the constant bank), so the library keeps no device copy of it.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/handscore.h"

namespace hs {

constexpr int kNdof = HS_NDOF;
constexpr int kMaxBones = HS_MAX_BONES;
constexpr int kMaxPrims = HS_MAX_PRIMS;
constexpr float kEllipsoidMarker = 2.0f;  // HsPrim.m[13] value that marks an ellipsoid

constexpr int kMaxChain = HS_MAX_DEPTH + 1;  // bones on a path from the palm
struct DevBone {
    int32_t parent, dof_z, dof_x, depth;  // depth in the tree (palm = 0)
    float off[3];
    float rest[9];                        // row-major Rz Ry Rx of the rest angles
    int8_t anc[kMaxChain];                // anc[k]: its ancestor at depth k (anc[depth] = the bone)
};

struct DevPrimDesc {
    int32_t bone, kind;
    float center[3];
    float dims[4];
    float inv_s[3];  // 1 / scale along local x, y, z
    int32_t caps;    // cone caps to render: bit 0 at y = -hl, bit 1 at y = +hl
    int32_t pad;     // (a whole number of 8-byte words)
};

// a collision proxy of the interpenetration test: an inscribed sphere of a
// primitive, centre in its bone's frame
struct DevProxy {
    float local[3];
    float radius;
    int32_t bone, finger;  // finger: the palm's child bone on the path to the palm (numbered), -1 on the palm
    int32_t fixed;         // centred at the origin of a bone attached to the palm: never moves relative to it
};
constexpr int kMaxProxies = HS_MAX_PROXIES;
constexpr int kMaxPairs = HS_MAX_PROXY_PAIRS;

// what every FK kernel copies to shared memory: header, limits, primitives, bones (about 5.6 KB)
struct alignas(8) DevModelCore {  // (8-aligned: kernels copy it in 8-byte words)
    int32_t n_bones, n_prims, max_depth, pad;
    int32_t kc_variant, n_proxies;  // HS_KC_*; proxies used by the penetration test
    float pen_weight;
    int32_t n_pairs;                // the pairs of proxies it tests (on different fingers, not both fixed)
    float lo[kNdof], hi[kNdof];
    DevPrimDesc prims[kMaxPrims];  // kernels copy the used prefix of prims and bones
    DevBone bones[kMaxBones];
};

// everything the FK kernels need about the model; it travels by value as a
// launch parameter, and the collision data of the penetration test stays
// there (read only when a kc variant needs it)
struct DevModel : DevModelCore {
    DevProxy proxies[kMaxProxies];
    uint16_t pairs[kMaxPairs];      // proxy i in the low byte, j in the high byte
};

struct Limits {
    float lo[kNdof], hi[kNdof];
};

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// U[0,1) from the top 24 bits (exact in float)
__device__ __forceinline__ float u01(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

// Random-number streams of the swarm (counter word 1 = stream << 16 | block)
constexpr uint32_t kStreamPso = 1, kStreamMutate = 2, kStreamInit = 3;

// ---- fast PTX arithmetic (documented approximate instructions) --------------
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Programmatic dependent launch: let the next kernel in the stream start its
// launch now; wait until the previous kernel has completed and its writes are
// visible (both are no-ops when the launch was not programmatic)
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Let `kernel` take up to `bytes` of dynamic shared memory on the current device
// (the default limit is 48 KB with the static part).  Once per (call site,
// device); safe from several host threads.
template <class Kernel>
inline cudaError_t opt_in_dynamic_smem(Kernel kernel, int bytes, std::atomic<uint32_t> (&done)[64])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[dev].store(1u, std::memory_order_release);
    return e;
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bit)
{
    if (status) atomicOr(status, bit);
}

// pack/unpack an inclusive int16 pixel box into two float-sized words
__device__ __forceinline__ float pack_i16x2(int a, int b)
{
    const uint32_t w = (uint32_t)(uint16_t)(int16_t)a | ((uint32_t)(uint16_t)(int16_t)b << 16);
    return __uint_as_float(w);
}
__device__ __forceinline__ int lo_i16(float w) { return (int)(int16_t)(__float_as_uint(w) & 0xFFFFu); }
__device__ __forceinline__ int hi_i16(float w) { return (int)(int16_t)(__float_as_uint(w) >> 16); }

}  // namespace hs
