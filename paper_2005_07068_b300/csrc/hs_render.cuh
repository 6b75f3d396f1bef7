// hs_render.cuh -- pieces shared by the two render + cost kernels: TMA and
// mbarrier helpers, the ray-quadric intersection, the per-pixel Eq. 4 terms and
// the per-particle finish (Eq. 4-5 from the integer sums).
#pragma once
#include <cuda.h>

#include <cfloat>
#include <climits>

#include "hs_args.cuh"

namespace hs {

constexpr float kFix = 16777216.0f;     // fixed-point scale of the depth sums (2^24 per mm)

// ---- mbarrier / TMA (inline PTX) ---------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// orders this thread's earlier generic-proxy accesses of shared memory before
// the async-proxy (TMA) writes it issues next
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// bounded wait: returns false (and flags the status word) if the phase never completes
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status)
{
    for (uint32_t spin = 0; spin < (1u << 22); ++spin)
        if (mbar_try_wait(bar, parity)) return true;
    set_status(status, HS_DEV_TMA_TIMEOUT);
    return false;
}

// ---- ray / quadric ----------------------------------------------------------------
// Nearest hit of pixel direction d = (a, b, 1) with one primitive, as the depth
// offset s from the primitive's centre depth t0 = C_z (depth = t0 + s), or +inf.
// In scaled local coordinates the ray is g + s h with h = M d and
// g = M (t0 d - C) = M (t0 a - C_x, t0 b - C_y, 0):
//   ellipsoid:  |p|^2 = 1
//   cone:       X^2 + Z^2 = (1 + kappa Y)^2, |Y| <= 1, and the caps at Y = -1, +1
//               that the model leaves visible (record word 12)
__device__ __forceinline__ float intersect(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                          float a, float b)
{
    const float t0 = r2.w, kap = r3.y;
    const float hx = fmaf(a, r0.x, fmaf(b, r0.w, r1.z));
    const float hy = fmaf(a, r0.y, fmaf(b, r1.x, r1.w));
    const float hz = fmaf(a, r0.z, fmaf(b, r1.y, r2.x));
    const float ex = fmaf(t0, a, -r2.y), ey = fmaf(t0, b, -r2.z);
    const float gx = fmaf(ex, r0.x, ey * r0.w);
    const float gy = fmaf(ex, r0.y, ey * r1.x);
    const float gz = fmaf(ex, r0.z, ey * r1.y);
    float best = INFINITY;
    if (kap > 1.5f) {
        const float A = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
        const float B = fmaf(gx, hx, fmaf(gy, hy, gz * hz));
        const float C = fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, -1.f)));
        const float disc = fmaf(B, B, -A * C);
        if (disc >= 0.f) {
            const float sq = sqrt_approx(disc);
            const float ia = rcp_approx(A);
            const float sn = (-B - sq) * ia;
            const float sf = (-B + sq) * ia;
            best = t0 + sn > 0.f ? sn : (t0 + sf > 0.f ? sf : INFINITY);
        }
    } else {
        const float w0 = fmaf(kap, gy, 1.f), w1 = kap * hy;
        const float A = fmaf(hx, hx, fmaf(hz, hz, -w1 * w1));
        const float B = fmaf(gx, hx, fmaf(gz, hz, -w0 * w1));
        const float C = fmaf(gx, gx, fmaf(gz, gz, -w0 * w0));
        const float disc = fmaf(B, B, -A * C);
        if (disc >= 0.f) {
            const float sq = sqrt_approx(disc);
            const float qq = -(B + copysignf(sq, B));
            const float s1 = qq * rcp_approx(A);
            const float s2 = C * rcp_approx(qq);
            const float y1 = fmaf(s1, hy, gy), y2 = fmaf(s2, hy, gy);
            if (fabsf(y1) <= 1.f && t0 + s1 > 0.f) best = fminf(best, s1);
            if (fabsf(y2) <= 1.f && t0 + s2 > 0.f) best = fminf(best, s2);
        }
        const uint32_t caps = __float_as_uint(r3.x);
        if (caps) {  // planar caps at Y = -1 (radius 1 - kappa) and Y = +1 (radius 1 + kappa)
            const float ihy = rcp_approx(hy);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!(caps & (1u << c))) continue;
                const float yc = c ? 1.f : -1.f;
                const float s = (yc - gy) * ihy;
                const float X = fmaf(s, hx, gx), Z = fmaf(s, hz, gz);
                const float w = 1.f + yc * kap;
                if (fmaf(X, X, Z * Z) <= w * w && t0 + s > 0.f) best = fminf(best, s);
            }
        }
    }
    return best;
}

// per-pixel terms of Eq. 4 (reading R1) as differences to the no-hit baseline,
// added to the lane's fixed-point / integer sums; returns r_m.  The rendered
// depth is zt0 + zs, split so that O_d - zt0 is exact (both ~500 mm) and the
// small part zs is subtracted after.
__device__ __forceinline__ bool add_pixel(float od, bool S, float zt0, float zs, const RenderArgs& a, long long& at,
                                          uint32_t& aa, uint32_t& ao, uint32_t& ah)
{
    const bool valid = S && od > 0.f;
    const float diff = fabsf((od - zt0) - zs);  // O_d - z without rounding at the ~500 mm scale
    const bool rm = !valid || diff < a.d_m;
    const float t = valid ? fminf(diff, a.d_M) : (S ? 0.f : a.d_M);
    // |t - d_M| <= d_M < 128 mm, so the 2^-24 mm fixed-point term fits in 32 bits;
    // the sum is carried in a 64-bit integer (integer adds, order independent)
    at += (long long)__float2int_rn((t - (valid ? a.d_M : 0.f)) * kFix);
    aa += (S && rm);
    ao += (rm && !S);
    ah += 1;
    return rm;
}

// the observation, rays and totals a particle is scored against: the call's own
// (one swarm) or those of the particle's swarm in a batch
struct ParticleView {
    int W, H, depth_f32;
    float inv_fx, off_x, inv_fy, off_y;
    const uint32_t* stats;
    const CUtensorMap* tm_depth;
    const CUtensorMap* tm_skin;
};

__device__ __forceinline__ ParticleView particle_view(const RenderArgs& a, int p, const CUtensorMap* tmd,
                                                      const CUtensorMap* tms)
{
    ParticleView v{a.W, a.H, a.depth_f32, a.inv_fx, a.off_x, a.inv_fy, a.off_y, a.stats, tmd, tms};
    if (a.batch.views) {
        const SwarmView& s = a.batch.views[a.batch.sid[p]];
        v = ParticleView{s.W, s.H, s.depth_f32, s.inv_fx, s.off_x, s.inv_fy, s.off_y, s.stats, &s.tm_depth,
                         &s.tm_skin};
    }
    return v;
}

// E of a particle none of whose primitives reaches the ROI: every pixel keeps
// the no-hit baseline
__device__ __forceinline__ void write_baseline(const RenderArgs& a, int p, const uint32_t* stats, float kcp)
{
    const uint32_t n_valid = stats[0], n_skin = stats[1];
    const float t_sum = a.d_M * (float)n_valid;
    const float D = n_skin == 0 ? a.lambda : t_sum / (float)n_skin + a.lambda;
    a.E[p] = D + a.lambda_k * kcp;
    if (a.parts) a.parts[p] = HsParts{t_sum, 0u, n_skin, 0u};
}

// Add one contributor's sums to particle p's workspace and take an exit ticket;
// the last of `contributors` forms E (Eq. 4-5) and clears the workspace.
__device__ __forceinline__ void flush_and_finish(const RenderArgs& a, int p, HsParticleWork* wk,
                                                 const uint32_t* stats, float kcp, long long acc_t, uint32_t acc_a,
                                                 uint32_t acc_o, uint32_t acc_h, uint32_t contributors)
{
    if (acc_t) atomicAdd(&wk->t_fix, (unsigned long long)acc_t);
    if (acc_a) atomicAdd(&wk->n_and, acc_a);
    if (acc_o) atomicAdd(&wk->n_or, acc_o);
    if (acc_h) atomicAdd(&wk->n_hit, acc_h);
    // release: the sums above are visible to whoever sees this ticket;
    // acquire: the last contributor sees every other one's sums
    uint32_t done;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(done) : "l"(&wk->exited) : "memory");
    if (done != contributors - 1) return;
    const long long tf = (long long)atomicAdd(&wk->t_fix, 0ull);
    const uint32_t sa = atomicAdd(&wk->n_and, 0u), so_d = atomicAdd(&wk->n_or, 0u);
    const uint32_t sh = atomicAdd(&wk->n_hit, 0u);
    const uint32_t n_valid = stats[0], n_skin = stats[1];
    // fixed point -> float from the two 32-bit halves (no 64-bit conversion)
    const float t_fix_f = (float)(int)(tf >> 32) * 4294967296.0f + (float)(uint32_t)(tf & 0xffffffffu);
    const float t_sum = t_fix_f * (1.0f / kFix) + a.d_M * (float)n_valid;
    const uint32_t so = so_d + n_skin;
    float D;
    if (so == 0) {
        D = a.lambda;
    } else {
        const float fa = (float)sa, fo = (float)so;
        D = t_sum / fo + a.lambda * (1.f - 2.f * fa / (fa + fo));
    }
    a.E[p] = D + a.lambda_k * kcp;
    if (a.parts) a.parts[p] = HsParts{t_sum, sa, so, sh};
    *wk = HsParticleWork{};  // every contributor is done: safe to clear
}

}  // namespace hs
