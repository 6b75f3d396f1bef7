// render_score.cu -- fused depth render + Eq. 4-5 cost + per-particle reduction.
//
// Section III.A: each hypothesis h is projected to a depth map r_d(h, C),
// compared with the observation O = (O_s, O_d) through the match map r_m and
// reduced to D(O, h, C) (Eq. 4), then E = D + lambda_k kc(h) (Eq. 5).  The
// paper renders 64 full images with OpenGL, replicates O 64 times and sums
// with a pyramid (Section IV, steps 1-3).  Here nothing is rendered to memory:
//
//  * grid (K, P): CTA (k, p) walks tiles k, k+K, ... of particle p's
//    screen-space box (union of its primitives' conservative boxes);
//  * the particle's 64-byte primitive records are staged in shared memory;
//  * each 16x16 observation tile (depth + skin) arrives by a 2-D TMA load,
//    double-buffered on two mbarriers (one shared copy of O, never replicated);
//  * each warp owns an 8x4 pixel block and culls the primitives against it
//    (warp-uniform bit mask), then every lane casts its pixel's ray against
//    the surviving quadrics in scaled local coordinates (FP32, shifted to the
//    primitive's depth t0 so the quadratic keeps its precision at ~500 mm);
//  * the per-pixel terms are reduced with warp shuffles and a CTA sum;
//  * the last CTA of a particle (atomic ticket) adds the K partials in a fixed
//    order, so E is deterministic.
//
// Pixels outside the particle's box render nothing, so their contribution is
// the particle-independent baseline (t = d_M on valid skin, S in the union).
// Each processed pixel therefore adds only its difference to that baseline,
// and the per-frame totals (hs_obs_prepare) supply the rest.
#include <cuda.h>

#include <cfloat>
#include <climits>

#include "hs_args.cuh"

namespace hs {

constexpr int kTW = 16, kTH = 16, kThreads = 256;

struct __align__(128) RenderSmem {
    unsigned char depth[2][kTW * kTH * 4];  // 2 stages, up to float32
    unsigned char skin[2][kTW * kTH];
    float4 prims[kMaxPrims * 4];
    uint64_t bar[2];
    float wsum_t[kThreads / 32];
    uint32_t wsum_c[kThreads / 32];
    int box[4];
    int last;
};

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
//   cone:       X^2 + Z^2 = (1 + kappa Y)^2, |Y| <= 1, caps at Y = -1, +1
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
        // planar caps at Y = -1 (radius 1 - kappa) and Y = +1 (radius 1 + kappa)
        const float ihy = rcp_approx(hy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float yc = c ? 1.f : -1.f;
            const float s = (yc - gy) * ihy;
            const float X = fmaf(s, hx, gx), Z = fmaf(s, hz, gz);
            const float w = 1.f + yc * kap;
            if (fmaf(X, X, Z * Z) <= w * w && t0 + s > 0.f) best = fminf(best, s);
        }
    }
    return best;
}

__device__ __forceinline__ bool box_overlaps(const float4& r3, int x0, int y0, int x1, int y1)
{
    return lo_i16(r3.z) <= x1 && hi_i16(r3.z) <= y1 && lo_i16(r3.w) >= x0 && hi_i16(r3.w) >= y0;
}

__global__ void __launch_bounds__(kThreads, 4)
    render_score_kernel(const __grid_constant__ CUtensorMap tm_depth, const __grid_constant__ CUtensorMap tm_skin,
                        const RenderArgs a)
{
    __shared__ RenderSmem sm;
    const int k = blockIdx.x, p = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const float4* src = a.prims + (size_t)p * a.n_prims * 4;
    for (int i = tid; i < a.n_prims * 4; i += kThreads) sm.prims[i] = src[i];
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // the particle's screen box in tiles (union of primitive boxes, clipped to the ROI)
    if (warp == 0) {
        int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
        for (int i = lane; i < a.n_prims; i += 32) {
            const float4 r3 = sm.prims[4 * i + 3];
            u0 = min(u0, lo_i16(r3.z));
            v0 = min(v0, hi_i16(r3.z));
            u1 = max(u1, lo_i16(r3.w));
            v1 = max(v1, hi_i16(r3.w));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u0 = min(u0, __shfl_xor_sync(0xffffffffu, u0, o));
            v0 = min(v0, __shfl_xor_sync(0xffffffffu, v0, o));
            u1 = max(u1, __shfl_xor_sync(0xffffffffu, u1, o));
            v1 = max(v1, __shfl_xor_sync(0xffffffffu, v1, o));
        }
        if (lane == 0) {
            u0 = max(u0, 0);
            v0 = max(v0, 0);
            u1 = min(u1, a.W - 1);
            v1 = min(v1, a.H - 1);
            if (u0 > u1 || v0 > v1) {
                sm.box[0] = sm.box[1] = sm.box[2] = sm.box[3] = 0;
            } else {
                sm.box[0] = u0 / kTW;
                sm.box[1] = v0 / kTH;
                sm.box[2] = u1 / kTW - u0 / kTW + 1;
                sm.box[3] = v1 / kTH - v0 / kTH + 1;
            }
        }
    }
    __syncthreads();
    const int tx0 = sm.box[0], ty0 = sm.box[1], ntx = sm.box[2];
    const int n_tiles = ntx * sm.box[3];
    const uint32_t tx_bytes = kTW * kTH * (a.depth_f32 ? 4u : 2u) + kTW * kTH;

    if (tid == 0 && k < n_tiles) {
        mbar_arrive_expect_tx(&sm.bar[0], tx_bytes);
        tma_load_2d(sm.depth[0], &tm_depth, (tx0 + k % ntx) * kTW, (ty0 + k / ntx) * kTH, &sm.bar[0]);
        tma_load_2d(sm.skin[0], &tm_skin, (tx0 + k % ntx) * kTW, (ty0 + k / ntx) * kTH, &sm.bar[0]);
    }

    float acc_t = 0.f;
    uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
    int it = 0;
    for (int i = k; i < n_tiles; i += a.K, ++it) {
        const int s = it & 1;
        const int tx = tx0 + i % ntx, ty = ty0 + i / ntx;
        const int nxt = i + a.K;
        if (tid == 0 && nxt < n_tiles) {
            mbar_arrive_expect_tx(&sm.bar[s ^ 1], tx_bytes);
            tma_load_2d(sm.depth[s ^ 1], &tm_depth, (tx0 + nxt % ntx) * kTW, (ty0 + nxt / ntx) * kTH, &sm.bar[s ^ 1]);
            tma_load_2d(sm.skin[s ^ 1], &tm_skin, (tx0 + nxt % ntx) * kTW, (ty0 + nxt / ntx) * kTH, &sm.bar[s ^ 1]);
        }
        // warp-level culling: this warp's 8x4 pixel block against every primitive box
        const int wx0 = tx * kTW + (warp & 1) * 8, wy0 = ty * kTH + (warp >> 1) * 4;
        const bool c0 = lane < a.n_prims && box_overlaps(sm.prims[4 * lane + 3], wx0, wy0, wx0 + 7, wy0 + 3);
        const bool c1 =
            lane + 32 < a.n_prims && box_overlaps(sm.prims[4 * (lane + 32) + 3], wx0, wy0, wx0 + 7, wy0 + 3);
        uint64_t mask = (uint64_t)__ballot_sync(0xffffffffu, c0) | ((uint64_t)__ballot_sync(0xffffffffu, c1) << 32);

        const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
        const float ra = __fdiv_rn((float)px + 0.5f - a.cx, a.fx);
        const float rb = __fdiv_rn((float)py + 0.5f - a.cy, a.fy);
        // nearest hit: depth z = t0 + s, kept as (t0, s) so the cost can form
        // O_d - z as (O_d - t0) - s without rounding at the ~500 mm scale
        float z = INFINITY, zt0 = 0.f, zs = 0.f;
        while (mask) {
            const int j = __ffsll((long long)mask) - 1;
            mask &= mask - 1;
            const float4* r = &sm.prims[4 * j];
            const float4 r2 = r[2];
            const float s = intersect(r[0], r[1], r2, r[3], ra, rb);
            const float zz = r2.w + s;
            if (zz < z) {
                z = zz;
                zt0 = r2.w;
                zs = s;
            }
        }

        mbar_wait_bounded(&sm.bar[s], (uint32_t)(it >> 1) & 1u, a.status);
        const int li = (py - ty * kTH) * kTW + (px - tx * kTW);
        const float od = a.depth_f32 ? reinterpret_cast<const float*>(sm.depth[s])[li]
                                     : (float)reinterpret_cast<const uint16_t*>(sm.depth[s])[li];
        const bool S = sm.skin[s][li] != 0;
        const bool in_roi = px < a.W && py < a.H;
        const bool hit = z < INFINITY;
        // per-pixel terms of Eq. 4 (reading R1), as differences to the no-hit baseline
        const bool valid = S && od > 0.f;
        const float diff = fabsf((od - zt0) - zs);
        const bool rm = hit && (!valid || diff < a.d_m);
        const float t = hit ? (valid ? fminf(diff, a.d_M) : (S ? 0.f : a.d_M)) : (valid ? a.d_M : 0.f);
        float dt = t - (valid ? a.d_M : 0.f);
        uint32_t c = (uint32_t)(S && rm) | ((uint32_t)(rm && !S) << 10) | ((uint32_t)hit << 20);
        if (!in_roi) {
            dt = 0.f;
            c = 0;
        } else if (a.dbg_depth) {
            const size_t o = ((size_t)p * a.H + py) * a.W + px;
            a.dbg_depth[o] = hit ? z : 0.f;
            a.dbg_mask[o] = (uint8_t)((hit ? 1 : 0) | (rm ? 2 : 0));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dt += __shfl_xor_sync(0xffffffffu, dt, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            sm.wsum_t[warp] = dt;
            sm.wsum_c[warp] = c;
        }
        __syncthreads();
        if (tid == 0) {
            float st = 0.f;
            uint32_t sc = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                st += sm.wsum_t[w];
                sc += sm.wsum_c[w];
            }
            acc_t += st;
            acc_a += sc & 1023u;
            acc_o += (sc >> 10) & 1023u;
            acc_h += sc >> 20;
        }
        __syncthreads();
    }

    // per-CTA partial, then the last CTA of the particle finishes it
    if (tid == 0) {
        a.partials[(size_t)p * a.K + k] =
            make_float4(acc_t, __uint_as_float(acc_a), __uint_as_float(acc_o), __uint_as_float(acc_h));
        __threadfence();
        const uint32_t prev = atomicAdd(&a.counters[p], 1u);
        sm.last = prev == (uint32_t)(a.K - 1);
    }
    __syncthreads();
    if (sm.last && warp == 0) {
        __threadfence();
        float st = 0.f;
        uint32_t sa = 0, so = 0, sh = 0;
        for (int j = lane; j < a.K; j += 32) {
            const float4 v = __ldcg(&a.partials[(size_t)p * a.K + j]);
            st += v.x;
            sa += __float_as_uint(v.y);
            so += __float_as_uint(v.z);
            sh += __float_as_uint(v.w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st += __shfl_xor_sync(0xffffffffu, st, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            so += __shfl_xor_sync(0xffffffffu, so, o);
            sh += __shfl_xor_sync(0xffffffffu, sh, o);
        }
        if (lane == 0) {
            const uint32_t n_valid = __ldcg(&a.stats[0]), n_skin = __ldcg(&a.stats[1]);
            const float t_sum = st + a.d_M * (float)n_valid;
            so += n_skin;
            float D;
            if (so == 0) {
                D = a.lambda;
            } else {
                const float fa = (float)sa, fo = (float)so;
                D = t_sum / fo + a.lambda * (1.f - 2.f * fa / (fa + fo));
            }
            a.E[p] = D + a.lambda_k * a.kc[p];
            if (a.parts) a.parts[p] = HsParts{t_sum, sa, so, sh};
            a.counters[p] = 0;
        }
    }
}

// per-frame totals of the observation: #(skin and depth > 0), #skin
__global__ void __launch_bounds__(256) obs_stats_kernel(const unsigned char* depth, int depth_pitch, int depth_f32,
                                                        const uint8_t* skin, int skin_pitch, int W, int H,
                                                        uint32_t* stats)
{
    uint32_t nv = 0, ns = 0;
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        for (int x = threadIdx.x; x < W; x += blockDim.x) {
            const bool S = skin[(size_t)y * skin_pitch + x] != 0;
            const float od = depth_f32 ? reinterpret_cast<const float*>(depth + (size_t)y * depth_pitch)[x]
                                       : (float)reinterpret_cast<const uint16_t*>(depth + (size_t)y * depth_pitch)[x];
            ns += S;
            nv += S && od > 0.f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[0], nv);
        atomicAdd(&stats[1], ns);
    }
}

cudaError_t launch_render_score(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                cudaStream_t stream)
{
    dim3 grid(args.K, args.P);
    render_score_kernel<<<grid, kThreads, 0, stream>>>(tm_depth, tm_skin, args);
    return cudaGetLastError();
}

cudaError_t launch_obs_stats(const unsigned char* depth, int depth_pitch, int depth_f32, const uint8_t* skin,
                             int skin_pitch, int W, int H, uint32_t* stats, cudaStream_t stream)
{
    const int blocks = H < 296 ? H : 296;
    obs_stats_kernel<<<blocks, 256, 0, stream>>>(depth, depth_pitch, depth_f32, skin, skin_pitch, W, H, stats);
    return cudaGetLastError();
}

}  // namespace hs
