// render_score.cu -- fused depth render + Eq. 4-5 cost + per-particle reduction.
//
// Section III.A: each hypothesis h is projected to a depth map r_d(h, C),
// compared with the observation O = (O_s, O_d) through the match map r_m and
// reduced to D(O, h, C) (Eq. 4), then E = D + lambda_k kc(h) (Eq. 5).  The
// paper renders 64 full images with OpenGL, replicates O 64 times and sums
// with a pyramid (Section IV, steps 1-3).  Here nothing is rendered to memory:
//
//  * grid (K, P) of 4-warp CTAs: the 4K warps of particle p split p's work
//    units, 16x4-pixel blocks of its screen box (union of its primitives'
//    conservative boxes, clipped to the ROI), dealt round-robin, so dense and
//    sparse parts of the hand spread over all warps; after the prologue no
//    warp waits for another;
//  * the particle's 64-byte primitive records are staged once per CTA in
//    shared memory;
//  * a unit's observation (16x4 depth + skin) arrives by a 2-D TMA load into
//    one of the warp's two shared-memory stages, issued one unit ahead (one
//    shared copy of O, never replicated);
//  * the warp culls the primitives against each 8x4 half of the unit
//    (warp-uniform masks) and skips the unit when nothing can render there;
//    otherwise every lane casts two rays (one per half) against the
//    quadrics in scaled local coordinates (FP32, taken at the primitive's
//    centre depth t0 so the quadratic keeps its precision at ~500 mm);
//  * per-lane sums are kept in 64-bit fixed point (2^-24 mm) and integer
//    counts, so the totals do not depend on which warp took which unit: E is
//    deterministic;
//  * each warp flushes its sums with one set of atomics when the queue runs
//    dry; the last warp of the particle (exit ticket) forms E and clears the
//    particle's workspace for the next call.
//
// Pixels where nothing renders keep the particle-independent baseline (t = d_M
// on valid skin, S in the union).  Each rendered pixel therefore adds only its
// difference to that baseline, and the per-frame totals (hs_obs_prepare)
// supply the rest.
#include "hs_render.cuh"

namespace hs {

// a work unit: 16x4 pixels = two 8x4 sub-blocks; lane (lx, ly) owns pixel
// (lx, ly) of both
constexpr int kUW = 16, kUH = 4, kSub = 2;
constexpr int kSlot = 384;  // one stage: depth [4][16] (<= float32, 256 B) at 0, skin [4][16] at 256

constexpr int kWarps = 4;  // warps per CTA; they share one staged copy of the records

struct RenderShared {
    float4 prims[kMaxPrims * 4];
    alignas(128) unsigned char tile[kWarps][2][kSlot];
    uint64_t bar[kWarps][2];
    int box[4];  // xa, v0, units per row, units
};

// the sub-block masks of unit (x0, y0): bit j of m[s] = primitive j's box
// overlaps 8x4 sub-block s (s = column)
__device__ __forceinline__ void cull_unit(const RenderShared& sm, int n_prims, int lane, int x0, int y0,
                                          uint64_t m[kSub])
{
    m[0] = m[1] = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        const bool present = j < n_prims;
        int u0 = 0, v0 = 0, u1 = 0, v1 = 0;
        if (present) {
            const float4 r3 = sm.prims[4 * j + 3];
            u0 = lo_i16(r3.z);
            v0 = hi_i16(r3.z);
            u1 = lo_i16(r3.w);
            v1 = hi_i16(r3.w);
        }
        const bool row = present && v0 <= y0 + 3 && v1 >= y0;
        m[0] |= (uint64_t)__ballot_sync(0xffffffffu, row && u0 <= x0 + 7 && u1 >= x0) << (32 * h);
        m[1] |= (uint64_t)__ballot_sync(0xffffffffu, row && u0 <= x0 + 15 && u1 >= x0 + 8) << (32 * h);
    }
}

// A CTA is four warps that share the staged records and otherwise run on their
// own (no barrier after the prologue).  The warps of particle p split p's
// units round-robin; a CTA frees its SM slot as soon as its warps are done.
__global__ void __launch_bounds__(kWarps * 32, 6)
    render_score_kernel(const __grid_constant__ CUtensorMap tm_depth, const __grid_constant__ CUtensorMap tm_skin,
                        const RenderArgs a)
{
    __shared__ RenderShared sm;
    const int p = a.order ? a.order[blockIdx.y] : (int)blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    HsParticleWork* wk = a.work + p;
    // the observation, rays and stats of this particle's swarm
    const ParticleView pv = particle_view(a, p, &tm_depth, &tm_skin);
    const int W = pv.W, H = pv.H, depth_f32 = pv.depth_f32;
    const float inv_fx = pv.inv_fx, off_x = pv.off_x, inv_fy = pv.inv_fy, off_y = pv.off_y;
    const uint32_t* stats = pv.stats;
    const CUtensorMap* tmd = pv.tm_depth;
    const CUtensorMap* tms = pv.tm_skin;
    const int esz = depth_f32 ? 4 : 2;

    if (lane < 2) mbar_init(&sm.bar[warp][lane], 1);
    if (tid == 0) mbar_fence_init();
    pdl_wait();  // the primitive records and kc come from the previous kernel
    const float4* src = a.prims + (size_t)p * a.n_prims * 4;
    for (int i = tid; i < a.n_prims * 4; i += kWarps * 32) sm.prims[i] = src[i];
    // the particle's screen box, clipped to the ROI, in 16x4 units
    if (warp == 0) {
        int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
        for (int i = lane; i < a.n_prims; i += 32) {
            const float4 r3 = src[4 * i + 3];
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
            u1 = min(u1, W - 1);
            v1 = min(v1, H - 1);
            const int xa = u0 & ~15;  // TMA: the uint8 skin needs x at a multiple of 16 bytes
            const bool empty = u0 > u1 || v0 > v1;
            const int nux = empty ? 1 : (u1 + 1 - xa + kUW - 1) / kUW;
            sm.box[0] = xa;
            sm.box[1] = v0;
            sm.box[2] = nux;
            sm.box[3] = empty ? 0 : nux * ((v1 - v0 + kUH) / kUH);
        }
    }
    __syncthreads();
    const int xa = sm.box[0], v0 = sm.box[1], nux = sm.box[2], n_units = sm.box[3];
    const float kcp = a.kc[p];

    if (n_units == 0) {  // nothing of the hand inside the ROI: E is the baseline
        pdl_launch_dependents();
        if (blockIdx.x == 0 && tid == 0) write_baseline(a, p, stats, kcp);
        return;
    }

    const uint32_t tx_bytes = kUW * kUH * (uint32_t)(esz + 1);
    long long acc_t = 0;
    uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
    uint32_t phases = 0u;  // bit s: parity of stage s's next completion
    bool ok = true;
    const int lx = lane & 7, ly = lane >> 3;
    // units of this warp: u = g, g + stride, ... ; their (column, row) advance
    // without divisions
    const int stride = gridDim.x * kWarps;
    const int sx = stride % nux, sy = stride / nux;
    int u = blockIdx.x * kWarps + warp;
    int ux = u % nux, uy = u / nux;  // unit u
    int s = 0;                       // stage of unit u
    uint64_t mk[kSub];
    auto prepare = [&](int cx, int cy, int stage, uint64_t m[kSub]) {
        const int x0 = xa + kUW * cx, y0 = v0 + kUH * cy;
        cull_unit(sm, a.n_prims, lane, x0, y0, m);
        if ((m[0] | m[1]) && lane == 0) {
            unsigned char* t = sm.tile[warp][stage];
            fence_proxy_async();  // the stage's last generic reads come before the refill
            mbar_arrive_expect_tx(&sm.bar[warp][stage], tx_bytes);
            tma_load_2d(t, tmd, x0, y0, &sm.bar[warp][stage]);
            tma_load_2d(t + 256, tms, x0, y0, &sm.bar[warp][stage]);
        }
    };
    mk[0] = mk[1] = 0;
    if (u < n_units) prepare(ux, uy, 0, mk);
    while (u < n_units && ok) {
        const int un = u + stride;
        int nx = ux + sx, ny = uy + sy;
        if (nx >= nux) {
            nx -= nux;
            ++ny;
        }
        uint64_t mn[kSub] = {0, 0};
        if (un < n_units) prepare(nx, ny, s ^ 1, mn);  // look-ahead: cull and start the next tile
        const uint64_t any = mk[0] | mk[1];
        if (any) {
            const int x0 = xa + kUW * ux, y0 = v0 + kUH * uy;
            const int px0 = x0 + lx, py = y0 + ly;
            const float ra[2] = {fmaf((float)px0, inv_fx, off_x), fmaf((float)(px0 + 8), inv_fx, off_x)};
            const float rb = fmaf((float)py, inv_fy, off_y);
            // nearest hit per pixel as (t0, s): depth z = t0 + s
            float z[kSub] = {INFINITY, INFINITY}, zt[kSub] = {0.f, 0.f}, zs[kSub] = {0.f, 0.f};
            uint64_t mask = any;
            while (mask) {
                const int j = __ffsll((long long)mask) - 1;
                mask &= mask - 1;
                const float4* r = &sm.prims[4 * j];
                const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
#pragma unroll
                for (int q = 0; q < kSub; ++q) {
                    if ((mk[q] >> j) & 1) {
                        const float sh = intersect(r0, r1, r2, r3, ra[q], rb);
                        const float zz = r2.w + sh;
                        if (zz < z[q]) {
                            z[q] = zz;
                            zt[q] = r2.w;
                            zs[q] = sh;
                        }
                    }
                }
            }
            ok = mbar_wait_bounded(&sm.bar[warp][s], (phases >> s) & 1u, a.status);
            phases ^= 1u << s;
            const unsigned char* t = sm.tile[warp][s];
#pragma unroll
            for (int q = 0; q < kSub; ++q) {
                const int xr = lx + 8 * q;
                const int px = x0 + xr;
                const bool hit = ok && z[q] < INFINITY && px < W && py < H;
                if (!__any_sync(0xffffffffu, hit)) continue;  // nothing rendered in this half
                if (hit) {
                    const int oi = ly * kUW + xr;
                    const float od = depth_f32 ? reinterpret_cast<const float*>(t)[oi]
                                                 : (float)reinterpret_cast<const uint16_t*>(t)[oi];
                    const bool rm = add_pixel(od, t[256 + oi] != 0, zt[q], zs[q], a, acc_t, acc_a, acc_o, acc_h);
                    if (a.dbg_depth) {
                        const size_t o = ((size_t)p * H + py) * W + px;
                        a.dbg_depth[o] = z[q];
                        a.dbg_mask[o] = (uint8_t)(1 | (rm ? 2 : 0));
                    }
                }
            }
            __syncwarp();  // every lane is done with this stage before it is refilled
        }
        mk[0] = mn[0];
        mk[1] = mn[1];
        u = un;
        ux = nx;
        uy = ny;
        s ^= 1;
    }
    // a unit prepared but never processed (a wait timed out) leaves no copy behind
    if (!ok && u < n_units && (mk[0] | mk[1])) mbar_wait_bounded(&sm.bar[warp][s], (phases >> s) & 1u, a.status);

    // the next kernel may start launching once every warp is past its units (it
    // still waits for this grid to finish before it reads E)
    pdl_launch_dependents();
    // flush this warp's sums; the last warp of the particle forms E and clears the workspace
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_t += __shfl_xor_sync(0xffffffffu, acc_t, o);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
        acc_o += __shfl_xor_sync(0xffffffffu, acc_o, o);
        acc_h += __shfl_xor_sync(0xffffffffu, acc_h, o);
    }
    if (lane == 0) flush_and_finish(a, p, wk, stats, kcp, acc_t, acc_a, acc_o, acc_h, gridDim.x * kWarps);
}

// per-frame totals of the observation: #(skin and depth > 0), #skin
__global__ void __launch_bounds__(256) obs_stats_kernel(const unsigned char* depth, int depth_pitch, int depth_f32,
                                                        const uint8_t* skin, int skin_pitch, int W, int H,
                                                        uint32_t* stats)
{
    __shared__ uint32_t red[2][8];
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
        red[0][threadIdx.x >> 5] = nv;
        red[1][threadIdx.x >> 5] = ns;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // one atomic pair per block keeps the two counters uncontended
        uint32_t tv = 0, ts = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tv += red[0][w];
            ts += red[1][w];
        }
        atomicAdd(&stats[0], tv);
        atomicAdd(&stats[1], ts);
    }
}

// per-frame totals of every swarm of a batch: block (row group, swarm)
__global__ void __launch_bounds__(256) obs_stats_multi_kernel(const BatchDev b)
{
    __shared__ uint32_t red[2][8];
    const SwarmView& v = b.views[blockIdx.y];
    uint32_t nv = 0, ns = 0;
    for (int y = blockIdx.x; y < v.H; y += gridDim.x) {
        for (int x = threadIdx.x; x < v.W; x += blockDim.x) {
            const bool S = v.skin[(size_t)y * v.skin_pitch + x] != 0;
            const float od = v.depth_f32 ? reinterpret_cast<const float*>(v.depth + (size_t)y * v.depth_pitch)[x]
                                         : (float)reinterpret_cast<const uint16_t*>(v.depth + (size_t)y * v.depth_pitch)[x];
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
        red[0][threadIdx.x >> 5] = nv;
        red[1][threadIdx.x >> 5] = ns;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tv = 0, ts = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tv += red[0][w];
            ts += red[1][w];
        }
        atomicAdd(&v.stats[0], tv);
        atomicAdd(&v.stats[1], ts);
    }
}

cudaError_t launch_obs_stats_multi(const BatchDev& batch, int max_H, cudaStream_t stream)
{
    const int rows = max_H < 16 ? max_H : 16;
    obs_stats_multi_kernel<<<dim3(rows, batch.S), 256, 0, stream>>>(batch);
    return cudaGetLastError();
}

cudaError_t launch_render_score(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(args.K, args.P);
    cfg.blockDim = dim3(kWarps * 32);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, render_score_kernel, tm_depth, tm_skin, args);
}

cudaError_t launch_obs_stats(const unsigned char* depth, int depth_pitch, int depth_f32, const uint8_t* skin,
                             int skin_pitch, int W, int H, uint32_t* stats, cudaStream_t stream)
{
    const int blocks = H < 148 ? H : 148;
    obs_stats_kernel<<<blocks, 256, 0, stream>>>(depth, depth_pitch, depth_f32, skin, skin_pitch, W, H, stats);
    return cudaGetLastError();
}

}  // namespace hs
