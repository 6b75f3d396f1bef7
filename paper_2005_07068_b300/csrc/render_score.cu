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
//  * each CTA turns the particle's 64-byte primitive records into raster
//    records in shared memory (the ray-quadric discriminant as a polynomial in
//    the pixel offsets, and what the roots need: make_raster);
//  * a unit's observation (16x4 depth + skin) arrives by a 2-D TMA load into
//    one of the warp's two shared-memory stages, issued one unit ahead (one
//    shared copy of O, never replicated);
//  * the warp culls the primitives against each 8x4 half of the unit
//    (warp-uniform masks) and skips the unit when nothing can render there;
//    otherwise every lane tests its two pixels (one per half) against each
//    primitive with the discriminant polynomial (five FMAs) and solves for
//    the root only where it is not negative (FP32, in scaled local
//    coordinates relative to the primitive's centre depth t0, so the
//    quadratic keeps its precision at ~500 mm);
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
#include "hs_units.cuh"

namespace hs {

constexpr int kWarps = 4;  // warps per CTA; they share one staged copy of the records

struct RenderShared {
    float4 rast[kMaxPrims * kRastVec];  // raster records of the particle's primitives
    int2 pbox[kMaxPrims];        // their pixel boxes (the packed words 14, 15 of the FK record)
    alignas(128) unsigned char tile[kWarps][kStages][kSlot];
    uint64_t bar[kWarps][kStages];
    int box[4];  // xa, v0, units per row, units
};

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

    if (lane < kStages) mbar_init(&sm.bar[warp][lane], 1);
    if (tid == 0) mbar_fence_init();
    pdl_wait();  // the primitive records and kc come from the previous kernel
    if (particle_stopped(a, p)) {
        pdl_launch_dependents();
        return;
    }
    const float4* src = a.prims + (size_t)p * a.n_prims * 4;
    stage_prims(src, a.n_prims, pv, sm.rast, sm.pbox, tid, kWarps * 32);
    if (warp == 0) unit_box(src, a.n_prims, pv.W, pv.H, lane, sm.box);
    __syncthreads();
    const float kcp = a.kc[p];

    if (sm.box[3] == 0) {  // nothing of the hand inside the ROI: E is the baseline
        pdl_launch_dependents();
        if (blockIdx.x == 0 && tid == 0) write_baseline(a, p, pv.stats, kcp);
        return;
    }

    long long acc_t = 0;
    uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
    uint32_t phases = 0u;
    // zero but in the test of the observation wait's time limit
    const uint32_t extra_tx = blockIdx.x == 0 && warp == 0 ? wk->tx_test : 0u;
    render_units_warp(sm.rast, sm.pbox, a.n_prims, sm.box, sm.tile[warp], sm.bar[warp], phases,
                      blockIdx.x * kWarps + warp, gridDim.x * kWarps, pv, a, p, lane, acc_t, acc_a, acc_o, acc_h,
                      extra_tx);

    // the next kernel may start launching once every warp is past its units (it
    // still waits for this grid to finish before it reads E)
    pdl_launch_dependents();
    // flush this warp's sums; the last warp of the particle forms E and clears the workspace
    warp_sum(acc_t, acc_a, acc_o, acc_h);
    if (lane == 0) flush_and_finish(a, p, wk, pv.stats, kcp, acc_t, acc_a, acc_o, acc_h, gridDim.x * kWarps);
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
