// render_strips.cu -- render + Eq. 4-5 cost by pixel strips (the strip kernel),
// the third layout of the same computation as render_score_kernel and the
// tile kernels (Section III.A: depth map r_d of hypothesis h, match map r_m,
// D of Eq. 4, E = D + lambda_k kc of Eq. 5).
//
//  * grid (K, P) of 4-warp CTAs; the particle's screen box (union of its
//    primitives' boxes, clipped to the ROI) is cut into strips 8 pixels wide
//    and SH rows tall, dealt round-robin to the 4K warps of the particle; a
//    warp renders its strips on its own (no CTA barrier after the prologue);
//  * a lane owns one column of the strip and one row of every 4-row step
//    (8 x 4 pixels per step, SH / 4 steps), and keeps the nearest hit of its
//    SH / 4 pixels in registers;
//  * per strip, the primitives whose box meets it are culled with two
//    ballots; for each of them every lane forms the du terms of its column's
//    discriminant polynomial once (Poly2Col), the coverage of all the steps of
//    the primitive's rows is one straight-line block (two FMAs per step, one
//    sign bit each; two steps per packed FP32 instruction), and the roots are
//    solved two steps at a time (raster_root_*2) where some lane of either
//    step can be hit -- the unit kernel's arithmetic lane by lane, so the
//    nearest depth is bit-identical to its;
//  * the strip's observation (16-pixel-wide 2-D TMA boxes, one per 4-row
//    band, the skin needs 16-byte rows) is loaded into one of the warp's two
//    shared-memory buffers while the previous strip renders;
//  * the rendered pixels add their Eq. 4 terms (reading R1) to the lane's
//    fixed-point / integer sums (add_pixel), and the last warp of the particle
//    forms E (flush_and_finish).
#include <atomic>

#include "hs_units.cuh"

namespace hs {

constexpr int kStripWarps = 4;
constexpr int kStripW = 8;  // strip width in pixels (a lane's column)

template <int SH>
struct StripShared {
    static constexpr int kBands = SH / 4;
    float4 rast[kMaxPrims * kRastVec];
    int2 pbox[kMaxPrims];
    // per warp, two buffers of kBands 16 x 4 boxes (depth at 0, skin at 256 of each slot)
    alignas(128) unsigned char obs[kStripWarps][2][kBands][kSlot];
    uint64_t bar[kStripWarps][2];
    int box[4];  // xa, v0, u1, v1 of the clipped box (u1 < 0: empty)
};

// primitives whose pixel box meets columns [x0, x0 + 7] and rows [y0, y1]: bit j
__device__ __forceinline__ uint64_t cull_strip(const int2* pbox, int n_prims, int lane, int x0, int y0, int y1)
{
    uint64_t m = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        bool in = false;
        if (j < n_prims) {
            const int2 bx = pbox[j];
            in = lo_i16(__int_as_float(bx.x)) <= x0 + kStripW - 1 && lo_i16(__int_as_float(bx.y)) >= x0 &&
                 hi_i16(__int_as_float(bx.x)) <= y1 && hi_i16(__int_as_float(bx.y)) >= y0;
        }
        m |= (uint64_t)__ballot_sync(0xffffffffu, in) << (32 * h);
    }
    return m;
}

// resident CTAs per SM the register budget is set for (80 registers a thread)
template <int SH>
constexpr int strip_min_ctas() { return 6; }

// The CTA's copy of particle p's raster records and pixel boxes, and p's
// screen box clipped to the ROI (sm.box: xa, v0, u1, v1; u1 < 0 when nothing
// is in the ROI).  Ends with a CTA barrier.
template <int SH>
__device__ __forceinline__ void strip_stage(StripShared<SH>& sm, const RenderArgs& a, int p, const ParticleView& pv,
                                            int tid, int lane, int warp)
{
    const int n_prims = a.n_prims;
    const float4* src = a.prims + (size_t)p * n_prims * 4;
    stage_prims(src, n_prims, pv, sm.rast, sm.pbox, tid, kStripWarps * 32);
    if (warp == 0) {
        int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
        for (int i = lane; i < n_prims; i += 32) {
            const float4 r3 = src[4 * i + 3];
            u0 = min(u0, lo_i16(r3.z));
            v0 = min(v0, hi_i16(r3.z));
            u1 = max(u1, lo_i16(r3.w));
            v1 = max(v1, hi_i16(r3.w));
        }
        u0 = __reduce_min_sync(0xffffffffu, u0);
        v0 = __reduce_min_sync(0xffffffffu, v0);
        u1 = __reduce_max_sync(0xffffffffu, u1);
        v1 = __reduce_max_sync(0xffffffffu, v1);
        if (lane == 0) {
            u0 = max(u0, 0);
            v0 = max(v0, 0);
            u1 = min(u1, pv.W - 1);
            v1 = min(v1, pv.H - 1);
            const bool empty = u0 > u1 || v0 > v1;
            sm.box[0] = u0 & ~15;  // TMA: the uint8 skin needs x at a multiple of 16 bytes
            sm.box[1] = v0;
            sm.box[2] = empty ? -1 : u1;
            sm.box[3] = v1;
        }
    }
    __syncthreads();
}

// One warp's strips q = first, first + stride, ... of particle p (staged by
// strip_stage): their render and Eq. 4 terms, added to the lane's sums.
// phases (bit b = parity of buffer b's next completion) and buf (the buffer
// the next load goes to) carry over from one call to the next.  extra_tx:
// zero, except in the test of the observation wait's time limit.  Returns
// false if an observation load did not arrive in time (status flagged; the
// warp's remaining strips are skipped and no copy is left in flight).
template <int SH>
__device__ __forceinline__ bool render_strips_warp(StripShared<SH>& sm, const RenderArgs& a, int p,
                                                   const ParticleView& pv, int lane, int warp, int first, int stride,
                                                   uint32_t extra_tx, uint32_t& phases, int& buf, long long& acc_t,
                                                   uint32_t& acc_a, uint32_t& acc_o, uint32_t& acc_h)
{
    constexpr int kSteps = SH / 4;
    const int n_prims = a.n_prims;
    const int xa = sm.box[0], by0 = sm.box[1], bx1 = sm.box[2], by1 = sm.box[3];
    const int nsx = (bx1 + 1 - xa + kStripW - 1) / kStripW;
    const int n_strips = nsx * ((by1 + 1 - by0 + SH - 1) / SH);
    const int W = pv.W, H = pv.H, depth_f32 = pv.depth_f32;
    const int lx = lane & 7, ly = lane >> 3;
    uint64_t* bar = sm.bar[warp];

    // the observation of strip (sx, sy) into buffer b: one 16 x 4 box of depth
    // and of skin per band of rows inside the box, issued by one lane each
    auto issue = [&](int sx, int sy, int b) {
        const int x16 = (xa + kStripW * sx) & ~15, y0 = by0 + SH * sy;
        const int nb = (min(y0 + SH - 1, by1) - y0) / 4 + 1;
        if (lane == 0) {
            fence_proxy_async();  // the buffer's last generic reads come before the refill
            mbar_arrive_expect_tx(&bar[b], (uint32_t)nb * 64u * (uint32_t)((depth_f32 ? 4 : 2) + 1) + extra_tx);
        }
        extra_tx = 0u;
        __syncwarp();
        if (lane < nb) {
            tma_load_2d(sm.obs[warp][b][lane], pv.tm_depth, x16, y0 + 4 * lane, &bar[b]);
            tma_load_2d(sm.obs[warp][b][lane] + 256, pv.tm_skin, x16, y0 + 4 * lane, &bar[b]);
        }
    };

    // strip q is (q mod nsx, q div nsx); the warp's strips advance by `stride`
    // without a division per strip: one cursor for the strip rendered, one for
    // the strip whose observation is loaded next
    const int ssy = stride / nsx, ssx = stride - ssy * nsx;
    auto advance = [&](int& cx, int& cy) {
        cx += ssx;
        cy += ssy;
        if (cx >= nsx) {
            cx -= nsx;
            ++cy;
        }
    };
    int sx = first % nsx, sy = first / nsx;  // the strip being rendered
    int nx = sx, ny = sy;                    // the strip after it
    advance(nx, ny);
    bool ok = true;
    int q = first;
    bool next_issued = false;  // the load of strip q + stride is in flight in buffer buf ^ 1
    if (first < n_strips) issue(sx, sy, buf);
    for (; q < n_strips; q += stride, buf ^= 1) {
        next_issued = q + stride < n_strips;
        if (next_issued) issue(nx, ny, buf ^ 1);  // the next strip's observation meanwhile
        const int x0 = xa + kStripW * sx, y0 = by0 + SH * sy;
        const int y1 = min(y0 + SH - 1, by1);
        // per pixel of the lane: the nearest depth so far
        float z[kSteps];
#pragma unroll
        for (int s = 0; s < kSteps; ++s) z[s] = INFINITY;
        const float fx = (float)(x0 + lx), fy0 = (float)(y0 + ly);
        uint64_t mask = cull_strip(sm.pbox, n_prims, lane, x0, y0, y1);
        while (mask) {  // warp-uniform walk over the strip's primitives, in index order
            const int j = __ffsll((long long)mask) - 1;
            mask &= mask - 1;
            const float4* R = sm.rast + kRastVec * j;
            const int2 pb = sm.pbox[j];
            const int s0 = (max(hi_i16(__int_as_float(pb.x)), y0) - y0) >> 2;
            const int s1 = (min(hi_i16(__int_as_float(pb.y)), y1) - y0) >> 2;
            const float4 q0 = R[0], q1 = R[1];
            const float du = fx - q0.x;
            const bool caps = __float_as_uint(R[4].w) != 0u;
            const Poly2Col PD = raster_disc_col(q0, q1, du);
            // coverage of every step of the primitive's rows at once
            // (independent polynomials, one sign bit each, no branch per step;
            // the polynomial is never -0, so a clear sign bit is disc >= 0, and
            // a NaN only costs roots that return +inf)
            // (two steps per packed FP32 instruction)
            const float2 nqy = f2(-q0.y), vv2 = f2(PD.vv), u12 = f2(PD.u1), u02 = f2(PD.u0);
            uint32_t neg = 0u;
#pragma unroll
            for (int s = 0; s < kSteps; s += 2) {
                const float2 dv = __fadd2_rn(make_float2(fy0 + (float)(4 * s), fy0 + (float)(4 * s + 4)), nqy);
                const float2 d = __ffma2_rn(dv, __ffma2_rn(dv, vv2, u12), u02);  // PD.at of both steps
                neg |= ((__float_as_uint(d.x) >> 31) << s) | ((__float_as_uint(d.y) >> 31) << (s + 1));
            }
            const uint32_t m = (caps ? ~0u : ~neg) & ((2u << s1) - (1u << s0));  // within the primitive's rows
            const uint32_t wm = __reduce_or_sync(0xffffffffu, m);  // steps some lane can hit
            if (!wm) continue;
            // the roots, two steps at a time (packed FP32) where some lane of either
            // step can be hit; the nearest depth per pixel
            const float4 q2 = R[2], q3 = R[3], q4 = R[4];
            const float t0 = q2.w;
            auto take2 = [&](int s, float2 sh) {
                const float2 zz = __fadd2_rn(f2(t0), sh);
                z[s] = fminf(z[s], ((m >> s) & 1u) ? zz.x : INFINITY);
                z[s + 1] = fminf(z[s + 1], ((m >> (s + 1)) & 1u) ? zz.y : INFINITY);
            };
            // a primitive in front of the camera (warp-uniform; all of them unless
            // one reaches the plane z = 1 mm) skips the far root and the depth tests
            const bool front = raster_in_front(lo_i16(__int_as_float(pb.x)));
            if (q3.w > 1.5f) {  // ellipsoid (warp-uniform)
                if (front) {
#pragma unroll
                    for (int s = 0; s < kSteps; s += 2) {
                        if (!((wm >> s) & 3u)) continue;  // no lane can be hit in either step (warp-uniform)
                        const float2 dv =
                            __fadd2_rn(make_float2(fy0 + (float)(4 * s), fy0 + (float)(4 * s + 4)), nqy);
                        const float2 disc = __ffma2_rn(dv, __ffma2_rn(dv, vv2, u12), u02);
                        const float2 sn = raster_near_ellipsoid2_front(raster_ray2(q2, q3, q4, f2(du), dv), disc);
                        const float2 sh = make_float2(((m >> s) & 1u) ? sn.x : INFINITY,
                                                      ((m >> (s + 1)) & 1u) ? sn.y : INFINITY);
                        const float2 zz = __fadd2_rn(f2(t0), sh);
                        z[s] = fminf(z[s], zz.x);
                        z[s + 1] = fminf(z[s + 1], zz.y);
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < kSteps; s += 2) {
                        if (!((wm >> s) & 3u)) continue;
                        const float2 dv =
                            __fadd2_rn(make_float2(fy0 + (float)(4 * s), fy0 + (float)(4 * s + 4)), nqy);
                        const float2 disc = __ffma2_rn(dv, __ffma2_rn(dv, vv2, u12), u02);
                        take2(s, raster_root_ellipsoid2(t0, raster_ray2(q2, q3, q4, f2(du), dv), disc));
                    }
                }
            } else {
                const float kap = q3.w;
                const uint32_t capw = __float_as_uint(q4.w);
                if (front) {
#pragma unroll
                    for (int s = 0; s < kSteps; s += 2) {
                        if (!((wm >> s) & 3u)) continue;
                        const float2 dv =
                            __fadd2_rn(make_float2(fy0 + (float)(4 * s), fy0 + (float)(4 * s + 4)), nqy);
                        const float2 disc = __ffma2_rn(dv, __ffma2_rn(dv, vv2, u12), u02);
                        take2(s, raster_root_cone2_front(kap, capw, raster_ray2(q2, q3, q4, f2(du), dv), disc));
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < kSteps; s += 2) {
                        if (!((wm >> s) & 3u)) continue;
                        const float2 dv =
                            __fadd2_rn(make_float2(fy0 + (float)(4 * s), fy0 + (float)(4 * s + 4)), nqy);
                        const float2 disc = __ffma2_rn(dv, __ffma2_rn(dv, vv2, u12), u02);
                        take2(s, raster_root_cone2(t0, kap, capw, raster_ray2(q2, q3, q4, f2(du), dv), disc));
                    }
                }
            }
        }
        ok = mbar_wait_bounded(&bar[buf], (phases >> buf) & 1u, a.status);
        phases ^= 1u << buf;
        if (!ok) break;
        {
            const int px = x0 + lx, c = (x0 & 15) + lx;  // column inside the 16-wide boxes
#pragma unroll
            for (int s = 0; s < kSteps; ++s) {
                const int py = y0 + 4 * s + ly;
                const bool hit = z[s] < INFINITY && px < W && py < H;
                if (!__any_sync(0xffffffffu, hit)) continue;  // nothing rendered in this step
                if (hit) {
                    const unsigned char* t = sm.obs[warp][buf][s];
                    const int oi = ly * 16 + c;
                    const float od = depth_f32 ? reinterpret_cast<const float*>(t)[oi]
                                               : (float)reinterpret_cast<const uint16_t*>(t)[oi];
                    const bool rm = add_pixel(od, t[256 + oi] != 0, z[s], a, acc_t, acc_a, acc_o, acc_h);
                    if (a.dbg_depth) {
                        const size_t o = ((size_t)p * H + py) * W + px;
                        a.dbg_depth[o] = z[s];
                        a.dbg_mask[o] = (uint8_t)(1 | (rm ? 2 : 0));
                    }
                }
            }
        }
        __syncwarp();  // every lane is done with this buffer before it is refilled
        sx = nx;
        sy = ny;
        advance(nx, ny);
    }
    if (!ok) {
        // the copies still expected -- the late one and the next strip's, if
        // issued -- are awaited (bounded) so that none is in flight when the
        // CTA leaves
        mbar_wait_bounded(&bar[buf], ((phases >> buf) & 1u) ^ 1u, a.status);
        if (next_issued) mbar_wait_bounded(&bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u, a.status);
    }
    return ok;
}

// Grid (K, P): CTA k of particle p takes p's strips k, k + K, ... (per warp:
// 4k + w, 4k + w + 4K, ...); the last warp of the particle forms E.
template <int SH>
__global__ void __launch_bounds__(kStripWarps * 32, strip_min_ctas<SH>())
    render_strips_kernel(const __grid_constant__ CUtensorMap tm_depth, const __grid_constant__ CUtensorMap tm_skin,
                         const RenderArgs a)
{
    __shared__ StripShared<SH> sm;
    const int p = a.order ? a.order[blockIdx.y] : (int)blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    HsParticleWork* wk = a.work + p;
    const ParticleView pv = particle_view(a, p, &tm_depth, &tm_skin);

    if (lane < 2) mbar_init(&sm.bar[warp][lane], 1);
    if (tid == 0) mbar_fence_init();
    pdl_wait();  // the primitive records and kc come from the previous kernel
    if (particle_stopped(a, p)) {
        pdl_launch_dependents();
        return;
    }
    strip_stage(sm, a, p, pv, tid, lane, warp);
    const float kcp = a.kc[p];
    if (sm.box[2] < 0) {  // nothing of the hand inside the ROI: E is the baseline
        pdl_launch_dependents();
        if (blockIdx.x == 0 && tid == 0) write_baseline(a, p, pv.stats, kcp);
        return;
    }
    long long acc_t = 0;
    uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
    uint32_t phases = 0u;
    int buf = 0;
    // zero but in the test of the observation wait's time limit (bytes the
    // particle's first load is armed for beyond those copied)
    const uint32_t extra_tx = blockIdx.x == 0 && warp == 0 ? wk->tx_test : 0u;
    render_strips_warp(sm, a, p, pv, lane, warp, blockIdx.x * kStripWarps + warp, gridDim.x * kStripWarps, extra_tx,
                       phases, buf, acc_t, acc_a, acc_o, acc_h);
    pdl_launch_dependents();
    warp_sum(acc_t, acc_a, acc_o, acc_h);
    if (lane == 0) flush_and_finish(a, p, wk, pv.stats, kcp, acc_t, acc_a, acc_o, acc_h, gridDim.x * kStripWarps);
}

// The persistent form (Section IV's parallelism between particles, dealt at
// run time): as many CTAs as the GPU keeps resident, each taking the next
// particle (of any swarm of a batch, in the call's order: largest ROI first)
// from a counter in the workspace's control block, rendering all of its
// strips with its four warps, forming its E, and taking the next, until
// every particle is done.  The last CTA to leave returns the counters to
// zero for the next call.
template <int SH>
__global__ void __launch_bounds__(kStripWarps * 32, strip_min_ctas<SH>())
    render_strips_persistent_kernel(const __grid_constant__ CUtensorMap tm_depth,
                                    const __grid_constant__ CUtensorMap tm_skin, const RenderArgs a)
{
    __shared__ StripShared<SH> sm;
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    RenderCtl* ctl = a.ctl;

    if (lane < 2) mbar_init(&sm.bar[warp][lane], 1);
    if (tid == 0) mbar_fence_init();
    pdl_wait();  // the primitive records and kc come from the previous kernel
    uint32_t phases = 0u;
    int buf = 0;
    bool alive = true;  // false once one of this warp's observation waits ran out (status flagged): the warp
                        // renders nothing more in this launch, and the call's results are void
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&ctl->next, 1u);
        __syncthreads();  // also: every warp is done with the previous particle's records
        const int item = s_item;
        if (item >= a.P) break;
        const int p = a.order ? a.order[item] : item;
        if (particle_stopped(a, p)) continue;
        HsParticleWork* wk = a.work + p;
        const ParticleView pv = particle_view(a, p, &tm_depth, &tm_skin);
        strip_stage(sm, a, p, pv, tid, lane, warp);
        const float kcp = a.kc[p];
        if (sm.box[2] < 0) {  // nothing of the hand inside the ROI: E is the baseline
            if (tid == 0) write_baseline(a, p, pv.stats, kcp);
            continue;
        }
        long long acc_t = 0;
        uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
        const uint32_t extra_tx = warp == 0 ? wk->tx_test : 0u;
        if (alive)
            alive = render_strips_warp(sm, a, p, pv, lane, warp, warp, kStripWarps, extra_tx, phases, buf, acc_t,
                                       acc_a, acc_o, acc_h);
        warp_sum(acc_t, acc_a, acc_o, acc_h);
        if (lane == 0) flush_and_finish(a, p, wk, pv.stats, kcp, acc_t, acc_a, acc_o, acc_h, kStripWarps);
    }
    pdl_launch_dependents();
    if (tid == 0) {
        // the last CTA to leave: every CTA has taken its last ticket, so the
        // counters can return to zero for the next call
        uint32_t done;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(done) : "l"(&ctl->exited) : "memory");
        if (done == gridDim.x - 1) {
            ctl->next = 0u;
            ctl->exited = 0u;
        }
    }
}

template <int SH>
static cudaError_t launch_strips(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                 bool persistent, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kStripWarps * 32);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!persistent) {
        cfg.gridDim = dim3(args.K, args.P);
        return cudaLaunchKernelEx(&cfg, render_strips_kernel<SH>, tm_depth, tm_skin, args);
    }
    // one CTA per resident slot of the device, at most one per particle
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_strips_persistent_kernel<SH>,
                                                          kStripWarps * 32, 0);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    cfg.gridDim = dim3((unsigned)(slots < args.P ? slots : args.P));
    return cudaLaunchKernelEx(&cfg, render_strips_persistent_kernel<SH>, tm_depth, tm_skin, args);
}

cudaError_t launch_render_strips(int variant, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                                 const RenderArgs& args, cudaStream_t stream)
{
    switch (variant) {
    case HS_RENDER_STRIPS_8x16: return launch_strips<16>(tm_depth, tm_skin, args, false, stream);
    case HS_RENDER_STRIPS_8x32: return launch_strips<32>(tm_depth, tm_skin, args, false, stream);
    case HS_RENDER_PERSISTENT_8x16: return launch_strips<16>(tm_depth, tm_skin, args, true, stream);
    case HS_RENDER_PERSISTENT_8x32: return launch_strips<32>(tm_depth, tm_skin, args, true, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hs
