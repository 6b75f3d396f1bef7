// hs_units.cuh -- the pixel-major render + Eq. 4 terms of one particle, shared
// by the unit kernel (render_score_kernel) and the persistent frame kernel
// (track_frame_kernel), so that both give the same nearest hit, the same
// integer sums and hence the same E.
//
//  * stage_prims: the particle's FK records become raster records (the
//    ray-quadric discriminant as a polynomial in the pixel offsets, and what
//    the roots need) plus pixel boxes, in shared memory;
//  * unit_box: the particle's screen box (union of its primitives' boxes,
//    clipped to the ROI) cut into 16x4-pixel work units;
//  * render_units_warp: one warp's units u = first, first + stride, ...  For
//    each unit the warp culls the primitives against each 8x4 half (ballots),
//    starts the TMA load of the next unit's observation (16x4 depth + skin)
//    into its other shared-memory stage, tests its two pixels per lane against
//    every remaining primitive with the discriminant polynomial, solves for
//    the root only when some lane can be hit, and adds the Eq. 4 terms of the
//    rendered pixels (reading R1) to the lane's fixed-point / integer sums.
//    Nearest hit: the smallest float depth.
#pragma once

#include "hs_render.cuh"

namespace hs {

// a work unit: 16x4 pixels = two 8x4 sub-blocks; lane (lx, ly) owns pixel
// (lx, ly) of both
constexpr int kUW = 16, kUH = 4, kSub = 2;
constexpr int kSlot = 384;    // one stage: depth [4][16] (<= float32, 256 B) at 0, skin [4][16] at 256
constexpr int kStages = 4;    // observation stages per warp: loads run kStages - 1 units ahead

// raster record + pixel box of primitives j = tid, tid + nthreads, ... from the
// 64-byte FK records rec (global or shared memory)
__device__ __forceinline__ void stage_prims(const float4* rec, int n_prims, const ParticleView& pv, float4* rast,
                                            int2* pbox, int tid, int nthreads)
{
    for (int j = tid; j < n_prims; j += nthreads) {
        store_raster(make_raster(rec + 4 * j, pv.inv_fx, pv.off_x, pv.inv_fy, pv.off_y), rast + kRastVec * j);
        const float4 r3 = rec[4 * j + 3];
        pbox[j] = make_int2(__float_as_int(r3.z), __float_as_int(r3.w));
    }
}

// the particle's pixel box (u0, v0)-(u1, v1) clipped to the ROI, in 16x4
// units: box = (xa, v0, units per row, units); xa is a multiple of 16 (TMA:
// the uint8 skin needs x at a multiple of 16 bytes); 0 units when nothing is
// in the ROI
__device__ __forceinline__ void unit_box_clip(int u0, int v0, int u1, int v1, int W, int H, int* box)
{
    u0 = max(u0, 0);
    v0 = max(v0, 0);
    u1 = min(u1, W - 1);
    v1 = min(v1, H - 1);
    const int xa = u0 & ~15;
    const bool empty = u0 > u1 || v0 > v1;
    const int nux = empty ? 1 : (u1 + 1 - xa + kUW - 1) / kUW;
    box[0] = xa;
    box[1] = v0;
    box[2] = nux;
    box[3] = empty ? 0 : nux * ((v1 - v0 + kUH) / kUH);
}

// one warp: the union of the primitives' pixel boxes, clipped (unit_box_clip)
__device__ __forceinline__ void unit_box(const float4* rec, int n_prims, int W, int H, int lane, int* box)
{
    int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
    for (int i = lane; i < n_prims; i += 32) {
        const float4 r3 = rec[4 * i + 3];
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
    if (lane == 0) unit_box_clip(u0, v0, u1, v1, W, H, box);
}

// the sub-block masks of unit (x0, y0): bit j of m[s] = primitive j's box
// overlaps 8x4 sub-block s (s = column)
__device__ __forceinline__ void cull_unit(const int2* pbox, int n_prims, int lane, int x0, int y0, uint64_t m[kSub])
{
    m[0] = m[1] = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        const bool present = j < n_prims;
        int u0 = 0, v0 = 0, u1 = 0, v1 = 0;
        if (present) {
            const int2 bx = pbox[j];
            u0 = lo_i16(__int_as_float(bx.x));
            v0 = hi_i16(__int_as_float(bx.x));
            u1 = lo_i16(__int_as_float(bx.y));
            v1 = hi_i16(__int_as_float(bx.y));
        }
        const bool row = present && v0 <= y0 + 3 && v1 >= y0;
        m[0] |= (uint64_t)__ballot_sync(0xffffffffu, row && u0 <= x0 + 7 && u1 >= x0) << (32 * h);
        m[1] |= (uint64_t)__ballot_sync(0xffffffffu, row && u0 <= x0 + 15 && u1 >= x0 + 8) << (32 * h);
    }
}

// One warp's units u = first, first + stride, ... of particle p (box from
// unit_box).  tile: the warp's kStages stages [kStages][kSlot] (128-byte
// aligned); bar: their mbarriers; phases: bit s = parity of stage s's next
// completion (kept by the caller across calls).  The observation of the
// warp's k-th unit goes to stage k % kStages, issued kStages - 1 units ahead,
// so that the L2 latency of the loads hides behind the units in between.
// Adds the rendered pixels' Eq. 4 terms to the lane's sums.  Returns false if
// an observation load did not arrive in time (status flagged; the warp's
// remaining units are skipped and no copy is left in flight).  extra_tx: zero,
// except in the test of that time limit (bytes the first load is armed for
// beyond those copied).  kFrontRoots: primitives in front of the camera take
// the shorter roots (same bits; the batch frame kernel, at 64 registers, keeps
// the general roots only, which spill less there).
template <bool kFrontRoots = true>
__device__ __forceinline__ bool render_units_warp(const float4* rast, const int2* pbox, int n_prims, const int* box,
                                                  unsigned char (*tile)[kSlot], uint64_t* bar, uint32_t& phases,
                                                  int first, int stride, const ParticleView& pv, const RenderArgs& a,
                                                  int p, int lane, long long& acc_t, uint32_t& acc_a,
                                                  uint32_t& acc_o, uint32_t& acc_h, uint32_t extra_tx = 0u)
{
    const int xa = box[0], v0 = box[1], nux = box[2], n_units = box[3];
    if (first >= n_units) return true;
    const int n_k = (n_units - first + stride - 1) / stride;  // units of this warp
    const int W = pv.W, H = pv.H, depth_f32 = pv.depth_f32;
    const uint32_t tx_bytes = kUW * kUH * (uint32_t)((depth_f32 ? 4 : 2) + 1);
    const int lx = lane & 7, ly = lane >> 3;
    // the warp's units advance in (column, row) without divisions: one cursor
    // for the loads in flight, one for the unit being rendered
    const int sx = stride % nux, sy = stride / nux;
    int ix = first % nux, iy = first / nux;  // unit of the next load
    int ux = ix, uy = iy;                    // unit being rendered
    auto advance = [&](int& cx, int& cy) {
        cx += sx;
        cy += sy;
        if (cx >= nux) {
            cx -= nux;
            ++cy;
        }
    };
    int issued = 0;
    auto issue = [&]() {  // the observation of the warp's unit number `issued`
        const int st = issued % kStages;
        if (lane == 0) {
            const int x0 = xa + kUW * ix, y0 = v0 + kUH * iy;
            fence_proxy_async();  // the stage's last generic reads come before the refill
            mbar_arrive_expect_tx(&bar[st], tx_bytes + (issued == 0 ? extra_tx : 0u));
            tma_load_2d(tile[st], pv.tm_depth, x0, y0, &bar[st]);
            tma_load_2d(tile[st] + 256, pv.tm_skin, x0, y0, &bar[st]);
        }
        advance(ix, iy);
        ++issued;
    };
    while (issued < n_k && issued < kStages - 1) issue();
    bool ok = true;
    int k = 0;
    for (; k < n_k && ok; ++k) {
        if (issued < n_k) issue();  // refills the stage the previous unit used (released by its __syncwarp)
        const int st = k % kStages;
        const int x0 = xa + kUW * ux, y0 = v0 + kUH * uy;
        uint64_t mk[kSub];
        cull_unit(pbox, n_prims, lane, x0, y0, mk);
        const uint64_t any = mk[0] | mk[1];
        const int px0 = x0 + lx, py = y0 + ly;
        // nearest depth per pixel
        float z[kSub] = {INFINITY, INFINITY};
        if (any) {
            const float fpx0 = (float)px0, fpx1 = (float)(px0 + 8), fpy = (float)py;
            // the primitive mask as two 32-bit words; the roots of each half only
            // when some lane of that half can be hit
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const uint32_t a0 = (uint32_t)(mk[0] >> (32 * w)), a1 = (uint32_t)(mk[1] >> (32 * w));
                uint32_t mask = a0 | a1;
                while (mask) {
                    const int b = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4* R = rast + kRastVec * (b + 32 * w);
                    const bool in0 = (a0 >> b) & 1u, in1 = (a1 >> b) & 1u;  // warp-uniform
                    const float4 q0 = R[0], q1 = R[1];
                    const float dv = fpy - q0.y;
                    const float2 du = __fadd2_rn(make_float2(fpx0, fpx1), f2(-q0.x));
                    const float2 d = raster_disc2(q0, q1, du, f2(dv));  // both halves' pixels
                    const float du0 = du.x, du1 = du.y, d0 = d.x, d1 = d.y;
                    const bool caps = __float_as_uint(R[4].w) != 0u;
                    const uint32_t v0 = __ballot_sync(0xffffffffu, in0 && (d0 >= 0.f || caps));
                    const uint32_t v1 = __ballot_sync(0xffffffffu, in1 && (d1 >= 0.f || caps));
                    if (v0 | v1) {
                        // the roots of both halves' pixels at once (packed FP32), kept
                        // where some lane of the half can be hit
                        const float4 q2 = R[2], q3 = R[3], q4 = R[4];
                        const float t0 = q2.w;
                        const Ray2 r = raster_ray2(q2, q3, q4, make_float2(du0, du1), f2(dv));
                        const float2 disc = make_float2(d0, d1);
                        // in front of the camera (warp-uniform): no far root, no depth tests
                        const bool front =
                            kFrontRoots && raster_in_front(lo_i16(__int_as_float(pbox[b + 32 * w].x)));
                        float2 sh;
                        if (q3.w > 1.5f && front) {
                            const float2 sn = raster_near_ellipsoid2_front(r, disc);
                            sh = make_float2(d0 >= 0.f ? sn.x : INFINITY, d1 >= 0.f ? sn.y : INFINITY);
                        } else {
                            const uint32_t capw = __float_as_uint(q4.w);
                            sh = q3.w > 1.5f ? raster_root_ellipsoid2(t0, r, disc)
                                 : front     ? raster_root_cone2_front(q3.w, capw, r, disc)
                                             : raster_root_cone2(t0, q3.w, capw, r, disc);
                        }
                        const float2 zz = __fadd2_rn(f2(t0), sh);
                        if (v0) z[0] = fminf(z[0], zz.x);
                        if (v1) z[1] = fminf(z[1], zz.y);
                    }
                }
            }
        }
        ok = mbar_wait_bounded(&bar[st], (phases >> st) & 1u, a.status);
        phases ^= 1u << st;
        const unsigned char* t = tile[st];
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
                const bool rm = add_pixel(od, t[256 + oi] != 0, z[q], a, acc_t, acc_a, acc_o, acc_h);
                if (a.dbg_depth) {
                    const size_t o = ((size_t)p * H + py) * W + px;
                    a.dbg_depth[o] = z[q];
                    a.dbg_mask[o] = (uint8_t)(1 | (rm ? 2 : 0));
                }
            }
        }
        __syncwarp();  // every lane is done with this stage before it is refilled
        advance(ux, uy);
    }
    // loads issued for units never rendered (a wait timed out) leave no copy behind
    for (; k < issued; ++k) {
        const int st = k % kStages;
        mbar_wait_bounded(&bar[st], (phases >> st) & 1u, a.status);
        phases ^= 1u << st;
    }
    return ok;
}

// a warp's sums to lane 0
__device__ __forceinline__ void warp_sum(long long& acc_t, uint32_t& acc_a, uint32_t& acc_o, uint32_t& acc_h)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_t += __shfl_xor_sync(0xffffffffu, acc_t, o);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
        acc_o += __shfl_xor_sync(0xffffffffu, acc_o, o);
        acc_h += __shfl_xor_sync(0xffffffffu, acc_h, o);
    }
}

}  // namespace hs
