// render_tiles.cu -- render + Eq. 4-5 cost organised by primitive (the tile
// renderer), the alternative to the pixel-major unit kernel.
//
// Same result as render_score_kernel (Section III.A: depth map of hypothesis
// h, match map r_m, D of Eq. 4, E of Eq. 5), different order of work:
//
//  * grid (K, P) of CTAs; CTA k of particle p takes tiles k, k + K, ... of
//    p's screen box (union of its primitives' boxes, clipped to the ROI) cut
//    into TW x TH tiles;
//  * per tile, the primitives whose box meets the tile are listed with the
//    exact rectangle box ∩ tile; the rectangles are cut into 32-pixel chunks
//    and the warps deal the chunks round-robin, so each lane tests exactly one
//    pixel of one primitive per step (pixel-exact culling, the primitive's
//    raster record held in registers while its chunks last): the discriminant
//    polynomial decides coverage, the roots are solved only on a hit;
//  * hits go to a z-buffer in shared memory with atomicMin on the bits of the
//    depth z = t0 + s (positive floats order as their bit patterns, so the
//    nearest surface wins whatever the order of the updates);
//  * meanwhile the tile's observation (depth + skin) arrives by TMA; a second
//    pass visits the tile's rendered pixels and adds their Eq. 4 terms to
//    integer sums;
//  * one set of atomics per CTA, and the last CTA of the particle forms E.
#include <atomic>

#include "hs_units.cuh"

namespace hs {

constexpr uint32_t kEmptyKey = 0x7f800000u;  // +inf: no hit
constexpr int kMaxDevices = 64;

__host__ __device__ constexpr int tile_align16(int x) { return (x + 15) / 16 * 16; }

// byte offsets of the dynamic shared memory of a TW x TH tile of a CTA of NW
// warps: the tile's buffers, then arrays sized for the model's n primitives
template <int TW, int TH, int NW>
struct TileLayout {
    static constexpr int kBoxes = (TW / 16) * (TH / 4);  // 16 x 4 TMA boxes per tile
    static constexpr int kDepth = 0;                      // box b at b * 256 (16 x 4 x <= 4 bytes)
    static constexpr int kSkin = kDepth + kBoxes * 256;   // box b at b * 128 (16 x 4 bytes)
    static constexpr int kZ = kSkin + kBoxes * 128;       // u32 [TH][TW]: depth bits
    static constexpr int kRast = kZ + TW * TH * 4;        // float4 [n][kRastVec]: raster records
    int pbox, rect, magic, pre, list, red, bar, box, bytes;
    __host__ __device__ explicit TileLayout(int n)
    {
        pbox = kRast + n * 16 * kRastVec;   // int2 [n]: packed pixel boxes
        rect = tile_align16(pbox + n * 8);  // int4 [n]: x0, y0, w, pixels
        magic = rect + n * 16;              // u32 [n]: ~2^31 / w, rounded up
        pre = tile_align16(magic + n * 4);  // int [n + 1]: first chunk of each entry
        list = tile_align16(pre + (n + 1) * 4);  // int [n]: primitive of each entry
        red = tile_align16(list + n * 4);   // per-warp sums: i64 [NW], then u32 [NW][3]
        bar = tile_align16(red + 20 * NW);  // mbarrier
        box = bar + 16;                     // int [8]
        bytes = box + 32;
    }
    static_assert(TW % 16 == 0 && TH % 4 == 0, "tiles are made of 16 x 4 TMA boxes");
    static_assert((TW & (TW - 1)) == 0, "TW is a power of two");
    static_assert(kDepth % 128 == 0 && kSkin % 128 == 0, "TMA destinations are 128-byte aligned");
};

// 64 registers: eight CTAs of four warps per SM (the arrays sized for the
// model, not for kMaxPrims, leave the shared memory for them)
template <int TW, int TH, int NW>
__global__ void __launch_bounds__(NW * 32, 32 / NW)
    render_tiles_kernel(const __grid_constant__ CUtensorMap tm_depth, const __grid_constant__ CUtensorMap tm_skin,
                        const RenderArgs a)
{
    using Lay = TileLayout<TW, TH, NW>;
    const Lay L(a.n_prims);
    extern __shared__ __align__(128) unsigned char smem[];
    float4* s_rast = reinterpret_cast<float4*>(smem + Lay::kRast);
    int2* s_pbox = reinterpret_cast<int2*>(smem + L.pbox);
    uint32_t* s_z = reinterpret_cast<uint32_t*>(smem + Lay::kZ);
    unsigned char* s_depth = smem + Lay::kDepth;
    unsigned char* s_skin = smem + Lay::kSkin;
    int4* s_rect = reinterpret_cast<int4*>(smem + L.rect);
    uint32_t* s_magic = reinterpret_cast<uint32_t*>(smem + L.magic);
    int* s_pre = reinterpret_cast<int*>(smem + L.pre);
    int* s_list = reinterpret_cast<int*>(smem + L.list);
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    int* s_box = reinterpret_cast<int*>(smem + L.box);

    const int p = a.order ? a.order[blockIdx.y] : (int)blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    HsParticleWork* wk = a.work + p;
    const ParticleView pv = particle_view(a, p, &tm_depth, &tm_skin);
    const uint32_t esz = pv.depth_f32 ? 4u : 2u;

    if (tid == 0) {
        mbar_init(s_bar, 1);
        mbar_fence_init();
    }
    pdl_wait();  // the primitive records and kc come from the previous kernel
    if (particle_stopped(a, p)) {
        pdl_launch_dependents();
        return;
    }
    const int n_prims = a.n_prims;
    const float4* src = a.prims + (size_t)p * n_prims * 4;
    stage_prims(src, n_prims, pv, s_rast, s_pbox, tid, NW * 32);  // raster form of each primitive, once per CTA
    if (warp == 0) {  // the particle's screen box, clipped to the ROI
        int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
        for (int i = lane; i < n_prims; i += 32) {
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
            u1 = min(u1, pv.W - 1);
            v1 = min(v1, pv.H - 1);
            const bool empty = u0 > u1 || v0 > v1;
            s_box[0] = u0 & ~15;  // TMA: the uint8 skin needs x at a multiple of 16 bytes
            s_box[1] = v0;
            s_box[2] = empty ? -1 : u1;
            s_box[3] = v1;
        }
    }
    __syncthreads();
    const int xa = s_box[0], by0 = s_box[1], bx1 = s_box[2], by1 = s_box[3];
    const float kcp = a.kc[p];
    if (bx1 < 0) {  // nothing of the hand inside the ROI: E is the baseline
        pdl_launch_dependents();
        if (blockIdx.x == 0 && tid == 0) write_baseline(a, p, pv.stats, kcp);
        return;
    }
    const int ntx = (bx1 + 1 - xa + TW - 1) / TW;
    const int ntiles = ntx * ((by1 + 1 - by0 + TH - 1) / TH);

    long long acc_t = 0;
    uint32_t acc_a = 0, acc_o = 0, acc_h = 0;
    uint32_t phase = 0;
    bool ok = true;
    // zero but in the test of the observation wait's time limit (bytes the
    // particle's first tile load is armed for beyond those copied)
    uint32_t extra_tx = blockIdx.x == 0 ? wk->tx_test : 0u;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int ty = t / ntx, tx = t - ty * ntx;
        const int tx0 = xa + tx * TW, ty0 = by0 + ty * TH;
        const int cx1 = min(tx0 + TW - 1, bx1), cy1 = min(ty0 + TH - 1, by1);
        if (warp == 0) {
            // the tile's observation: the 16 x 4 boxes that meet the clipped tile
            // (each starts inside the ROI), issued by the lanes of warp 0
            const int nbx = (cx1 - tx0) / 16 + 1, nby = (cy1 - ty0) / 4 + 1;
            if (lane == 0) {
                fence_proxy_async();  // the last tile's generic reads come before these writes
                mbar_arrive_expect_tx(s_bar, (uint32_t)(nbx * nby) * 64u * (esz + 1u) + extra_tx);
            }
            __syncwarp();
            for (int b = lane; b < nbx * nby; b += 32) {
                const int byy = b / nbx, bx = b - byy * nbx;
                const int slot = byy * (TW / 16) + bx;
                tma_load_2d(s_depth + slot * 256, pv.tm_depth, tx0 + 16 * bx, ty0 + 4 * byy, s_bar);
                tma_load_2d(s_skin + slot * 128, pv.tm_skin, tx0 + 16 * bx, ty0 + 4 * byy, s_bar);
            }
            // the primitives whose box meets the clipped tile: rectangle, divisor, chunk prefix
            int count = 0, chunks = 0;
            for (int h = 0; h < (n_prims + 31) / 32; ++h) {
                const int j = lane + 32 * h;
                int rx0 = 0, ry0 = 0, rw = 0, n = 0;
                if (j < n_prims) {
                    const int2 bx = s_pbox[j];
                    rx0 = max(lo_i16(__int_as_float(bx.x)), tx0);
                    ry0 = max(hi_i16(__int_as_float(bx.x)), ty0);
                    const int rx1 = min(lo_i16(__int_as_float(bx.y)), cx1);
                    const int ry1 = min(hi_i16(__int_as_float(bx.y)), cy1);
                    if (rx1 >= rx0 && ry1 >= ry0) {
                        rw = rx1 - rx0 + 1;
                        n = rw * (ry1 - ry0 + 1);
                    }
                }
                const uint32_t in = __ballot_sync(0xffffffffu, n > 0);
                const int ch = (n + 31) >> 5;
                int incl = ch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (n > 0) {
                    const int slot = count + __popc(in & ((1u << lane) - 1u));
                    s_list[slot] = j;
                    s_rect[slot] = make_int4(rx0, ry0, rw, n);
                    // y = (idx * m) >> 31 is floor(idx / w) for every m in
                    // [2^31 / w, (2^31 + 2^18) / w) when idx < 2^13: the float
                    // quotient is within 128 of 2^31 / w, so +256 lands inside
                    s_magic[slot] = __float2uint_rd(2147483648.0f / (float)rw) + 256u;
                    s_pre[slot] = chunks + incl - ch;
                }
                chunks += __shfl_sync(0xffffffffu, incl, 31);
                count += __popc(in);
            }
            if (lane == 0) {
                s_pre[count] = chunks;
                s_box[4] = count;
            }
        }
        const int rows = cy1 - ty0 + 1;  // rows of the tile inside the particle's box
        for (int i = tid; i < TW * rows / 4; i += NW * 32)
            reinterpret_cast<uint4*>(s_z)[i] = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
        __syncthreads();

        // raster: chunk c of the tile's list goes to warp c mod NW
        const int total = s_pre[s_box[4]];
        int k = 0;
        for (int c = warp; c < total;) {
            while (c >= s_pre[k + 1]) ++k;  // warp-uniform walk along the list
            const int j = s_list[k];
            const int4 rc = s_rect[k];
            const uint32_t mg = s_magic[k];
            const int c0 = s_pre[k], c1 = s_pre[k + 1];
            const float4* R = s_rast + kRastVec * j;
            const float4 q0 = R[0], q1 = R[1], q2 = R[2], q3 = R[3], q4 = R[4];  // in registers for the chunks
            const bool front = raster_in_front(lo_i16(__int_as_float(s_pbox[j].x)));
            for (; c < c1; c += NW) {
                const int idx = ((c - c0) << 5) + lane;
                if (idx < rc.w) {
                    const int y = (int)(((unsigned long long)(uint32_t)idx * mg) >> 31);
                    const int px = rc.x + idx - y * rc.z, py = rc.y + y;
                    const float du = (float)px - q0.x, dv = (float)py - q0.y;
                    const float disc = raster_disc(q0, q1, du, dv);
                    const float zz = raster_maybe(q4, disc) ? raster_hit_z(q2, q3, q4, du, dv, disc, front) : INFINITY;
                    if (zz < INFINITY) atomicMin(&s_z[(py - ty0) * TW + (px - tx0)], __float_as_uint(zz));
                }
            }
        }
        extra_tx = 0u;
        ok = __syncthreads_and(mbar_wait_bounded(s_bar, phase, a.status));
        if (!ok) break;
        phase ^= 1u;

        // cost: every rendered pixel of the tile against the observation
        for (int i = tid; i < TW * rows; i += NW * 32) {
            const uint32_t key = s_z[i];
            if (key == kEmptyKey) continue;
            const float z = __uint_as_float(key);
            const int ly = i / TW, lx = i % TW;
            const int b = (ly >> 2) * (TW / 16) + (lx >> 4), oi = ((ly & 3) << 4) | (lx & 15);
            const float od = pv.depth_f32 ? reinterpret_cast<const float*>(s_depth + b * 256)[oi]
                                          : (float)reinterpret_cast<const uint16_t*>(s_depth + b * 256)[oi];
            const bool rm = add_pixel(od, s_skin[b * 128 + oi] != 0, z, a, acc_t, acc_a, acc_o, acc_h);
            if (a.dbg_depth) {
                const size_t o = ((size_t)p * pv.H + ty0 + ly) * pv.W + tx0 + lx;
                a.dbg_depth[o] = z;
                a.dbg_mask[o] = (uint8_t)(1 | (rm ? 2 : 0));
            }
        }
        __syncthreads();  // the z-buffer and the observation tile are refilled for the next tile
    }
    // a tile load that timed out leaves no copy behind
    if (!ok) mbar_wait_bounded(s_bar, phase, a.status);
    pdl_launch_dependents();

#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_t += __shfl_xor_sync(0xffffffffu, acc_t, o);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
        acc_o += __shfl_xor_sync(0xffffffffu, acc_o, o);
        acc_h += __shfl_xor_sync(0xffffffffu, acc_h, o);
    }
    long long* red_t = reinterpret_cast<long long*>(smem + L.red);
    uint32_t* red_c = reinterpret_cast<uint32_t*>(smem + L.red + 8 * NW);
    if (lane == 0) {
        red_t[warp] = acc_t;
        red_c[3 * warp] = acc_a;
        red_c[3 * warp + 1] = acc_o;
        red_c[3 * warp + 2] = acc_h;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NW; ++w) {
            acc_t += red_t[w];
            acc_a += red_c[3 * w];
            acc_o += red_c[3 * w + 1];
            acc_h += red_c[3 * w + 2];
        }
        flush_and_finish(a, p, wk, pv.stats, kcp, acc_t, acc_a, acc_o, acc_h, gridDim.x);
    }
}

template <int TW, int TH, int NW>
static cudaError_t launch_tiles(const CUtensorMap& tm_depth, const CUtensorMap& tm_skin, const RenderArgs& args,
                                cudaStream_t stream)
{
    using Lay = TileLayout<TW, TH, NW>;
    auto kern = render_tiles_kernel<TW, TH, NW>;
    // the shared-memory opt-in, once per device
    static std::atomic<uint32_t> opted[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!opted[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay(kMaxPrims).bytes);
        if (e != cudaSuccess) return e;
        opted[dev].store(1u, std::memory_order_release);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(args.K, args.P);
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = Lay(args.n_prims).bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr_pdl[1];
    attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr_pdl;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tm_depth, tm_skin, args);
}

cudaError_t launch_render_tiles(int variant, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                                const RenderArgs& args, cudaStream_t stream)
{
    switch (variant) {
    case HS_RENDER_TILES_32x16: return launch_tiles<32, 16, 4>(tm_depth, tm_skin, args, stream);
    case HS_RENDER_TILES_32x32: return launch_tiles<32, 32, 4>(tm_depth, tm_skin, args, stream);
    case HS_RENDER_TILES_64x32: return launch_tiles<64, 32, 4>(tm_depth, tm_skin, args, stream);
    case HS_RENDER_TILES_64x64: return launch_tiles<64, 64, 8>(tm_depth, tm_skin, args, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hs
