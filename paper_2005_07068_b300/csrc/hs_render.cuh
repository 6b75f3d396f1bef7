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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// an observation load waits at most this long (wall clock) ...
constexpr unsigned long long kTmaWaitNs = 500000000ull;
// ... and at most this many polls, should the clock not advance
constexpr uint32_t kTmaWaitPolls = 1u << 22;

// bounded wait: returns false (and flags the status word) if the phase does
// not complete within kTmaWaitNs (try_wait may suspend the thread for a
// system-dependent time per call, so the limit is kept in wall-clock time)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t spin = 0; spin < kTmaWaitPolls; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kTmaWaitNs) break;
    }
    set_status(status, HS_DEV_TMA_TIMEOUT);
    return false;
}

// ---- ray / quadric ----------------------------------------------------------------
// A primitive in scaled local coordinates is the quadric
//   ellipsoid:  |p|^2 = 1
//   cone:       X^2 + Z^2 = (1 + kappa Y)^2, |Y| <= 1, and the caps at Y = -1, +1
//               that the model leaves visible (record word 12)
// and the ray of pixel (u, v), d = (a, b, 1) with a = u inv_fx + off_x, meets it
// at depth t0 + s where the quadratic A s^2 + 2 B s + C = 0 holds (t0 = C_z, the
// primitive's centre depth).  Written relative to the ray through the projected
// centre, d = d_c + (alpha, beta, 0) with t0 d_c = C, the local ray is g + s h
// with k = M (alpha, beta, 0), g = t0 k, h = h_c + k, h_c = M d_c.
//
// Its discriminant B^2 - A C is a quadratic polynomial in the pixel offsets
// (du, dv) = (u - u_c, v - v_c) from the projected centre (the quartic and
// cubic terms cancel exactly, because shifting s does not change it).  Written
// with the identity (x.Dy)^2 - (x.Dx)(y.Dy) = -sum_{i<j} d_i d_j (x_i y_j - x_j y_i)^2
// for diagonal D, its coefficients are sums of squares of small terms, with no
// cancellation of the ~t0^2 |h_c|^2 parts:
//   ellipsoid: disc = |h_c|^2 + 2 h_c.k + |k|^2 - t0^2 |h_c x k|^2
//   cone:      disc = h_X^2 + h_Z^2 + 2 (h_X k_X + h_Z k_Z) + 2 kappa t0 (h_X n_XY - h_Z n_YZ)
//                     + k_X^2 + k_Z^2 + 2 t0 kappa (k_X n_XY - k_Z n_YZ)
//                     + t0^2 (kappa^2 (n_XY^2 + n_YZ^2) - n_XZ^2)
//              (h = h_c, n_ij = h_i k_j - h_j k_i)
// So a pixel is tested for coverage with one polynomial; the roots, which need
// A, B, C, are formed only where the discriminant is not negative.  The
// polynomial is evaluated by poly2, one association everywhere (the dv terms
// outermost), so a kernel that forms a pixel column's du terms once (Poly2Col)
// gets the same bits as one that evaluates it whole.
//
// Raster record (5 float4, built once per CTA from the 64-byte FK record):
//   q0 = (u_c, v_c, c0, c_u)   q1 = (c_v, c_uu, c_uv, c_vv)   disc polynomial
//   q2 = (k_u, t0)             q3 = (k_v, kappa or ellipsoid marker)
//   q4 = (h_c, caps)           k = du k_u + dv k_v
constexpr int kRastVec = 5;

struct RasterPrim {
    float4 q0, q1, q2, q3, q4;
};

__device__ __forceinline__ float poly2(float c0, float cu, float cv, float cuu, float cuv, float cvv, float du, float dv)
{
    return fmaf(dv, fmaf(dv, cvv, fmaf(du, cuv, cv)), fmaf(du, fmaf(du, cuu, cu), c0));
}
// a quadratic with its du terms formed once for a pixel column: poly2_col(du) then at(dv)
struct Poly2Col {
    float u0, u1, vv;
    __device__ __forceinline__ float at(float dv) const { return fmaf(dv, fmaf(dv, vv, u1), u0); }
};
__device__ __forceinline__ Poly2Col poly2_col(float c0, float cu, float cv, float cuu, float cuv, float cvv, float du)
{
    return Poly2Col{fmaf(du, fmaf(du, cuu, cu), c0), fmaf(du, cuv, cv), cvv};
}

__device__ __forceinline__ RasterPrim make_raster(const float4* rec, float inv_fx, float off_x, float inv_fy,
                                                  float off_y)
{
    const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3];
    const float m0[3] = {r0.x, r0.y, r0.z}, m1[3] = {r0.w, r1.x, r1.y}, m2[3] = {r1.z, r1.w, r2.x};
    const float t0 = r2.w, kap = r3.y;
    // projected centre direction and pixel (correctly rounded reciprocals: a
    // few ulps in u_c, v_c shift the silhouette by ~1e-4 px at most)
    const float it0 = __frcp_rn(t0);
    const float ac = r2.y * it0, bc = r2.z * it0;
    const float uc = (ac - off_x) * __frcp_rn(inv_fx), vc = (bc - off_y) * __frcp_rn(inv_fy);
    float hc[3], ku[3], kv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        hc[i] = fmaf(ac, m0[i], fmaf(bc, m1[i], m2[i]));
        ku[i] = m0[i] * inv_fx;
        kv[i] = m1[i] * inv_fy;
    }
    // (u, v) coefficients of the linear forms, and of products of two of them
    struct L { float u, v; };
    auto cr = [&](int i, int j) { return L{hc[i] * ku[j] - hc[j] * ku[i], hc[i] * kv[j] - hc[j] * kv[i]}; };
    const L kX{ku[0], kv[0]}, kY{ku[1], kv[1]}, kZ{ku[2], kv[2]};
    float c0, cu, cv, cuu, cuv, cvv;
    const float t2 = t0 * t0;
    if (kap > 1.5f) {  // ellipsoid
        const L n0 = cr(1, 2), n1 = cr(2, 0), n2 = cr(0, 1);
        c0 = hc[0] * hc[0] + hc[1] * hc[1] + hc[2] * hc[2];
        cu = 2.f * (hc[0] * kX.u + hc[1] * kY.u + hc[2] * kZ.u);
        cv = 2.f * (hc[0] * kX.v + hc[1] * kY.v + hc[2] * kZ.v);
        cuu = (kX.u * kX.u + kY.u * kY.u + kZ.u * kZ.u) - t2 * (n0.u * n0.u + n1.u * n1.u + n2.u * n2.u);
        cuv = 2.f * ((kX.u * kX.v + kY.u * kY.v + kZ.u * kZ.v) - t2 * (n0.u * n0.v + n1.u * n1.v + n2.u * n2.v));
        cvv = (kX.v * kX.v + kY.v * kY.v + kZ.v * kZ.v) - t2 * (n0.v * n0.v + n1.v * n1.v + n2.v * n2.v);
    } else {  // cone
        const L nXY = cr(0, 1), nYZ = cr(1, 2), nXZ = cr(0, 2);
        const float tk = t0 * kap, tk2 = t2 * kap * kap;
        c0 = hc[0] * hc[0] + hc[2] * hc[2];
        cu = 2.f * (hc[0] * kX.u + hc[2] * kZ.u) + 2.f * tk * (hc[0] * nXY.u - hc[2] * nYZ.u);
        cv = 2.f * (hc[0] * kX.v + hc[2] * kZ.v) + 2.f * tk * (hc[0] * nXY.v - hc[2] * nYZ.v);
        cuu = kX.u * kX.u + kZ.u * kZ.u + 2.f * tk * (kX.u * nXY.u - kZ.u * nYZ.u) +
              tk2 * (nXY.u * nXY.u + nYZ.u * nYZ.u) - t2 * nXZ.u * nXZ.u;
        cuv = 2.f * (kX.u * kX.v + kZ.u * kZ.v) +
              2.f * tk * (kX.u * nXY.v + kX.v * nXY.u - kZ.u * nYZ.v - kZ.v * nYZ.u) +
              2.f * tk2 * (nXY.u * nXY.v + nYZ.u * nYZ.v) - 2.f * t2 * nXZ.u * nXZ.v;
        cvv = kX.v * kX.v + kZ.v * kZ.v + 2.f * tk * (kX.v * nXY.v - kZ.v * nYZ.v) +
              tk2 * (nXY.v * nXY.v + nYZ.v * nYZ.v) - t2 * nXZ.v * nXZ.v;
    }
    RasterPrim R;
    R.q0 = make_float4(uc, vc, c0, cu);
    R.q1 = make_float4(cv, cuu, cuv, cvv);
    R.q2 = make_float4(ku[0], ku[1], ku[2], t0);
    R.q3 = make_float4(kv[0], kv[1], kv[2], kap);
    R.q4 = make_float4(hc[0], hc[1], hc[2], r3.x);
    return R;
}

// the record into shared memory (5 float4 at d)
__device__ __forceinline__ void store_raster(const RasterPrim& R, float4* d)
{
    d[0] = R.q0;
    d[1] = R.q1;
    d[2] = R.q2;
    d[3] = R.q3;
    d[4] = R.q4;
}

// the discriminant at pixel offsets (du, dv): >= 0 where the quadric's surface
// can be hit (for a cone with visible caps the caps are tested regardless)
__device__ __forceinline__ float raster_disc(const float4& q0, const float4& q1, float du, float dv)
{
    return poly2(q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, du, dv);
}
// the discriminant's du terms for a pixel column
__device__ __forceinline__ Poly2Col raster_disc_col(const float4& q0, const float4& q1, float du)
{
    return poly2_col(q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, du);
}

// The ray of the pixel at offsets (du, dv) in the primitive's scaled frame:
// h = h_c + k and g = t0 k with k = du k_u + dv k_v (the point of the ray at
// depth t0 + s is g + s h).
struct RasterRay {
    float hx, hy, hz, gx, gy, gz;
};
__device__ __forceinline__ RasterRay raster_ray(const float4& q2, const float4& q3, const float4& q4, float du,
                                                float dv)
{
    const float t0 = q2.w;
    const float kx = fmaf(du, q2.x, dv * q3.x), ky = fmaf(du, q2.y, dv * q3.y), kz = fmaf(du, q2.z, dv * q3.z);
    return RasterRay{q4.x + kx, q4.y + ky, q4.z + kz, t0 * kx, t0 * ky, t0 * kz};
}

// Nearest hit with an ellipsoid (|g + s h| = 1) given the discriminant, as the
// depth offset s from its centre depth t0, or +inf.  (__fmul_rn: the roots'
// last products are never fused with a later add, so every kernel rounds them
// alike.)
__device__ __forceinline__ float raster_root_ellipsoid(float t0, const RasterRay& r, float disc)
{
    float best = INFINITY;
    if (disc >= 0.f) {
        const float A = fmaf(r.hx, r.hx, fmaf(r.hy, r.hy, r.hz * r.hz));
        const float B = fmaf(r.gx, r.hx, fmaf(r.gy, r.hy, r.gz * r.hz));
        const float sq = sqrt_approx(disc);
        const float ia = rcp_approx(A);
        const float sn = __fmul_rn(-B - sq, ia);
        const float sf = __fmul_rn(-B + sq, ia);  // the camera is inside the ellipsoid: the far root, if in front
        best = t0 + sn > 0.f ? sn : (t0 + sf > 0.f ? sf : INFINITY);
    }
    return best;
}

// Nearest hit with a truncated cone (X^2 + Z^2 = (1 + kappa Y)^2, |Y| <= 1, and
// its planar caps where the bits of caps say they are visible) given the
// discriminant, as the depth offset s from t0, or +inf.
__device__ __forceinline__ float raster_root_cone(float t0, float kap, uint32_t caps, const RasterRay& r, float disc)
{
    float best = INFINITY;
    if (disc >= 0.f) {
        const float w0 = fmaf(kap, r.gy, 1.f), w1 = kap * r.hy;
        const float A = fmaf(r.hx, r.hx, fmaf(r.hz, r.hz, -w1 * w1));
        const float B = fmaf(r.gx, r.hx, fmaf(r.gz, r.hz, -w0 * w1));
        const float C = fmaf(r.gx, r.gx, fmaf(r.gz, r.gz, -w0 * w0));
        const float sq = sqrt_approx(disc);
        const float qq = -(B + copysignf(sq, B));
        const float s1 = __fmul_rn(qq, rcp_approx(A));
        const float s2 = __fmul_rn(C, rcp_approx(qq));
        const float y1 = fmaf(s1, r.hy, r.gy), y2 = fmaf(s2, r.hy, r.gy);
        if (fabsf(y1) <= 1.f && t0 + s1 > 0.f) best = s1;
        if (fabsf(y2) <= 1.f && t0 + s2 > 0.f) best = fminf(best, s2);
    }
    if (caps) {  // planar caps at Y = -1 (radius 1 - kappa) and Y = +1 (radius 1 + kappa)
        const float ihy = rcp_approx(r.hy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(caps & (1u << c))) continue;
            const float yc = c ? 1.f : -1.f;
            const float s = __fmul_rn(yc - r.gy, ihy);
            const float X = fmaf(s, r.hx, r.gx), Z = fmaf(s, r.hz, r.gz);
            const float w = 1.f + yc * kap;
            if (fmaf(X, X, Z * Z) <= w * w && t0 + s > 0.f) best = fminf(best, s);
        }
    }
    return best;
}

// Nearest hit of the pixel at offsets (du, dv) with one primitive, given its
// discriminant there, as the depth offset s from the primitive's centre depth
// t0 (depth = t0 + s), or +inf.
__device__ __forceinline__ float raster_hit(const float4& q2, const float4& q3, const float4& q4, float du, float dv,
                                            float disc)
{
    const RasterRay r = raster_ray(q2, q3, q4, du, dv);
    return q3.w > 1.5f ? raster_root_ellipsoid(q2.w, r, disc)
                       : raster_root_cone(q2.w, q3.w, __float_as_uint(q4.w), r, disc);
}

// ---- two pixels at once with packed FP32 (fma / add / mul .f32x2) ----
// Each function below is its single-pixel namesake's operations applied to
// two pixels at once, lane by lane (the packed operations round every
// component exactly as the scalar ones), so both give the same bits.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
struct Ray2 {
    float2 hx, hy, hz, gx, gy, gz;
};
// raster_disc for the pixels (du.x, dv.x) and (du.y, dv.y)
__device__ __forceinline__ float2 raster_disc2(const float4& q0, const float4& q1, float2 du, float2 dv)
{
    return __ffma2_rn(dv, __ffma2_rn(dv, f2(q1.w), __ffma2_rn(du, f2(q1.z), f2(q1.x))),
                      __ffma2_rn(du, __ffma2_rn(du, f2(q1.y), f2(q0.w)), f2(q0.z)));
}
// raster_ray for the pixels (du.x, dv.x) and (du.y, dv.y)
__device__ __forceinline__ Ray2 raster_ray2(const float4& q2, const float4& q3, const float4& q4, float2 du2,
                                            float2 dv)
{
    const float2 t02 = f2(q2.w);
    const float2 kx = __ffma2_rn(du2, f2(q2.x), __fmul2_rn(dv, f2(q3.x)));
    const float2 ky = __ffma2_rn(du2, f2(q2.y), __fmul2_rn(dv, f2(q3.y)));
    const float2 kz = __ffma2_rn(du2, f2(q2.z), __fmul2_rn(dv, f2(q3.z)));
    return Ray2{__fadd2_rn(f2(q4.x), kx), __fadd2_rn(f2(q4.y), ky), __fadd2_rn(f2(q4.z), kz),
                __fmul2_rn(t02, kx), __fmul2_rn(t02, ky), __fmul2_rn(t02, kz)};
}
// raster_root_ellipsoid for both pixels
__device__ __forceinline__ float2 raster_root_ellipsoid2(float t0, const Ray2& r, float2 disc)
{
    const float2 A = __ffma2_rn(r.hx, r.hx, __ffma2_rn(r.hy, r.hy, __fmul2_rn(r.hz, r.hz)));
    const float2 B = __ffma2_rn(r.gx, r.hx, __ffma2_rn(r.gy, r.hy, __fmul2_rn(r.gz, r.hz)));
    const float2 sq = make_float2(sqrt_approx(disc.x), sqrt_approx(disc.y));
    const float2 ia = make_float2(rcp_approx(A.x), rcp_approx(A.y));
    const float2 nB = neg2(B);
    const float2 sn = __fmul2_rn(__fadd2_rn(nB, neg2(sq)), ia);
    const float2 sf = __fmul2_rn(__fadd2_rn(nB, sq), ia);
    const float2 tn = __fadd2_rn(f2(t0), sn), tf = __fadd2_rn(f2(t0), sf);
    float2 best;
    best.x = disc.x >= 0.f ? (tn.x > 0.f ? sn.x : (tf.x > 0.f ? sf.x : INFINITY)) : INFINITY;
    best.y = disc.y >= 0.f ? (tn.y > 0.f ? sn.y : (tf.y > 0.f ? sf.y : INFINITY)) : INFINITY;
    return best;
}
// raster_root_cone for both pixels
__device__ __forceinline__ float2 raster_root_cone2(float t0, float kap, uint32_t caps, const Ray2& r, float2 disc)
{
    const float2 t02 = f2(t0), kap2 = f2(kap);
    const float2 w0 = __ffma2_rn(kap2, r.gy, f2(1.f)), w1 = __fmul2_rn(kap2, r.hy);
    const float2 nw0 = neg2(w0), nw1 = neg2(w1);
    const float2 A = __ffma2_rn(r.hx, r.hx, __ffma2_rn(r.hz, r.hz, __fmul2_rn(nw1, w1)));
    const float2 B = __ffma2_rn(r.gx, r.hx, __ffma2_rn(r.gz, r.hz, __fmul2_rn(nw0, w1)));
    const float2 C = __ffma2_rn(r.gx, r.gx, __ffma2_rn(r.gz, r.gz, __fmul2_rn(nw0, w0)));
    const float2 sq = make_float2(sqrt_approx(disc.x), sqrt_approx(disc.y));
    const float2 qq = neg2(__fadd2_rn(B, make_float2(copysignf(sq.x, B.x), copysignf(sq.y, B.y))));
    const float2 s1 = __fmul2_rn(qq, make_float2(rcp_approx(A.x), rcp_approx(A.y)));
    const float2 s2 = __fmul2_rn(C, make_float2(rcp_approx(qq.x), rcp_approx(qq.y)));
    const float2 y1 = __ffma2_rn(s1, r.hy, r.gy), y2 = __ffma2_rn(s2, r.hy, r.gy);
    const float2 u1 = __fadd2_rn(t02, s1), u2 = __fadd2_rn(t02, s2);
    float2 best = make_float2(INFINITY, INFINITY);
    if (disc.x >= 0.f) {
        if (fabsf(y1.x) <= 1.f && u1.x > 0.f) best.x = s1.x;
        if (fabsf(y2.x) <= 1.f && u2.x > 0.f) best.x = fminf(best.x, s2.x);
    }
    if (disc.y >= 0.f) {
        if (fabsf(y1.y) <= 1.f && u1.y > 0.f) best.y = s1.y;
        if (fabsf(y2.y) <= 1.f && u2.y > 0.f) best.y = fminf(best.y, s2.y);
    }
    if (caps) {
        const float2 ihy = make_float2(rcp_approx(r.hy.x), rcp_approx(r.hy.y));
        const float2 ngy = neg2(r.gy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(caps & (1u << c))) continue;
            const float yc = c ? 1.f : -1.f;
            const float2 s = __fmul2_rn(__fadd2_rn(f2(yc), ngy), ihy);
            const float2 X = __ffma2_rn(s, r.hx, r.gx), Z = __ffma2_rn(s, r.hz, r.gz);
            const float2 rr = __ffma2_rn(X, X, __fmul2_rn(Z, Z));
            const float w = 1.f + yc * kap;
            const float ww = w * w;
            const float2 u = __fadd2_rn(t02, s);
            if (rr.x <= ww && u.x > 0.f) best.x = fminf(best.x, s.x);
            if (rr.y <= ww && u.y > 0.f) best.y = fminf(best.y, s.y);
        }
    }
    return best;
}

// ---- primitives in front of the camera ----
// FK gives a primitive whose solid lies beyond the plane z = 1 mm its screen
// box, and one that reaches the plane the sentinel box from -32767 (a box
// clamped there is treated alike).  Every point of a primitive in front has
// depth >= 1 mm, so a covered pixel's near root lies in front of the camera:
// the roots' FP32 error (~1e-3 mm at 500 mm) cannot make t0 + s <= 0.  Its
// renderer may then skip the far root and the tests of positive depth, and
// the depths are bit for bit those of the general functions above.
__device__ __forceinline__ bool raster_in_front(int box_u0) { return box_u0 != -32767; }

// raster_root_ellipsoid for a primitive in front, as the depth t0 + s of the
// near root (the same operations, so the same bits); call where disc >= 0
__device__ __forceinline__ float raster_z_ellipsoid_front(float t0, const RasterRay& r, float disc)
{
    const float A = fmaf(r.hx, r.hx, fmaf(r.hy, r.hy, r.hz * r.hz));
    const float B = fmaf(r.gx, r.hx, fmaf(r.gy, r.hy, r.gz * r.hz));
    const float sq = sqrt_approx(disc);
    const float ia = rcp_approx(A);
    return t0 + __fmul_rn(-B - sq, ia);
}
// raster_root_cone for a primitive in front (no test of positive depth)
__device__ __forceinline__ float raster_root_cone_front(float kap, uint32_t caps, const RasterRay& r, float disc)
{
    float best = INFINITY;
    if (disc >= 0.f) {
        const float w0 = fmaf(kap, r.gy, 1.f), w1 = kap * r.hy;
        const float A = fmaf(r.hx, r.hx, fmaf(r.hz, r.hz, -w1 * w1));
        const float B = fmaf(r.gx, r.hx, fmaf(r.gz, r.hz, -w0 * w1));
        const float C = fmaf(r.gx, r.gx, fmaf(r.gz, r.gz, -w0 * w0));
        const float sq = sqrt_approx(disc);
        const float qq = -(B + copysignf(sq, B));
        const float s1 = __fmul_rn(qq, rcp_approx(A));
        const float s2 = __fmul_rn(C, rcp_approx(qq));
        const float y1 = fmaf(s1, r.hy, r.gy), y2 = fmaf(s2, r.hy, r.gy);
        if (fabsf(y1) <= 1.f) best = s1;
        if (fabsf(y2) <= 1.f) best = fminf(best, s2);
    }
    if (caps) {
        const float ihy = rcp_approx(r.hy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(caps & (1u << c))) continue;
            const float yc = c ? 1.f : -1.f;
            const float s = __fmul_rn(yc - r.gy, ihy);
            const float X = fmaf(s, r.hx, r.gx), Z = fmaf(s, r.hz, r.gz);
            const float w = 1.f + yc * kap;
            if (fmaf(X, X, Z * Z) <= w * w) best = fminf(best, s);
        }
    }
    return best;
}
// The depth t0 + s of the nearest hit (raster_hit), or +inf; where raster_maybe
// holds.  front: the primitive is in front of the camera (raster_in_front).
__device__ __forceinline__ float raster_hit_z(const float4& q2, const float4& q3, const float4& q4, float du, float dv,
                                              float disc, bool front)
{
    const RasterRay r = raster_ray(q2, q3, q4, du, dv);
    const float t0 = q2.w;
    if (!front)
        return t0 + (q3.w > 1.5f ? raster_root_ellipsoid(t0, r, disc)
                                 : raster_root_cone(t0, q3.w, __float_as_uint(q4.w), r, disc));
    return q3.w > 1.5f ? raster_z_ellipsoid_front(t0, r, disc)
                       : t0 + raster_root_cone_front(q3.w, __float_as_uint(q4.w), r, disc);
}

// raster_root_ellipsoid2 for a primitive in front: the near root s (the same
// operations, so the same bits), NaN where disc < 0.  The caller selects it
// by its coverage bits before adding t0, as after the general functions'
// selects: a packed add that directly follows the root's packed product was
// measured to round differently (contracted), one ulp on some pixels.
__device__ __forceinline__ float2 raster_near_ellipsoid2_front(const Ray2& r, float2 disc)
{
    const float2 A = __ffma2_rn(r.hx, r.hx, __ffma2_rn(r.hy, r.hy, __fmul2_rn(r.hz, r.hz)));
    const float2 B = __ffma2_rn(r.gx, r.hx, __ffma2_rn(r.gy, r.hy, __fmul2_rn(r.gz, r.hz)));
    const float2 sq = make_float2(sqrt_approx(disc.x), sqrt_approx(disc.y));
    const float2 ia = make_float2(rcp_approx(A.x), rcp_approx(A.y));
    return __fmul2_rn(__fadd2_rn(neg2(B), neg2(sq)), ia);
}
// raster_root_cone2 for a primitive in front (no test of positive depth)
__device__ __forceinline__ float2 raster_root_cone2_front(float kap, uint32_t caps, const Ray2& r, float2 disc)
{
    const float2 kap2 = f2(kap);
    const float2 w0 = __ffma2_rn(kap2, r.gy, f2(1.f)), w1 = __fmul2_rn(kap2, r.hy);
    const float2 nw0 = neg2(w0), nw1 = neg2(w1);
    const float2 A = __ffma2_rn(r.hx, r.hx, __ffma2_rn(r.hz, r.hz, __fmul2_rn(nw1, w1)));
    const float2 B = __ffma2_rn(r.gx, r.hx, __ffma2_rn(r.gz, r.hz, __fmul2_rn(nw0, w1)));
    const float2 C = __ffma2_rn(r.gx, r.gx, __ffma2_rn(r.gz, r.gz, __fmul2_rn(nw0, w0)));
    const float2 sq = make_float2(sqrt_approx(disc.x), sqrt_approx(disc.y));
    const float2 qq = neg2(__fadd2_rn(B, make_float2(copysignf(sq.x, B.x), copysignf(sq.y, B.y))));
    const float2 s1 = __fmul2_rn(qq, make_float2(rcp_approx(A.x), rcp_approx(A.y)));
    const float2 s2 = __fmul2_rn(C, make_float2(rcp_approx(qq.x), rcp_approx(qq.y)));
    const float2 y1 = __ffma2_rn(s1, r.hy, r.gy), y2 = __ffma2_rn(s2, r.hy, r.gy);
    float2 best = make_float2(INFINITY, INFINITY);
    if (disc.x >= 0.f) {
        if (fabsf(y1.x) <= 1.f) best.x = s1.x;
        if (fabsf(y2.x) <= 1.f) best.x = fminf(best.x, s2.x);
    }
    if (disc.y >= 0.f) {
        if (fabsf(y1.y) <= 1.f) best.y = s1.y;
        if (fabsf(y2.y) <= 1.f) best.y = fminf(best.y, s2.y);
    }
    if (caps) {
        const float2 ihy = make_float2(rcp_approx(r.hy.x), rcp_approx(r.hy.y));
        const float2 ngy = neg2(r.gy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(caps & (1u << c))) continue;
            const float yc = c ? 1.f : -1.f;
            const float2 s = __fmul2_rn(__fadd2_rn(f2(yc), ngy), ihy);
            const float2 X = __ffma2_rn(s, r.hx, r.gx), Z = __ffma2_rn(s, r.hz, r.gz);
            const float2 rr = __ffma2_rn(X, X, __fmul2_rn(Z, Z));
            const float w = 1.f + yc * kap;
            const float ww = w * w;
            if (rr.x <= ww) best.x = fminf(best.x, s.x);
            if (rr.y <= ww) best.y = fminf(best.y, s.y);
        }
    }
    return best;
}

// true when the primitive must be tested at a pixel whose discriminant is disc
__device__ __forceinline__ bool raster_maybe(const float4& q4, float disc)
{
    return disc >= 0.f || __float_as_uint(q4.w) != 0u;
}

// per-pixel terms of Eq. 4 (reading R1) as differences to the no-hit baseline,
// added to the lane's fixed-point / integer sums; returns r_m.  z: the rendered
// depth, t0 + s rounded once to FP32 (within 2^-24 of it, 3e-5 mm at 500 mm);
// O_d - z is exact wherever it can fall below d_M (the two are then within a
// factor of two of each other).
__device__ __forceinline__ bool add_pixel(float od, bool S, float z, const RenderArgs& a, long long& at, uint32_t& aa,
                                          uint32_t& ao, uint32_t& ah)
{
    const bool valid = S && od > 0.f;
    const float diff = fabsf(od - z);
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

// true when particle p belongs to a swarm of a batch that has stopped (the
// batch step's stop flag): its E is not scored again this frame.  Read after
// the programmatic-launch wait (the previous step kernel writes the flag).
__device__ __forceinline__ bool particle_stopped(const RenderArgs& a, int p)
{
    return a.batch.views && swarm_stop_gen(a.batch, a.batch.sid[p]) != 0u;
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

// E of Eq. 5 from a particle's sums (reading R1): tf = sum of the rendered
// pixels' depth-term differences to the no-hit baseline (fixed point, 2^-24
// mm), sa = sum(S and r_m), so_d = sum(r_m and not S); the frame's totals
// stats = (#valid skin pixels, #skin pixels) supply the baseline.
// D = sum t / sum(S or r_m) + lambda (1 - 2 sum(S and r_m) / (sum(S and r_m) + sum(S or r_m))),
// D = lambda for an empty union; E = D + lambda_k kc.
__device__ __forceinline__ float form_E(long long tf, uint32_t sa, uint32_t so_d, const uint32_t* stats, float d_M,
                                        float lambda, float lambda_k, float kcp, float& t_sum, uint32_t& so)
{
    const uint32_t n_valid = stats[0], n_skin = stats[1];
    // fixed point -> float from the two 32-bit halves (no 64-bit conversion)
    const float t_fix_f = (float)(int)(tf >> 32) * 4294967296.0f + (float)(uint32_t)(tf & 0xffffffffu);
    t_sum = t_fix_f * (1.0f / kFix) + d_M * (float)n_valid;
    so = so_d + n_skin;
    float D;
    if (so == 0) {
        D = lambda;
    } else {
        const float fa = (float)sa, fo = (float)so;
        D = t_sum / fo + lambda * (1.f - 2.f * fa / (fa + fo));
    }
    return D + lambda_k * kcp;
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
    float t_sum;
    uint32_t so;
    a.E[p] = form_E(tf, sa, so_d, stats, a.d_M, a.lambda, a.lambda_k, kcp, t_sum, so);
    if (a.parts) a.parts[p] = HsParts{t_sum, sa, so, sh};
    *wk = HsParticleWork{};  // every contributor is done: safe to clear
}

}  // namespace hs
