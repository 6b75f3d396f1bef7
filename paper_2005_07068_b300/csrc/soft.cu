// soft.cu -- the smoothed objective E_s and its gradient with respect to the
// 26 pose parameters (the differentiable counterpart of render_score_batch).
//
// E (Eq. 4-5, Section III.A) is piecewise constant in the pose at every
// silhouette and depth threshold, so the gradient polish descends E_s, which
// keeps E's terms and replaces each hard decision by a smooth one:
//
//  * primitive j covers pixel p with alpha_j = sigma(delta_j / tau), delta_j =
//    Delta_j / |grad_pixel Delta_j| the first-order signed distance (pixels) to
//    j's silhouette from the ray-quadric discriminant Delta_j; a cone's alpha
//    is multiplied by sigma(delta_Y / tau), its end cut softened with
//    delta_Y = (1 - |Y_e|) L (L = projected half-length of the axis in pixels,
//    at least the cone's radius in pixels; Y_e = the axial coordinate of the
//    root well inside the silhouette, of the ray's closest approach to the
//    axis near and outside it, blended by w = sigma(delta / tau - 2));
//  * the depth of j is the near root of the ray-quadric equation written as
//    C / (-B + sqrt(Delta+)) in the camera-ray parameter (bounded as A -> 0;
//    B < 0 required), with the soft positive part Delta+ = (Delta +
//    sqrt(Delta^2 + (tau |grad Delta|)^2)) / 2; its offset from the centre
//    depth is clamped smoothly (C1) to twice the primitive's bounding radius;
//  * a cone seen within a few degrees of a surface generator fades out:
//    alpha also times a^4 / (a^4 + (0.06 tau)^4), a = A / |h|^2;
//  * the primitives touching the pixel are composited front to back in depth
//    order: c = 1 - prod (1 - alpha), z~ = sum T_j alpha_j z_j / c;
//  * per pixel: diff = sqrt((O_d - z~)^2 + tau_mm^2), t_hit = smin(diff, d_M)
//    (width tau_mm) on valid pixels, r_m's test sigma((d_m - diff) / tau_mm),
//    t = c t_hit + (1 - c) t_miss, r_m = c m; then D_s and E_s as Eq. 4-5.
//
// soft_forward_kernel forms E_s (fixed-point integer sums, like the hard
// path); soft_backward_kernel recomputes each pixel and pushes dE_s/d(pixel
// terms) back through the compositing and each primitive's coverage and depth
// to its record (M, C: 12 numbers) and, for cones, to L; pose_grad_kernel maps
// those adjoints to the 26 pose parameters with the FK's tangents (each bone
// frame's derivative for each parameter from the world axes of its joints).
#include <atomic>

#include "hs_fk.cuh"
#include "hs_render.cuh"

namespace hs {

constexpr int kSoftThreads = 128;
constexpr int kSoftMargin = 8;      // pixels around each box where alpha may still exceed kAlphaMin
constexpr float kAlphaMin = 1e-7f;  // touches below this are dropped

// The smoothed objective is itself an approximation (its tolerance against the
// FP64 oracle is far above a few ulps), so its arithmetic takes the hardware's
// approximate forms: reciprocal and square root (rcp_approx, sqrt_approx),
// __fdividef and __expf / __logf.
__device__ __forceinline__ float sigm(float x) { return __fdividef(1.f, 1.f + __expf(-x)); }

// Adjoints are summed as 64-bit fixed point with 2^-40 resolution (|value| <
// 2^23), so that the totals do not depend on the order of the atomic adds.
// The conversion uses 32-bit halves: v 2^40 is exact in FP32 (a power-of-two
// scaling), its high and low words are then exact FP32 integers.
constexpr float kAdjScale = 1099511627776.0f;  // 2^40
__device__ __forceinline__ long long adj_to_fix(float v)
{
    const float w = v * kAdjScale;
    const float hi = floorf(w * 2.3283064365386963e-10f);  // w / 2^32
    const float lo = fmaf(-hi, 4294967296.0f, w);          // exact: w - hi 2^32, in [0, 2^32)
    return ((long long)__float2int_rn(hi) << 32) + (long long)__float2uint_rn(lo);
}
// A warp's exact sum of 64-bit fixed-point values (mod 2^64, as the 64-bit
// adds they replace): f = l0 + l1 2^21 + l2 2^42 with l0, l1 in [0, 2^21) and
// l2 in [-2^21, 2^21), so each limb's sum over 32 lanes fits in 32 bits and
// takes one integer warp reduction.  Returns the three limb sums (the same
// on every lane); fix_from_limbs recombines them.
__device__ __forceinline__ int3 warp_sum_limbs(long long f)
{
    const unsigned long long u = (unsigned long long)f;
    const int l0 = (int)(u & 0x1fffffull), l1 = (int)((u >> 21) & 0x1fffffull), l2 = (int)(f >> 42);
    return make_int3(__reduce_add_sync(0xffffffffu, l0), __reduce_add_sync(0xffffffffu, l1),
                     __reduce_add_sync(0xffffffffu, l2));
}
__device__ __forceinline__ long long fix_from_limbs(int3 s)
{
    return (long long)((unsigned long long)(long long)s.x + ((unsigned long long)(long long)s.y << 21) +
                       ((unsigned long long)(long long)s.z << 42));
}
__device__ __forceinline__ float adj_from_fix(long long f)
{
    const float hi = (float)(int)(f >> 32), lo = (float)(uint32_t)(f & 0xffffffffu);
    return fmaf(hi, 4294967296.0f, lo) * (1.0f / kAdjScale);
}

// everything a primitive's coverage and depth at one pixel depend on
struct SoftPrimEval {
    float h[3], g[3], hu[3], gu[3], hv[3], gv[3];
    float A, B, C, Au, Bu, Cu, Av, Bv, Cv;
    float D, Du, Dv, N, delta, q, Dp, r;
    float num, den, s_raw, s;     // root offset from t0 before / after the clamp
    float sig_d, w, Ye, sig_y;    // cones
    float sstar, sstar_c, hh, a_rel, fade;
    float alpha, z;
    bool ok;
};

// smooth clamp of a depth offset to the bounding radius R: identity for
// |s| <= R, sign(s) R (2 - exp(1 - |s| / R)) beyond (C1, |.| < 2R)
__device__ __forceinline__ float clamp_offset(float s, float R, float& ds)
{
    const float as = fabsf(s);
    if (as <= R) {
        ds = 1.f;
        return s;
    }
    const float ex = __expf(1.f - __fdividef(as, R));
    ds = ex;
    return copysignf(R * (2.f - ex), s);
}

// The quadric of a record in the form p^T Q p + 2 q^T p - 1 along p = g + s h:
// ellipsoid Q = I, q = 0; cone Q = diag(1, -kappa^2, 1), q = (0, -kappa, 0).
// Record columns of M: c0 = (r0.x, r0.y, r0.z), c1 = (r0.w, r1.x, r1.y),
// c2 = (r1.z, r1.w, r2.x); centre (r2.y, r2.z, r2.w), t0 = r2.w.
__device__ __forceinline__ void soft_eval(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                          float L, float Rb, float a, float b, float ifx, float ify, float tau,
                                          SoftPrimEval& e)
{
    const bool cone = r3.y < 1.5f;
    const float kap = cone ? r3.y : 0.f;
    const float Qy = cone ? -kap * kap : 1.f, qy = cone ? -kap : 0.f;
    const float t0 = r2.w;
    const float c0[3] = {r0.x, r0.y, r0.z}, c1[3] = {r0.w, r1.x, r1.y}, c2[3] = {r1.z, r1.w, r2.x};
    const float ex = fmaf(t0, a, -r2.y), ey = fmaf(t0, b, -r2.z);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        e.h[i] = fmaf(a, c0[i], fmaf(b, c1[i], c2[i]));
        e.g[i] = fmaf(ex, c0[i], ey * c1[i]);
        e.hu[i] = c0[i] * ifx;
        e.gu[i] = t0 * e.hu[i];
        e.hv[i] = c1[i] * ify;
        e.gv[i] = t0 * e.hv[i];
    }
    const float Q[3] = {1.f, Qy, 1.f};
    float A = 0.f, B = 0.f, C = -1.f, Au = 0.f, Bu = 0.f, Cu = 0.f, Av = 0.f, Bv = 0.f, Cv = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        A = fmaf(Q[i] * e.h[i], e.h[i], A);
        B = fmaf(Q[i] * e.g[i], e.h[i], B);
        C = fmaf(Q[i] * e.g[i], e.g[i], C);
        Au = fmaf(2.f * Q[i] * e.h[i], e.hu[i], Au);
        Av = fmaf(2.f * Q[i] * e.h[i], e.hv[i], Av);
        Bu = fmaf(Q[i], fmaf(e.gu[i], e.h[i], e.g[i] * e.hu[i]), Bu);
        Bv = fmaf(Q[i], fmaf(e.gv[i], e.h[i], e.g[i] * e.hv[i]), Bv);
        Cu = fmaf(2.f * Q[i] * e.g[i], e.gu[i], Cu);
        Cv = fmaf(2.f * Q[i] * e.g[i], e.gv[i], Cv);
    }
    B = fmaf(qy, e.h[1], B);
    C = fmaf(2.f * qy, e.g[1], C);
    Bu = fmaf(qy, e.hu[1], Bu);
    Bv = fmaf(qy, e.hv[1], Bv);
    Cu = fmaf(2.f * qy, e.gu[1], Cu);
    Cv = fmaf(2.f * qy, e.gv[1], Cv);
    e.A = A; e.B = B; e.C = C; e.Au = Au; e.Bu = Bu; e.Cu = Cu; e.Av = Av; e.Bv = Bv; e.Cv = Cv;
    e.D = fmaf(B, B, -A * C);
    e.Du = fmaf(2.f * B, Bu, -fmaf(Au, C, A * Cu));
    e.Dv = fmaf(2.f * B, Bv, -fmaf(Av, C, A * Cv));
    e.N = fmaxf(sqrt_approx(fmaf(e.Du, e.Du, e.Dv * e.Dv)), 1e-30f);
    e.delta = __fdividef(e.D, e.N);
    const float tn = tau * e.N;
    e.q = sqrt_approx(fmaf(e.D, e.D, tn * tn));
    e.Dp = 0.5f * (e.D + e.q);
    e.r = sqrt_approx(e.Dp);
    // near root in the camera-ray parameter t = t0 + s: t = C_cam / (-B_cam + r) with
    // B_cam = B - t0 A and C_cam = C - 2 t0 B + t0^2 A, i.e. s = num / den below
    e.num = C - t0 * (B + e.r);
    e.den = fmaf(t0, A, -B) + e.r;
    e.ok = A > 0.f && fmaf(-t0, A, B) < 0.f && e.den > 0.f;
    float ds;
    e.s_raw = e.ok ? __fdividef(e.num, e.den) : 0.f;
    e.s = clamp_offset(e.s_raw, Rb, ds);
    e.z = t0 + e.s;
    e.ok = e.ok && e.z > 0.f;
    const float itau = rcp_approx(tau);
    e.sig_d = sigm(e.delta * itau);
    float alpha = e.sig_d;
    if (cone && e.ok) {
        e.w = sigm(fmaf(e.delta, itau, -2.f));
        e.sstar = __fdividef(-B, A);
        float dss;
        e.sstar_c = clamp_offset(e.sstar, Rb, dss);
        e.Ye = fmaf(fmaf(e.w, e.s - e.sstar_c, e.sstar_c), e.h[1], e.g[1]);  // g_y + (w s + (1 - w) s*) h_y
        e.sig_y = sigm((1.f - fabsf(e.Ye)) * L * itau);
        e.hh = fmaf(e.h[0], e.h[0], fmaf(e.h[1], e.h[1], e.h[2] * e.h[2]));
        e.a_rel = __fdividef(A, e.hh);
        const float a4 = e.a_rel * e.a_rel * e.a_rel * e.a_rel, f0 = 0.06f * tau, f4 = f0 * f0 * f0 * f0;
        e.fade = __fdividef(a4, a4 + f4);
        alpha *= e.sig_y * e.fade;
    }
    e.alpha = e.ok ? alpha : 0.f;
}

// push (d alpha, d z) of one evaluation back to the record (adj[0..8] = M in
// record order, adj[9..11] = C) and to L (adj[12])
__device__ __forceinline__ void soft_backprop(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                              float L, float Rb, float a, float b, float ifx, float ify, float tau,
                                              const SoftPrimEval& e, float ga, float gz, float* adj)
{
    if (!e.ok) return;
    const bool cone = r3.y < 1.5f;
    const float kap = cone ? r3.y : 0.f;
    const float Qy = cone ? -kap * kap : 1.f, qy = cone ? -kap : 0.f;
    const float Q[3] = {1.f, Qy, 1.f};
    const float t0 = r2.w;
    float gA = 0.f, gB = 0.f, gC = 0.f, gD = 0.f, gN = 0.f, gr = 0.f, gdelta = 0.f, gt0 = 0.f;
    float gh[3] = {0.f, 0.f, 0.f}, gg[3] = {0.f, 0.f, 0.f};
    // alpha = sig_d (x sig_y x fade for a cone); z = t0 + s, s = clamp(s_raw)
    float gsd = ga, gs = gz;
    gt0 += gz;
    const float itau = rcp_approx(tau);
    if (cone) {
        gsd = ga * e.sig_y * e.fade;
        // fade = a^4 / (a^4 + f^4), a = A / |h|^2
        const float f0 = 0.06f * tau, f4 = f0 * f0 * f0 * f0;
        const float a4 = e.a_rel * e.a_rel * e.a_rel * e.a_rel;
        const float dfade = __fdividef(4.f * e.a_rel * e.a_rel * e.a_rel * f4, (a4 + f4) * (a4 + f4));
        const float gar = ga * e.sig_d * e.sig_y * dfade;
        const float ihh = rcp_approx(e.hh);
        gA += gar * ihh;
#pragma unroll
        for (int i = 0; i < 3; ++i) gh[i] += -gar * 2.f * e.a_rel * e.h[i] * ihh;
        const float gdy = ga * e.sig_d * e.fade * e.sig_y * (1.f - e.sig_y) * itau;  // d alpha / d delta_Y
        if (gdy != 0.f) {
            adj[12] += gdy * (1.f - fabsf(e.Ye));
            const float gY = -gdy * L * (e.Ye >= 0.f ? 1.f : -1.f);
            // Y_e = g_y + u h_y, u = w s + (1 - w) s*_c, s*_c = clamp(-B / A)
            const float u = fmaf(e.w, e.s - e.sstar_c, e.sstar_c);
            gg[1] += gY;
            gh[1] += gY * u;
            const float gu_ = gY * e.h[1];
            gs += gu_ * e.w;
            const float gw = gu_ * (e.s - e.sstar_c);
            gdelta += gw * e.w * (1.f - e.w) * itau;
            float dss;
            clamp_offset(e.sstar, Rb, dss);
            const float gss = gu_ * (1.f - e.w) * dss;  // d / d s* (s* = -B / A)
            const float iA = rcp_approx(e.A);
            gB += -gss * iA;
            gA += -gss * e.sstar * iA;
        }
    }
    gdelta += gsd * e.sig_d * (1.f - e.sig_d) * itau;
    // s = clamp(s_raw), s_raw = num / den, num = C - t0 (B + r), den = t0 A - B + r
    float dcl;
    clamp_offset(e.s_raw, Rb, dcl);
    const float gsr = gs * dcl;
    const float iden = rcp_approx(e.den);
    const float gnum = gsr * iden, gden = -gsr * e.s_raw * iden;
    gC += gnum;
    gt0 += -gnum * (e.B + e.r) + gden * e.A;
    gB += -t0 * gnum - gden;
    gr += -t0 * gnum + gden;
    gA += gden * t0;
    // r = sqrt(Dp), Dp = (D + q) / 2, q = sqrt(D^2 + (tau N)^2)
    const float gDp = 0.5f * gr * rcp_approx(e.r);
    const float iq = rcp_approx(e.q);
    gD += 0.5f * gDp * fmaf(e.D, iq, 1.f);
    gN += 0.5f * gDp * (tau * tau * e.N * iq);
    // delta = D / N (skipped when sigma saturated: then delta / N may overflow)
    if (gdelta != 0.f) {
        gD += __fdividef(gdelta, e.N);
        gN += -__fdividef(gdelta * e.delta, e.N);
    }
    // N = |(Du, Dv)|
    const float gNN = __fdividef(gN, e.N);
    const float gDu = gNN * e.Du, gDv = gNN * e.Dv;
    // D = B^2 - A C
    gB += 2.f * e.B * gD;
    gA += -e.C * gD;
    gC += -e.A * gD;
    // Du = 2 B Bu - Au C - A Cu, and likewise for v
    gB += 2.f * (e.Bu * gDu + e.Bv * gDv);
    const float gBu = 2.f * e.B * gDu, gBv = 2.f * e.B * gDv;
    const float gAu = -e.C * gDu, gAv = -e.C * gDv;
    gC += -(e.Au * gDu + e.Av * gDv);
    gA += -(e.Cu * gDu + e.Cv * gDv);
    const float gCu = -e.A * gDu, gCv = -e.A * gDv;
    // quadratic forms -> ray vectors h, g, h_u, g_u, h_v, g_v
    float ghu[3], ghv[3], ggu[3], ggv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float qi = i == 1 ? qy : 0.f;
        gh[i] += 2.f * Q[i] * e.h[i] * gA + (Q[i] * e.g[i] + qi) * gB + 2.f * Q[i] * (e.hu[i] * gAu + e.hv[i] * gAv) +
                 Q[i] * (e.gu[i] * gBu + e.gv[i] * gBv);
        gg[i] += Q[i] * e.h[i] * gB + 2.f * (Q[i] * e.g[i] + qi) * gC + Q[i] * (e.hu[i] * gBu + e.hv[i] * gBv) +
                 2.f * Q[i] * (e.gu[i] * gCu + e.gv[i] * gCv);
        ghu[i] = 2.f * Q[i] * e.h[i] * gAu + (Q[i] * e.g[i] + qi) * gBu;
        ghv[i] = 2.f * Q[i] * e.h[i] * gAv + (Q[i] * e.g[i] + qi) * gBv;
        ggu[i] = Q[i] * e.h[i] * gBu + 2.f * (Q[i] * e.g[i] + qi) * gCu;
        ggv[i] = Q[i] * e.h[i] * gBv + 2.f * (Q[i] * e.g[i] + qi) * gCv;
    }
    // g_u = t0 h_u, g_v = t0 h_v
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gt0 += ggu[i] * e.hu[i] + ggv[i] * e.hv[i];
        ghu[i] = fmaf(t0, ggu[i], ghu[i]);
        ghv[i] = fmaf(t0, ggv[i], ghv[i]);
    }
    // h = a c0 + b c1 + c2, g = ex c0 + ey c1 with ex = t0 a - Cx, ey = t0 b - Cy,
    // h_u = c0 ifx, h_v = c1 ify
    const float ex = fmaf(t0, a, -r2.y), ey = fmaf(t0, b, -r2.z);
    const float c0[3] = {r0.x, r0.y, r0.z}, c1[3] = {r0.w, r1.x, r1.y};
    float gex = 0.f, gey = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        adj[i] += gh[i] * a + gg[i] * ex + ghu[i] * ifx;
        adj[3 + i] += gh[i] * b + gg[i] * ey + ghv[i] * ify;
        adj[6 + i] += gh[i];
        gex += gg[i] * c0[i];
        gey += gg[i] * c1[i];
    }
    adj[9] += -gex;
    adj[10] += -gey;
    adj[11] += gt0 + gex * a + gey * b;
}

// cone axis half-length in pixels (at least its radius in pixels) from a record:
// row k of M is column k of R over the scale s_k, so the axis (local y) is
// M_row1 / |M_row1|^2 and the scales are 1 / |M_row k|
__device__ __forceinline__ float cone_pixel_length(const float4& r0, const float4& r1, const float4& r2,
                                                   const float4& r3, float fx, float fy)
{
    const float m0[3] = {r0.x, r0.w, r1.z}, m1[3] = {r0.y, r1.x, r1.w}, m2[3] = {r0.z, r1.y, r2.x};
    const float n1 = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
    const float ax = rsqrtf(m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2]);
    const float az = rsqrtf(m2[0] * m2[0] + m2[1] * m2[1] + m2[2] * m2[2]);
    float E0[3], E1[3];
    const float C[3] = {r2.y, r2.z, r2.w};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        E0[i] = C[i] - m1[i] / n1;
        E1[i] = C[i] + m1[i] / n1;
    }
    const float du = fx * (E1[0] / E1[2] - E0[0] / E0[2]), dv = fy * (E1[1] / E1[2] - E0[1] / E0[2]);
    const float half = 0.5f * sqrtf(du * du + dv * dv);
    const float r_px = fmaxf(ax, az) * (1.f + fabsf(r3.y)) * fx / C[2];
    return fmaxf(half, r_px);
}

// Work layout of soft_backward_kernel.  A CTA of kSoftWarps warps works on one strip
// of 32 pixels of the particle's union box (row-major order) at a time; lane
// l of every warp stands for pixel l of the strip.
//  A. the warps split the primitives (j = w, w + kSoftWarps, ...): each lane
//     evaluates primitive j at its pixel (soft_eval) and, where alpha >
//     kAlphaMin, appends (alpha, z, j) to the pixel's list;
//  B. warp 0 sorts each pixel's list front to back (depth, then primitive
//     index: the forward kernel's order), composites it, forms the pixel's
//     terms of Eq. 4 and pushes dE_s back through the compositing to every
//     entry's (d alpha, d z);
//  C. the warps split the primitives again: the lanes whose pixel
//     lists primitive j push its (d alpha, d z) back to its record (soft_eval
//     again, then soft_backprop), and the warp sums the 13 adjoints.
// So a strip's chain of evaluations is split kSoftWarps ways, and the lists
// are sized for one strip (32 pixels), not for every thread of the CTA.
constexpr int kSoftWarps = kSoftThreads / 32;

// byte offsets of soft_backward_kernel's dynamic shared memory (each 16-byte aligned)
struct SoftLayout {
    size_t rec, box, L, R, uni, adj, al, zl, Tl, jl, mp, cnt, pres, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline SoftLayout soft_layout(int n, bool bwd)
{
    SoftLayout l;
    l.rec = 0;                                         // float4 [n][4]
    l.box = align16(l.rec + (size_t)n * 64);           // int4 [n]: box + margin, clipped
    l.L = align16(l.box + (size_t)n * 16);             // float [n]: cone length in pixels
    l.R = align16(l.L + (size_t)n * 4);                // float [n]: bounding radius (depth clamp)
    l.uni = align16(l.R + (size_t)n * 4);              // int [4]: union box
    l.adj = align16(l.uni + 16);                       // int64 [n][kAdj] (backward, fixed point 2^-40)
    l.al = align16(l.adj + (bwd ? (size_t)n * kAdj * 8 : 0));  // float [n][32]: alpha, then d E / d z
    l.zl = align16(l.al + (size_t)n * 32 * 4);                 // float [n][32]: depth
    l.Tl = align16(l.zl + (size_t)n * 32 * 4);                 // float [n][32]: transmittance, then d E / d alpha
    l.jl = align16(l.Tl + (bwd ? (size_t)n * 32 * 4 : 0));     // uint8 [n][32]: primitive of each entry
    l.mp = align16(l.jl + (size_t)n * 32);                     // uint8 [n][32]: entry of a primitive + 1 (backward)
    l.cnt = align16(l.mp + (bwd ? (size_t)n * 32 : 0));        // int [32]: entries of each pixel's list
    l.pres = align16(l.cnt + 32 * 4);                          // uint64: primitives listed by some pixel
    l.bytes = align16(l.pres + 8);
    return l;
}

// Set-up shared by the forward and backward kernels: particle p's records
// into shared memory, each primitive's cone length in pixels, bounding radius
// (for the depth clamp) and pixel box plus margin, and the union box
// (s_uni: u0, v0, width, height).  Ends with a CTA barrier.
__device__ __forceinline__ void soft_setup(const SoftArgs& a, int p, int tid, float4* s_rec, int4* s_box, float* s_L,
                                           float* s_R, int* s_uni)
{
    const int n = a.n_prims;
    const float4* src = a.prims + (size_t)p * n * 4;
    for (int i = tid; i < n * 4; i += kSoftThreads) s_rec[i] = src[i];
    __syncthreads();
    if (tid < n) {
        const float4 r0 = s_rec[4 * tid], r1 = s_rec[4 * tid + 1], r2 = s_rec[4 * tid + 2], r3 = s_rec[4 * tid + 3];
        s_L[tid] = r3.y < 1.5f ? cone_pixel_length(r0, r1, r2, r3, a.fx, a.fy) : 0.f;
        // bounding radius from the record's scales (1 / |row k of M|); constant in the pose
        const float sx = rsqrtf(r0.x * r0.x + r0.w * r0.w + r1.z * r1.z);
        const float sy = rsqrtf(r0.y * r0.y + r1.x * r1.x + r1.w * r1.w);
        const float sz = rsqrtf(r0.z * r0.z + r1.y * r1.y + r2.x * r2.x);
        if (r3.y < 1.5f) {
            const float rm = fmaxf(sx, sz) * (1.f + fabsf(r3.y));
            s_R[tid] = sqrtf(sy * sy + rm * rm);
        } else {
            s_R[tid] = fmaxf(sx, fmaxf(sy, sz));
        }
        int u0 = lo_i16(r3.z) - kSoftMargin, v0 = hi_i16(r3.z) - kSoftMargin;
        int u1 = lo_i16(r3.w) + kSoftMargin, v1 = hi_i16(r3.w) + kSoftMargin;
        u0 = max(u0, 0);
        v0 = max(v0, 0);
        u1 = min(u1, a.W - 1);
        v1 = min(v1, a.H - 1);
        s_box[tid] = make_int4(u0, v0, u1, v1);
    }
    __syncthreads();
    if (tid == 0) {
        int u0 = INT_MAX, v0 = INT_MAX, u1 = INT_MIN, v1 = INT_MIN;
        for (int j = 0; j < n; ++j) {
            const int4 bx = s_box[j];
            if (bx.x > bx.z || bx.y > bx.w) continue;
            u0 = min(u0, bx.x);
            v0 = min(v0, bx.y);
            u1 = max(u1, bx.z);
            v1 = max(v1, bx.w);
        }
        s_uni[0] = u0;
        s_uni[1] = v0;
        s_uni[2] = u1 >= u0 ? u1 - u0 + 1 : 0;
        s_uni[3] = v1 >= v0 ? v1 - v0 + 1 : 0;
    }
    __syncthreads();
}

// A covered pixel's smoothed terms of Eq. 4 (reading R1) from its composited
// depth zt: t_hit and t_miss (the depth term where the hand is / is not
// rendered), m (the smoothed r_m test), and the derivatives the backward pass
// needs: dsmin = d smin / d diff, dm = d m / d diff.
__device__ __forceinline__ void soft_pixel_terms(float od, bool S, float zt, float d_m, float d_M, float tm,
                                                 float& t_hit, float& m, float& t_miss, float& dd, float& diff,
                                                 float& dsmin, float& dm)
{
    const bool valid = S && od > 0.f;
    dd = od - zt;
    diff = sqrt_approx(fmaf(dd, dd, tm * tm));
    const float itm = rcp_approx(tm);
    dsmin = 0.f;
    dm = 0.f;
    if (valid) {
        const float m0 = fminf(diff, d_M);
        t_hit = m0 - tm * __logf(__expf(-(diff - m0) * itm) + __expf(-(d_M - m0) * itm));
        dsmin = sigm((d_M - diff) * itm);
        m = sigm((d_m - diff) * itm);
        dm = -m * (1.f - m) * itm;
        t_miss = d_M;
    } else {
        t_hit = S ? 0.f : d_M;
        m = 1.f;
        t_miss = 0.f;
    }
}

__global__ void __launch_bounds__(kSoftThreads, 5) soft_backward_kernel(const SoftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n_prims;
    const int p = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SoftLayout lay = soft_layout(n, true);
    float4* s_rec = reinterpret_cast<float4*>(smem + lay.rec);
    int4* s_box = reinterpret_cast<int4*>(smem + lay.box);
    float* s_L = reinterpret_cast<float*>(smem + lay.L);
    float* s_R = reinterpret_cast<float*>(smem + lay.R);
    int* s_uni = reinterpret_cast<int*>(smem + lay.uni);
    unsigned long long* s_adj = reinterpret_cast<unsigned long long*>(smem + lay.adj);
    float* s_al = reinterpret_cast<float*>(smem + lay.al);
    float* s_zl = reinterpret_cast<float*>(smem + lay.zl);
    float* s_Tl = reinterpret_cast<float*>(smem + lay.Tl);
    uint8_t* s_jl = smem + lay.jl;
    uint8_t* s_mp = smem + lay.mp;
    int* s_cnt = reinterpret_cast<int*>(smem + lay.cnt);
    unsigned long long* s_pres = reinterpret_cast<unsigned long long*>(smem + lay.pres);

    for (int i = tid; i < n * kAdj; i += kSoftThreads) s_adj[i] = 0ull;
    for (int i = tid; i < n * 32; i += kSoftThreads) s_mp[i] = 0;
    if (tid < 32) s_cnt[tid] = 0;
    soft_setup(a, p, tid, s_rec, s_box, s_L, s_R, s_uni);
    const int bu0 = s_uni[0], bv0 = s_uni[1], bw = s_uni[2], bh = s_uni[3];
    const int npix = bw * bh;

    // d E_s / d (sum t, sum and, sum or) from the forward pass's sums
    float G_t = 0.f, G_and = 0.f, G_or = 0.f;
    {
        const float St = a.sums[3 * p], Sa = a.sums[3 * p + 1], So = a.sums[3 * p + 2];
        if (So > 0.f) {
            const float den = Sa + So;
            G_t = 1.f / So;
            G_and = -2.f * a.lambda * So / (den * den);
            G_or = -St / (So * So) + 2.f * a.lambda * Sa / (den * den);
        }
    }
    const float tm = a.tau_mm;
    for (int base = blockIdx.x * 32; base < npix; base += gridDim.x * 32) {
        // lane l of every warp stands for pixel base + l of the union box
        const int i = base + lane;
        const bool pix = i < npix;
        const int v = pix ? bv0 + i / bw : 0, u = pix ? bu0 + i % bw : 0;
        const float ra = fmaf((float)u, a.inv_fx, a.off_x);
        const float rb = fmaf((float)v, a.inv_fy, a.off_y);
        // A: this warp's primitives at the lane's pixel, appended to its list
        for (int j = warp; j < n; j += kSoftWarps) {
            const int4 bx = s_box[j];
            if (!pix || u < bx.x || u > bx.z || v < bx.y || v > bx.w) continue;
            SoftPrimEval e;
            soft_eval(s_rec[4 * j], s_rec[4 * j + 1], s_rec[4 * j + 2], s_rec[4 * j + 3], s_L[j], s_R[j], ra, rb,
                      a.inv_fx, a.inv_fy, a.tau, e);
            if (!(e.alpha > kAlphaMin)) continue;
            const int k = atomicAdd(&s_cnt[lane], 1);
            s_al[k * 32 + lane] = e.alpha;
            s_zl[k * 32 + lane] = e.z;
            s_jl[k * 32 + lane] = (uint8_t)j;
        }
        __syncthreads();
        // B: warp 0 sorts, composites, forms the pixel's terms and pushes dE_s back
        // through the compositing (lane = pixel)
        if (warp == 0) {
            const int cnt = s_cnt[lane];
            // front to back: depth, then primitive index (insertion sort of a short list)
            for (int k = 1; k < cnt; ++k) {
                const float ak = s_al[k * 32 + lane], zk = s_zl[k * 32 + lane];
                const uint8_t jk = s_jl[k * 32 + lane];
                int m = k;
                while (m > 0) {
                    const float zm = s_zl[(m - 1) * 32 + lane];
                    const uint8_t jm = s_jl[(m - 1) * 32 + lane];
                    if (!(zm > zk || (zm == zk && jm > jk))) break;
                    s_al[m * 32 + lane] = s_al[(m - 1) * 32 + lane];
                    s_zl[m * 32 + lane] = zm;
                    s_jl[m * 32 + lane] = jm;
                    --m;
                }
                s_al[m * 32 + lane] = ak;
                s_zl[m * 32 + lane] = zk;
                s_jl[m * 32 + lane] = jk;
            }
            uint64_t present = 0ull;  // primitives in this pixel's list
            float T = 1.f, Nz = 0.f;
            for (int k = 0; k < cnt; ++k) {
                const float al = s_al[k * 32 + lane];
                s_Tl[k * 32 + lane] = T;
                Nz = fmaf(T * al, s_zl[k * 32 + lane], Nz);
                T *= 1.f - al;
            }
            const float c = 1.f - T;
            if (cnt > 0 && c > 0.f) {
                const float zt = __fdividef(Nz, c);
                const float od = a.depth_f32
                                     ? reinterpret_cast<const float*>(a.depth + (size_t)v * a.depth_pitch)[u]
                                     : (float)reinterpret_cast<const uint16_t*>(a.depth + (size_t)v * a.depth_pitch)[u];
                const bool S = a.skin[(size_t)v * a.skin_pitch + u] != 0;
                const bool valid = S && od > 0.f;
                float t_hit, m, t_miss, dd, diff, dsmin, dm;
                soft_pixel_terms(od, S, zt, a.d_m, a.d_M, tm, t_hit, m, t_miss, dd, diff, dsmin, dm);
                {
                    // per-entry adjoints of alpha and z through the compositing (back to front);
                    // each entry's (d alpha, d z) replaces its (T, alpha) in place
                    const float gr_ = S ? G_and : G_or;
                    const float gc = G_t * (t_hit - t_miss) + gr_ * m;
                    const float gzt = valid ? (G_t * c * dsmin + gr_ * c * dm) * __fdividef(-dd, diff) : 0.f;
                    const float ic = rcp_approx(c);
                    const float gN = gzt * ic;
                    const float gct = gc - gzt * zt * ic;
                    float Rsuf = 0.f, Psuf = 1.f;
                    for (int k = cnt - 1; k >= 0; --k) {
                        const float al = s_al[k * 32 + lane], zk = s_zl[k * 32 + lane];
                        const float Tk = s_Tl[k * 32 + lane];
                        s_Tl[k * 32 + lane] = gN * Tk * (zk - Rsuf) + gct * Tk * Psuf;  // d E / d alpha
                        s_al[k * 32 + lane] = gN * Tk * al;                            // d E / d z
                        const int j = s_jl[k * 32 + lane];
                        s_mp[j * 32 + lane] = (uint8_t)(k + 1);
                        present |= 1ull << j;
                        Rsuf = fmaf(al, zk, (1.f - al) * Rsuf);
                        Psuf *= 1.f - al;
                    }
                }
            }
            {
                const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)present);
                const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(present >> 32));
                if (lane == 0) *s_pres = ((unsigned long long)hi << 32) | lo;
            }
            s_cnt[lane] = 0;  // the list is consumed (the reverse pass finds entries through s_mp)
        }
        __syncthreads();
        {
            // C: the warps split the primitives again; the lanes whose pixel lists
            // primitive j push its (d alpha, d z) back to its record; the warp sums
            // the 13 adjoints in fixed point and 13 lanes add them to the CTA's
            const uint64_t pres = *s_pres;
            for (int j = warp; j < n; j += kSoftWarps) {
                if (!((pres >> j) & 1ull)) continue;
                const int k = (int)s_mp[j * 32 + lane] - 1;
                long long f[kAdj];
#pragma unroll
                for (int q = 0; q < kAdj; ++q) f[q] = 0;
                if (k >= 0) {
                    s_mp[j * 32 + lane] = 0;
                    const float ga = s_Tl[k * 32 + lane], gz = s_al[k * 32 + lane];
                    const float4 r0 = s_rec[4 * j], r1 = s_rec[4 * j + 1], r2 = s_rec[4 * j + 2], r3 = s_rec[4 * j + 3];
                    SoftPrimEval e;
                    soft_eval(r0, r1, r2, r3, s_L[j], s_R[j], ra, rb, a.inv_fx, a.inv_fy, a.tau, e);
                    float adj[kAdj];
#pragma unroll
                    for (int q = 0; q < kAdj; ++q) adj[q] = 0.f;
                    soft_backprop(r0, r1, r2, r3, s_L[j], s_R[j], ra, rb, a.inv_fx, a.inv_fy, a.tau, e, ga, gz, adj);
#pragma unroll
                    for (int q = 0; q < kAdj; ++q) f[q] = adj_to_fix(adj[q]);
                }
                int3 mine = make_int3(0, 0, 0);  // lane q keeps adjoint q's limb sums
#pragma unroll
                for (int q = 0; q < kAdj; ++q) {
                    const int3 sq = warp_sum_limbs(f[q]);
                    if (lane == q) mine = sq;
                }
                const long long tot = fix_from_limbs(mine);
                if (lane < kAdj && tot != 0) atomicAdd(&s_adj[j * kAdj + lane], (unsigned long long)tot);
            }
            __syncthreads();  // the lists are free for the next strip
        }
    }

    __syncthreads();
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.adj) + (size_t)p * n * kAdj;
    for (int i = tid; i < n * kAdj; i += kSoftThreads)
        if (s_adj[i] != 0ull) atomicAdd(&dst[i], s_adj[i]);
}

// The forward pass (E_s and its sums) with every warp on its own: a CTA takes
// 128-pixel pieces of the particle's union box (k, k + K, ... over the
// particle's K CTAs), each lane walks its pixel's primitives, keeps its list
// front to back in shared memory (sorted on insertion: depth, then primitive
// index, the order soft_backward_kernel sorts in) and composites it.  No CTA
// barrier per piece: where the box holds many pixels per CTA this is faster
// than the backward kernel's split of each strip over the warps.
struct SoftFwdLayout {
    size_t rec, box, L, R, uni, al, zl, bytes;
};

__host__ __device__ inline SoftFwdLayout soft_fwd_layout(int n)
{
    SoftFwdLayout l;
    l.rec = 0;                                          // float4 [n][4]
    l.box = align16(l.rec + (size_t)n * 64);            // int4 [n]: box + margin, clipped
    l.L = align16(l.box + (size_t)n * 16);              // float [n]: cone length in pixels
    l.R = align16(l.L + (size_t)n * 4);                 // float [n]: bounding radius (depth clamp)
    l.uni = align16(l.R + (size_t)n * 4);               // int [4]: union box
    l.al = align16(l.uni + 16);                         // float [n][threads]: alpha
    l.zl = align16(l.al + (size_t)n * kSoftThreads * 4);  // float [n][threads]: depth
    l.bytes = align16(l.zl + (size_t)n * kSoftThreads * 4);
    return l;
}

__global__ void __launch_bounds__(kSoftThreads) soft_forward_kernel(const SoftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n_prims;
    const int p = blockIdx.y, tid = threadIdx.x;
    const SoftFwdLayout lay = soft_fwd_layout(n);
    float4* s_rec = reinterpret_cast<float4*>(smem + lay.rec);
    int4* s_box = reinterpret_cast<int4*>(smem + lay.box);
    float* s_L = reinterpret_cast<float*>(smem + lay.L);
    float* s_R = reinterpret_cast<float*>(smem + lay.R);
    int* s_uni = reinterpret_cast<int*>(smem + lay.uni);
    float* s_al = reinterpret_cast<float*>(smem + lay.al);
    float* s_zl = reinterpret_cast<float*>(smem + lay.zl);
    soft_setup(a, p, tid, s_rec, s_box, s_L, s_R, s_uni);
    const int bu0 = s_uni[0], bv0 = s_uni[1], bw = s_uni[2], bh = s_uni[3];
    const int npix = bw * bh;

    long long acc_t = 0, acc_a = 0, acc_o = 0;
    const float tm = a.tau_mm;
    for (int i = blockIdx.x * kSoftThreads + tid; i < npix; i += gridDim.x * kSoftThreads) {
        const int v = bv0 + i / bw, u = bu0 + i % bw;
        const float ra = fmaf((float)u, a.inv_fx, a.off_x);
        const float rb = fmaf((float)v, a.inv_fy, a.off_y);
        int cnt = 0;
        for (int j = 0; j < n; ++j) {
            const int4 bx = s_box[j];
            if (u < bx.x || u > bx.z || v < bx.y || v > bx.w) continue;
            SoftPrimEval e;
            soft_eval(s_rec[4 * j], s_rec[4 * j + 1], s_rec[4 * j + 2], s_rec[4 * j + 3], s_L[j], s_R[j], ra, rb,
                      a.inv_fx, a.inv_fy, a.tau, e);
            if (!(e.alpha > kAlphaMin)) continue;
            // insert, keeping the list sorted front to back (depth, then primitive index)
            int k = cnt++;
            while (k > 0 && s_zl[(k - 1) * kSoftThreads + tid] > e.z) {
                s_al[k * kSoftThreads + tid] = s_al[(k - 1) * kSoftThreads + tid];
                s_zl[k * kSoftThreads + tid] = s_zl[(k - 1) * kSoftThreads + tid];
                --k;
            }
            s_al[k * kSoftThreads + tid] = e.alpha;
            s_zl[k * kSoftThreads + tid] = e.z;
        }
        if (cnt == 0) continue;
        float T = 1.f, Nz = 0.f;
        for (int k = 0; k < cnt; ++k) {
            const float al = s_al[k * kSoftThreads + tid];
            Nz = fmaf(T * al, s_zl[k * kSoftThreads + tid], Nz);
            T *= 1.f - al;
        }
        const float c = 1.f - T;
        if (!(c > 0.f)) continue;
        const float zt = __fdividef(Nz, c);
        const float od = a.depth_f32 ? reinterpret_cast<const float*>(a.depth + (size_t)v * a.depth_pitch)[u]
                                     : (float)reinterpret_cast<const uint16_t*>(a.depth + (size_t)v * a.depth_pitch)[u];
        const bool S = a.skin[(size_t)v * a.skin_pitch + u] != 0;
        float t_hit, m, t_miss, dd, diff, dsmin, dm;
        soft_pixel_terms(od, S, zt, a.d_m, a.d_M, tm, t_hit, m, t_miss, dd, diff, dsmin, dm);
        // |c (t_hit - t_miss)| <= d_M < 127 and c m <= 1: 32-bit fixed point per pixel
        acc_t += (long long)__float2int_rn(c * (t_hit - t_miss) * kFix);
        if (S)
            acc_a += (long long)__float2int_rn(c * m * kFix);
        else
            acc_o += (long long)__float2int_rn(c * m * kFix);
    }

    // CTA sums, then the particle's last CTA forms E_s
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_t += __shfl_xor_sync(0xffffffffu, acc_t, o);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
        acc_o += __shfl_xor_sync(0xffffffffu, acc_o, o);
    }
    __shared__ long long red[3][kSoftThreads / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red[0][warp] = acc_t;
        red[1][warp] = acc_a;
        red[2][warp] = acc_o;
    }
    __syncthreads();
    if (tid != 0) return;
    for (int w = 1; w < kSoftThreads / 32; ++w) {
        acc_t += red[0][w];
        acc_a += red[1][w];
        acc_o += red[2][w];
    }
    SoftWork* wk = a.work + p;
    if (acc_t) atomicAdd(reinterpret_cast<unsigned long long*>(&wk->t), (unsigned long long)acc_t);
    if (acc_a) atomicAdd(reinterpret_cast<unsigned long long*>(&wk->a), (unsigned long long)acc_a);
    if (acc_o) atomicAdd(reinterpret_cast<unsigned long long*>(&wk->o), (unsigned long long)acc_o);
    uint32_t done;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(done) : "l"(&wk->exited) : "memory");
    if (done != gridDim.x - 1) return;
    const long long tf = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&wk->t), 0ull);
    const long long af = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&wk->a), 0ull);
    const long long of = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&wk->o), 0ull);
    const uint32_t n_valid = a.stats[0], n_skin = a.stats[1];
    const float St = (float)tf * (1.f / kFix) + a.d_M * (float)n_valid;
    const float Sa = (float)af * (1.f / kFix);
    const float So = (float)of * (1.f / kFix) + (float)n_skin;
    const float D = So > 0.f ? St / So + a.lambda * (1.f - 2.f * Sa / (Sa + So)) : a.lambda;
    a.E[p] = D + a.lambda_k * a.kc[p];
    if (a.sums) {
        a.sums[3 * p] = St;
        a.sums[3 * p + 1] = Sa;
        a.sums[3 * p + 2] = So;
    }
    *wk = SoftWork{};
}

// ---- pose gradient: record adjoints -> d E_s / d pose ------------------------------

// fixed-point scale of the penetration adjoint d pen / d c (sums of unit vectors)
constexpr float kPenGradFix = 4294967296.0f;  // 2^32

// Model: DevModelCore for the paper's kc, DevModel when the kc variant needs
// the collision data (then the adjoint of the interpenetration term is added)
constexpr int kGradThreads = 256;  // threads of pose_grad_kernel (one CTA per particle)

template <class Model>
__global__ void __launch_bounds__(kGradThreads) pose_grad_kernel(const __grid_constant__ Model model_param, const GradArgs a)
{
    __shared__ FkShared sh;
    __shared__ long long s_gc[kMaxProxies * 3];  // d pen / d (proxy centre), fixed point
    __shared__ CollideSmem<Model> s_col;
    extern __shared__ float s_tan[];  // [26][n_bones][12]: dR (9), dP (3) of every bone for every DOF,
                                      // then [n_prims][26]: each primitive's contribution,
                                      // then [n_prims][13]: its adjoints
    fk_load_model(sh, model_param);
    const int p = blockIdx.x, t = threadIdx.x;
    const float* pose = a.poses + (size_t)p * kNdof;
    const CollideShared* mp = collide_load(s_col, model_param);
    fk_particle(sh, mp, pose, make_float4(a.fx, a.fy, a.cx, a.cy), a.prims + (size_t)p * sh.model.n_prims * 4, a.kc + p,
                a.status);
    __syncthreads();
    const int nb = sh.model.n_bones, np = sh.model.n_prims;
    const bool pen_term = mp && sh.model.kc_variant != HS_KC_ABDUCTION;  // (uniform over the CTA)
    if (pen_term) {
        // d pen / d c_i = sum over the penetrating pairs (i, j) of -(c_i - c_j) / |c_i - c_j|
        // (and + for c_j), the same pairs and the same test as the sum in FK;
        // accumulated in fixed point so that the order of the pairs does not matter
        for (int i = t; i < 3 * sh.model.n_proxies; i += kGradThreads) s_gc[i] = 0ll;
        __syncthreads();
        for (int k = t; k < sh.model.n_pairs; k += kGradThreads) {
            const uint32_t ij = mp->pairs[k];
            const int i = ij & 0xffu, j = ij >> 8;
            const float4 ci = sh.pc[i], cj = sh.pc[j];
            const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)), rr = ci.w + cj.w;
            if (d2 < rr * rr) {
                const float d = sqrtf(d2);
                if (rr - d > 0.f && d > 0.f) {
                    const float id = 1.f / d;
                    const long long ux = __float2ll_rn(dx * id * kPenGradFix);
                    const long long uy = __float2ll_rn(dy * id * kPenGradFix);
                    const long long uz = __float2ll_rn(dz * id * kPenGradFix);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * i]), (unsigned long long)(-ux));
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * i + 1]), (unsigned long long)(-uy));
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * i + 2]), (unsigned long long)(-uz));
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * j]), (unsigned long long)ux);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * j + 1]), (unsigned long long)uy);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&s_gc[3 * j + 2]), (unsigned long long)uz);
                }
            }
        }
    }
    float* s_contrib = s_tan + (size_t)kNdof * nb * 12;
    // Tangents of every bone frame for every pose parameter, each (parameter d,
    // bone k) on its own thread.  An angle turns everything below its joint
    // about a world axis w through the joint's position J, so
    //   dR_k / dq_d = [w]x R_k,  dP_k / dq_d = w x (P_k - J),
    // summed over the joints of bone k's path that q_d drives (the palm's
    // three angles drive every bone; the translation q_0..2 drives no frame).
    // The axes, from the global frames FK formed (G = U Rz Rx for a finger
    // joint with U = R_parent rest; G = Mount Rz Ry Rx for the palm,
    // Mount = diag(1, -1, -1)):
    //   finger z angle: U e_z;  finger x angle: U Rz e_x = G e_x;
    //   palm q5: Mount e_z;  q4: Mount Rz(q5) e_y;  q3: Mount Rz Ry e_x = G_palm e_x.
    for (int i = t; i < kNdof * nb; i += kGradThreads) {
        const int d = i / nb, k = i - d * nb;
        const DevBone& Bk = sh.model.bones[k];
        float W[3] = {0.f, 0.f, 0.f}, V[3] = {0.f, 0.f, 0.f};  // sum of axes w, sum of w x J
        if (d >= 3 && d <= 5) {
            // the palm's angles; its joint is the wrist (J = 0)
            if (d == 5) {
                W[2] = -1.f;
            } else if (d == 4) {
                W[0] = -sh.sn[5];
                W[1] = -sh.cs[5];
            } else {
                W[0] = sh.bR[0][0];
                W[1] = sh.bR[0][3];
                W[2] = sh.bR[0][6];
            }
        } else if (d >= 6) {
            for (int lv = 1; lv <= Bk.depth; ++lv) {
                const int b = Bk.anc[lv];
                const DevBone& B = sh.model.bones[b];
                if (B.dof_z != d && B.dof_x != d) continue;
                float w[3];
                if (B.dof_z == d) {
                    const float* Rp = sh.bR[B.parent];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        w[r] = fmaf(Rp[3 * r], B.rest[2], fmaf(Rp[3 * r + 1], B.rest[5], Rp[3 * r + 2] * B.rest[8]));
                } else {
#pragma unroll
                    for (int r = 0; r < 3; ++r) w[r] = sh.bR[b][3 * r];
                }
                const float* J = sh.bP[b];
                W[0] += w[0];
                W[1] += w[1];
                W[2] += w[2];
                V[0] += w[1] * J[2] - w[2] * J[1];
                V[1] += w[2] * J[0] - w[0] * J[2];
                V[2] += w[0] * J[1] - w[1] * J[0];
            }
        }
        float* dR = s_tan + ((size_t)d * nb + k) * 12;
        float* dP = dR + 9;
        const float* R = sh.bR[k];
        const float* P = sh.bP[k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // column c of dR = W x (column c of R)
            const float x = R[c], y = R[3 + c], z = R[6 + c];
            dR[c] = W[1] * z - W[2] * y;
            dR[3 + c] = W[2] * x - W[0] * z;
            dR[6 + c] = W[0] * y - W[1] * x;
        }
        dP[0] = W[1] * P[2] - W[2] * P[1] - V[0];
        dP[1] = W[2] * P[0] - W[0] * P[2] - V[1];
        dP[2] = W[0] * P[1] - W[1] * P[0] - V[2];
    }
    // the primitives' adjoints from fixed point (and their slots cleared for
    // the next backward pass)
    long long* adjp = a.adj + (size_t)p * np * kAdj;
    float* s_ad = s_contrib + (size_t)np * kNdof;  // [n_prims][13]
    for (int i = t; i < np * kAdj; i += kGradThreads) s_ad[i] = adj_from_fix(adjp[i]);
    __syncthreads();
    for (int i = t; i < np * kAdj; i += kGradThreads) adjp[i] = 0ll;  // ready for the next backward pass
    // every (primitive, parameter) contribution on its own thread
    for (int jk = t; jk < np * kNdof; jk += kGradThreads) {
        const int j = jk / kNdof, k = jk - j * kNdof;
        const DevPrimDesc& D = sh.model.prims[j];
        float ad[kAdj];
#pragma unroll
        for (int q = 0; q < kAdj; ++q) ad[q] = s_ad[j * kAdj + q];
        const float* R = sh.bR[D.bone];
        const float* O = sh.bP[D.bone];
        const bool cone = D.kind == HS_PRIM_ECONE;
        float C[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            C[i] = sh.q[i] + R[3 * i] * D.center[0] + R[3 * i + 1] * D.center[1] + R[3 * i + 2] * D.center[2] + O[i];
        // cone length in pixels: ends C -+ hl R[:,1], branch of the max taken on these values
        float E0[3], E1[3], du = 0.f, dv = 0.f, half = 0.f, r_px = 0.f;
        const float hl = D.dims[2];
        if (cone) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                E0[i] = C[i] - hl * R[3 * i + 1];
                E1[i] = C[i] + hl * R[3 * i + 1];
            }
            du = a.fx * (E1[0] / E1[2] - E0[0] / E0[2]);
            dv = a.fy * (E1[1] / E1[2] - E0[1] / E0[2]);
            half = 0.5f * sqrtf(du * du + dv * dv);
            r_px = fmaxf(D.dims[0], D.dims[1]) * (1.f + fabsf(D.dims[3])) * a.fx / C[2];
        }
        {
            const float* dR = s_tan + ((size_t)k * nb + D.bone) * 12;
            const float* dP = dR + 9;
            float acc = 0.f;
            // record M: rec[3c + i] = R[3c + i] inv_s_i
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int i = 0; i < 3; ++i) acc = fmaf(ad[3 * c + i], dR[3 * c + i] * D.inv_s[i], acc);
            float dC[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dC[i] = (k == i ? 1.f : 0.f) + dR[3 * i] * D.center[0] + dR[3 * i + 1] * D.center[1] +
                        dR[3 * i + 2] * D.center[2] + dP[i];
                acc = fmaf(ad[9 + i], dC[i], acc);
            }
            if (cone && ad[12] != 0.f) {
                float dL;
                if (half >= r_px) {
                    float dE0[3], dE1[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        dE0[i] = dC[i] - hl * dR[3 * i + 1];
                        dE1[i] = dC[i] + hl * dR[3 * i + 1];
                    }
                    const float ddu = a.fx * ((dE1[0] * E1[2] - E1[0] * dE1[2]) / (E1[2] * E1[2]) -
                                              (dE0[0] * E0[2] - E0[0] * dE0[2]) / (E0[2] * E0[2]));
                    const float ddv = a.fy * ((dE1[1] * E1[2] - E1[1] * dE1[2]) / (E1[2] * E1[2]) -
                                              (dE0[1] * E0[2] - E0[1] * dE0[2]) / (E0[2] * E0[2]));
                    dL = half > 0.f ? 0.25f * (du * ddu + dv * ddv) / half : 0.f;
                } else {
                    dL = -r_px * dC[2] / C[2];
                }
                acc = fmaf(ad[12], dL, acc);
            }
            s_contrib[j * kNdof + k] = acc;
        }
    }
    __syncthreads();
    if (t < kNdof) {
        float g = 0.f;
        for (int j = 0; j < np; ++j) g += s_contrib[j * kNdof + t];  // fixed order: deterministic
        // kc(h) = sum over (11, 15), (15, 19), (19, 23) of max(q_b - q_a, 0)
        // (not part of kc under HS_KC_PEN)
        if (sh.model.kc_variant != HS_KC_PEN) {
            const int pa[3] = {11, 15, 19}, pb[3] = {15, 19, 23};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (sh.q[pa[i]] - sh.q[pb[i]] < 0.f) {
                    if (t == pa[i]) g -= a.lambda_k;
                    if (t == pb[i]) g += a.lambda_k;
                }
            }
        }
        if (pen_term) {
            // + lambda_k w d pen / d q_t = sum_i (d pen / d c_i) . (dR_b local_i + dP_b),
            // b the proxy's bone, with the bone tangents of DOF t formed above
            float gp = 0.f;
            for (int i = 0; i < sh.model.n_proxies; ++i) {
                const DevProxy& X = mp->proxies[i];
                const float* dR = s_tan + ((size_t)t * nb + X.bone) * 12;
                const float* dP = dR + 9;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float dc = fmaf(dR[3 * c], X.local[0], fmaf(dR[3 * c + 1], X.local[1],
                                                                         fmaf(dR[3 * c + 2], X.local[2], dP[c])));
                    gp = fmaf(__ll2float_rn(s_gc[3 * i + c]) * (1.f / kPenGradFix), dc, gp);
                }
            }
            g = fmaf(a.lambda_k * sh.model.pen_weight, gp, g);
        }
        // the FK clamps the pose to the limits: no gradient outside them
        const float x = pose[t];
        if (!(x >= sh.model.lo[t] && x <= sh.model.hi[t])) g = 0.f;
        a.grad[(size_t)p * kNdof + t] = g;
    }
}

// ---- launchers ----------------------------------------------------------------------

static constexpr int kMaxDevicesSoft = 64;
static constexpr int kMaxSoftCtas = 256;  // CTAs per particle at most in the automatic choice

// kern: the forward or the backward kernel; smem(n): its dynamic shared memory
// for n primitives; opted: its per-device flag of the shared-memory opt-in
template <class Kernel, class Smem>
static cudaError_t launch_soft_impl(Kernel kern, Smem smem_of, std::atomic<uint32_t>* opted, const SoftArgs& args,
                                   cudaStream_t stream)
{
    const size_t smem = smem_of(args.n_prims);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevicesSoft) return cudaErrorInvalidDevice;
    if (!opted[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(kMaxPrims));
        if (e != cudaSuccess) return e;
        opted[dev].store(1u, std::memory_order_release);
    }
    int K = args.K;
    if (K == 0) {
        // CTAs per particle: one resident wave of this kernel in all (a grid a
        // little over one wave would take about two waves' time); each CTA takes
        // the particle's 32-pixel strips in a grid-stride loop
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSoftThreads, smem);
        if (e != cudaSuccess) return e;
        K = args.P > 0 ? sms * per_sm / args.P : 1;
        K = K < 1 ? 1 : (K > kMaxSoftCtas ? kMaxSoftCtas : K);
    }
    kern<<<dim3(K, args.P), kSoftThreads, smem, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_soft(bool backward, const SoftArgs& args, cudaStream_t stream)
{
    static std::atomic<uint32_t> opted[2][kMaxDevicesSoft];
    if (backward)
        return launch_soft_impl(soft_backward_kernel, [](int n) { return soft_layout(n, true).bytes; }, opted[1], args,
                                stream);
    return launch_soft_impl(soft_forward_kernel, [](int n) { return soft_fwd_layout(n).bytes; }, opted[0], args,
                            stream);
}

cudaError_t launch_pose_grad(const DevModel& model, const GradArgs& args, cudaStream_t stream)
{
    const size_t smem =
        ((size_t)kNdof * model.n_bones * 12 + (size_t)model.n_prims * (kNdof + kAdj)) * sizeof(float);
    static std::atomic<uint32_t> opted[2][64];
    const int smem_max = (kNdof * kMaxBones * 12 + kMaxPrims * (kNdof + kAdj)) * 4;
    if (model.kc_variant == HS_KC_ABDUCTION) {
        const cudaError_t e = opt_in_dynamic_smem(pose_grad_kernel<DevModelCore>, smem_max, opted[0]);
        if (e != cudaSuccess) return e;
        pose_grad_kernel<DevModelCore><<<args.P, kGradThreads, smem, stream>>>(static_cast<const DevModelCore&>(model), args);
    } else {
        const cudaError_t e = opt_in_dynamic_smem(pose_grad_kernel<DevModel>, smem_max, opted[1]);
        if (e != cudaSuccess) return e;
        pose_grad_kernel<DevModel><<<args.P, kGradThreads, smem, stream>>>(model, args);
    }
    return cudaGetLastError();
}

}  // namespace hs
