// hs_fk.cuh -- forward kinematics of one particle by one 64-thread CTA
// (Eq. 1-3, Section II.A; Tables 1-2), shared by pose_fk and the fused swarm
// step.  Threads 0..25 clamp the pose; one thread per bone builds its local
// rotation; the tree is composed level by level in shared memory; one thread
// per primitive emits the 64-byte camera-space record (M = S^-1 R^T columns,
// centre C, visible caps, kappa, conservative pixel box) that the renderer
// intersects rays against.  kc(h) (after Eq. 5) is computed from the clamped
// pose.
#pragma once

#include <cfloat>
#include <cstddef>
#include <type_traits>

#include "hs_args.cuh"

namespace hs {

constexpr float kPenFix = 1048576.0f;  // fixed-point scale of the penetration sum (2^20 per mm)

struct FkShared {
    DevModelCore model;
    float4 pc[kMaxProxies];          // collision proxies relative to the wrist: centre, radius
    unsigned long long pen_fix;      // their penetration sum, fixed point
    float q[kNdof];
    float sn[kNdof], cs[kNdof];  // sin and cos of the clamped angles
    float lR[kMaxBones][9];
    float bR[kMaxBones][9];
    float bP[kMaxBones][3];
    int bad;
};

__device__ __forceinline__ void mat3_mul(const float* a, const float* b, float* c)
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            c[3 * r + k] = fmaf(a[3 * r], b[k], fmaf(a[3 * r + 1], b[3 + k], a[3 * r + 2] * b[6 + k]));
}

// local rotation of the palm: diag(1, -1, -1) Rz(q5) Ry(q4) Rx(q3), from the
// sines and cosines of the angles
__device__ __forceinline__ void palm_local(const float* sn, const float* cs, float* R)
{
    const float sx = sn[3], cx = cs[3], sy = sn[4], cy = cs[4], sz = sn[5], cz = cs[5];
    const float Rz[9] = {cz, -sz, 0.f, sz, cz, 0.f, 0.f, 0.f, 1.f};
    const float Ry[9] = {cy, 0.f, sy, 0.f, 1.f, 0.f, -sy, 0.f, cy};
    const float Rx[9] = {1.f, 0.f, 0.f, 0.f, cx, -sx, 0.f, sx, cx};
    float T[9];
    mat3_mul(Rz, Ry, T);
    mat3_mul(T, Rx, R);
#pragma unroll
    for (int k = 3; k < 9; ++k) R[k] = -R[k];
}

// local rotation of a finger bone: rest Rz(theta_z) Rx(theta_x) (a missing
// degree of freedom is a zero angle)
__device__ __forceinline__ void bone_local(const DevBone& B, const float* sn, const float* cs, float* R)
{
    float sz = 0.f, cz = 1.f, sx = 0.f, cx = 1.f;
    if (B.dof_z >= 0) {
        sz = sn[B.dof_z];
        cz = cs[B.dof_z];
    }
    if (B.dof_x >= 0) {
        sx = sn[B.dof_x];
        cx = cs[B.dof_x];
    }
    const float ZX[9] = {cz, -sz * cx, sz * sx, sz, cz * cx, -cz * sx, 0.f, sx, cx};  // Rz Rx
    mat3_mul(B.rest, ZX, R);
}

__device__ __forceinline__ int clamp_i16(float v)
{
    return (int)fminf(fmaxf(v, -32767.0f), 32767.0f);
}

// one coalesced copy of the model (a by-value launch parameter) into shared
// memory; later accesses use thread-dependent bone / primitive indices
__device__ __forceinline__ void fk_load_model(FkShared& sh, const DevModelCore& mp)
{
    // only the used part: header and limits, then the n_prims primitives and n_bones bones, in
    // 8-byte words (every lane's read of the parameter is a constant-cache request of its own,
    // so wider words mean fewer requests)
    static_assert(offsetof(DevModelCore, prims) % 8 == 0 && offsetof(DevModelCore, bones) % 8 == 0 &&
                      sizeof(DevPrimDesc) % 8 == 0 && sizeof(DevBone) % 8 == 0,
                  "the model copy moves 8-byte words");
    const uint2* srcw = reinterpret_cast<const uint2*>(&mp);
    uint2* dstw = reinterpret_cast<uint2*>(&sh.model);
    constexpr int head = (int)(offsetof(DevModelCore, prims) / 8);
    const int prim_end = head + mp.n_prims * (int)(sizeof(DevPrimDesc) / 8);
    constexpr int bones0 = (int)(offsetof(DevModelCore, bones) / 8);
    const int bone_words = mp.n_bones * (int)(sizeof(DevBone) / 8);
#pragma unroll 1
    for (int i = threadIdx.x; i < prim_end; i += blockDim.x) dstw[i] = srcw[i];
#pragma unroll 1
    for (int i = threadIdx.x; i < bone_words; i += blockDim.x) dstw[bones0 + i] = srcw[bones0 + i];
}

// Widen [amin, amax] x [bmin, bmax] by the ray-direction range (a = x/z,
// b = y/z) of the solid ellipse(s) {C + A w : |w| <= 1} with A A^T = Sg
// (xx, yy, zz, xy, xz, yz).  A plane through the camera with normal n touches
// it where (n.C)^2 = n^T Sg n; with n = (1, 0, -a) that is the quadratic
// a^2 (Cz^2 - Szz) - 2 a (Cx Cz - Sxz) + (Cx^2 - Sxx) = 0, whose roots are the
// exact bounds.  Its discriminant is expanded so that the ~Cz^2 Cx^2 terms
// cancel symbolically.  Returns false unless the solid lies beyond the plane
// z = 1 mm.  The box made from these bounds keeps a pixel of margin on every
// side, so approximate square roots and reciprocals (relative error ~1e-7)
// cannot make it miss a covered pixel.
__device__ __forceinline__ bool ellipse_ray_bounds(const float C[3], const float Sg[6], float& amin, float& amax,
                                                   float& bmin, float& bmax)
{
    const float ez = sqrt_approx(fmaxf(Sg[2], 0.f));  // z half-extent
    if (!(C[2] - ez >= 1.0f)) return false;
    const float al = fmaf(C[2], C[2], -Sg[2]);
    const float ial = rcp_approx(al);
    {
        const float be = fmaf(C[0], C[2], -Sg[4]);
        const float disc = fmaf(Sg[0], C[2] * C[2], fmaf(-2.f * Sg[4], C[0] * C[2], fmaf(Sg[2], C[0] * C[0],
                                fmaf(Sg[4], Sg[4], -Sg[0] * Sg[2]))));
        const float sq = sqrt_approx(fmaxf(disc, 0.f));
        amin = fminf(amin, (be - sq) * ial);
        amax = fmaxf(amax, (be + sq) * ial);
    }
    {
        const float be = fmaf(C[1], C[2], -Sg[5]);
        const float disc = fmaf(Sg[1], C[2] * C[2], fmaf(-2.f * Sg[5], C[1] * C[2], fmaf(Sg[2], C[1] * C[1],
                                fmaf(Sg[5], Sg[5], -Sg[1] * Sg[2]))));
        const float sq = sqrt_approx(fmaxf(disc, 0.f));
        bmin = fminf(bmin, (be - sq) * ial);
        bmax = fmaxf(bmax, (be + sq) * ial);
    }
    return true;
}

// FK of the raw pose `pose` [26] (global or shared memory): writes the particle's
// n_prims records to prims [n_prims][4] and kc.  cam = (fx, fy, cx, cy).  Every
// thread of the CTA must call it (it synchronises the CTA).
// emit(j, rec) is called by the thread that formed primitive j's record
// (float[16], as stored), e.g. to derive more from it while it is in registers.
struct NoEmit {
    __device__ void operator()(int, const float*) const {}
};

// The collision data of the kc variants in shared memory: a CTA copies it
// once from the launch parameter (whose reads with a different address in
// every lane the constant cache serves one address at a time) and every FK
// of the CTA then reads the copy.
struct CollideShared {
    DevProxy proxies[kMaxProxies];
    uint16_t pairs[kMaxPairs];  // proxy i in the low byte, j in the high byte
};
// what a kernel of model type M keeps for it: kernels launched only for the
// paper's kc take the smaller DevModelCore and keep nothing
template <class M>
using CollideSmem = typename std::conditional<std::is_same<M, DevModel>::value, CollideShared, char>::type;

// copy the model's collision data into dst when its kc variant needs it (all
// threads of the CTA; the first barrier of fk_particle publishes the copy);
// returns the copy, or nullptr for the paper's kc
__device__ __forceinline__ const CollideShared* collide_load(CollideShared& dst, const DevModel& m)
{
    if (m.kc_variant == HS_KC_ABDUCTION) return nullptr;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(m.proxies);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst.proxies);
    const int pw = m.n_proxies * (int)(sizeof(DevProxy) / 4);
    for (int i = threadIdx.x; i < pw; i += blockDim.x) d[i] = src[i];
    const uint32_t* srp = reinterpret_cast<const uint32_t*>(m.pairs);
    uint32_t* dp = reinterpret_cast<uint32_t*>(dst.pairs);
    const int qw = (m.n_pairs + 1) / 2;
    for (int i = threadIdx.x; i < qw; i += blockDim.x) dp[i] = srp[i];
    return &dst;
}
__device__ __forceinline__ const CollideShared* collide_load(char&, const DevModelCore&) { return nullptr; }

// col: the collision data (collide_load), nullptr for the paper's kc.
template <class Emit = NoEmit>
__device__ __forceinline__ void fk_particle(FkShared& sh, const CollideShared* col, const float* pose, float4 cam,
                                            float4* prims, float* kc, uint32_t* status, const Emit& emit = Emit())
{
    const DevModelCore& model = sh.model;
    float* q = sh.q;
    float(*lR)[9] = sh.lR;
    float(*bR)[9] = sh.bR;
    float(*bP)[3] = sh.bP;
    int& bad = sh.bad;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    __syncthreads();
    if (t < kNdof) {
        float v = pose[t];
        if (!isfinite(v)) atomicOr(&bad, 1);
        const float qc = fminf(fmaxf(v, model.lo[t]), model.hi[t]);
        q[t] = qc;
        if (t >= 3) sincosf(qc, &sh.sn[t], &sh.cs[t]);  // every angle at once
    }
    __syncthreads();

    // frame of each bone: one thread per bone composes its path from the palm,
    // G_k = G_{k-1} L(a_k) and P_k = G_{k-1} off(a_k) + P_{k-1} (a_k its
    // ancestor at depth k), forming each local rotation L from the angles'
    // sines and cosines as it goes: no barrier per level, none between local
    // and global frames (positions relative to the wrist; its translation is
    // added once per primitive).  Each thread also keeps its own L in lR.
    if (t < model.n_bones) {
        float G[9], P[3] = {0.f, 0.f, 0.f};
        palm_local(sh.sn, sh.cs, G);
        const DevBone& Bt = model.bones[t];
        const int d = Bt.depth;
        if (t == 0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) lR[0][k] = G[k];
        }
        // levels 1..3 (a hand's fingers are three bones deep): their local
        // rotations first (anc[k] is the palm beyond the bone's depth, so the
        // reads stay in bounds and need no branch), then the products
        constexpr int kFast = 3;
        float L[kFast][9];
#pragma unroll
        for (int k = 0; k < kFast; ++k) bone_local(model.bones[Bt.anc[k + 1]], sh.sn, sh.cs, L[k]);
#pragma unroll
        for (int k = 1; k <= kFast; ++k) {
            if (k <= d) {
                const DevBone& B = model.bones[Bt.anc[k]];
                float Gn[9], Pn[3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    Pn[i] = fmaf(G[3 * i], B.off[0], fmaf(G[3 * i + 1], B.off[1], fmaf(G[3 * i + 2], B.off[2], P[i])));
                mat3_mul(G, L[k - 1], Gn);
#pragma unroll
                for (int i = 0; i < 3; ++i) P[i] = Pn[i];
#pragma unroll
                for (int k2 = 0; k2 < 9; ++k2) G[k2] = Gn[k2];
            }
            if (k == d) {
#pragma unroll
                for (int q2 = 0; q2 < 9; ++q2) lR[t][q2] = L[k - 1][q2];
            }
        }
        for (int k = kFast + 1; k <= d; ++k) {  // deeper chains, level by level
            const DevBone& B = model.bones[Bt.anc[k]];
            float Lk[9], Gn[9], Pn[3];
            bone_local(B, sh.sn, sh.cs, Lk);
            if (k == d) {
#pragma unroll
                for (int q2 = 0; q2 < 9; ++q2) lR[t][q2] = Lk[q2];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
                Pn[i] = fmaf(G[3 * i], B.off[0], fmaf(G[3 * i + 1], B.off[1], fmaf(G[3 * i + 2], B.off[2], P[i])));
            mat3_mul(G, Lk, Gn);
#pragma unroll
            for (int i = 0; i < 3; ++i) P[i] = Pn[i];
#pragma unroll
            for (int k2 = 0; k2 < 9; ++k2) G[k2] = Gn[k2];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) bR[t][k] = G[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) bP[t][i] = P[i];
    }
    __syncthreads();

    // intersection-ready primitive records
    if (t < model.n_prims) {
        const DevPrimDesc& D = model.prims[t];
        const float* R = bR[D.bone];
        const float* O = bP[D.bone];
        float C[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            C[i] = q[i] + fmaf(R[3 * i], D.center[0], fmaf(R[3 * i + 1], D.center[1], fmaf(R[3 * i + 2], D.center[2], O[i])));
        const bool cone = D.kind == HS_PRIM_ECONE;
        const float is0 = D.inv_s[0], is1 = D.inv_s[1], is2 = D.inv_s[2];
        // column j of M = S^-1 R^T is (R[j][0]/s0, R[j][1]/s1, R[j][2]/s2)
        float rec[16];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rec[3 * j + 0] = R[3 * j + 0] * is0;
            rec[3 * j + 1] = R[3 * j + 1] * is1;
            rec[3 * j + 2] = R[3 * j + 2] * is2;
        }
        // the centre itself (the renderer forms M (t0 d - C) per pixel, which keeps
        // its precision where M C - t0 M d would cancel two ~500 mm terms)
        rec[9] = C[0];
        rec[10] = C[1];
        rec[11] = C[2];
        rec[12] = __uint_as_float(cone ? (uint32_t)D.caps : 0u);  // visible cone caps
        rec[13] = cone ? D.dims[3] : kEllipsoidMarker;
        // the exact ray-direction bounds of the solid (a, b ranges), from its
        // ellipse(s): the ellipsoid itself, or the cone's two end ellipses (the
        // truncated cone is their convex hull, whose box is the union of theirs)
        float amin = FLT_MAX, amax = -FLT_MAX, bmin = FLT_MAX, bmax = -FLT_MAX;
        bool behind = false;
        if (cone) {
            const float ax = D.dims[0], az = D.dims[1], hl = D.dims[2], kap = D.dims[3];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float sgn = c ? 1.f : -1.f;
                const float g = 1.f + sgn * kap;  // section scale at Y = sgn
                const float u2 = ax * ax * g * g, w2 = az * az * g * g;
                float Sg[6];  // u2 r0 r0^T + w2 r2 r2^T (r_k = column k of R)
                Sg[0] = fmaf(u2, R[0] * R[0], w2 * R[2] * R[2]);
                Sg[1] = fmaf(u2, R[3] * R[3], w2 * R[5] * R[5]);
                Sg[2] = fmaf(u2, R[6] * R[6], w2 * R[8] * R[8]);
                Sg[3] = fmaf(u2, R[0] * R[3], w2 * R[2] * R[5]);
                Sg[4] = fmaf(u2, R[0] * R[6], w2 * R[2] * R[8]);
                Sg[5] = fmaf(u2, R[3] * R[6], w2 * R[5] * R[8]);
                const float Cc[3] = {fmaf(sgn * hl, R[1], C[0]), fmaf(sgn * hl, R[4], C[1]),
                                     fmaf(sgn * hl, R[7], C[2])};
                behind |= !ellipse_ray_bounds(Cc, Sg, amin, amax, bmin, bmax);
            }
        } else {
            const float s0 = D.dims[0] * D.dims[0], s1 = D.dims[1] * D.dims[1], s2 = D.dims[2] * D.dims[2];
            float Sg[6];  // R diag(s^2) R^T
            Sg[0] = fmaf(R[0] * R[0], s0, fmaf(R[1] * R[1], s1, R[2] * R[2] * s2));
            Sg[1] = fmaf(R[3] * R[3], s0, fmaf(R[4] * R[4], s1, R[5] * R[5] * s2));
            Sg[2] = fmaf(R[6] * R[6], s0, fmaf(R[7] * R[7], s1, R[8] * R[8] * s2));
            Sg[3] = fmaf(R[0] * R[3], s0, fmaf(R[1] * R[4], s1, R[2] * R[5] * s2));
            Sg[4] = fmaf(R[0] * R[6], s0, fmaf(R[1] * R[7], s1, R[2] * R[8] * s2));
            Sg[5] = fmaf(R[3] * R[6], s0, fmaf(R[4] * R[7], s1, R[5] * R[8] * s2));
            behind = !ellipse_ray_bounds(C, Sg, amin, amax, bmin, bmax);
        }
        int u0, v0, u1, v1;
        if (behind) {
            u0 = v0 = -32767;
            u1 = v1 = 32767;
        } else {
            u0 = clamp_i16(ceilf(fmaf(cam.x, amin, cam.z - 0.5f)) - 1.f);
            u1 = clamp_i16(floorf(fmaf(cam.x, amax, cam.z - 0.5f)) + 1.f);
            v0 = clamp_i16(ceilf(fmaf(cam.y, bmin, cam.w - 0.5f)) - 1.f);
            v1 = clamp_i16(floorf(fmaf(cam.y, bmax, cam.w - 0.5f)) + 1.f);
        }
        rec[14] = pack_i16x2(u0, v0);
        rec[15] = pack_i16x2(u1, v1);
        float4* dst = prims + (size_t)t * 4;
        dst[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
        dst[1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
        dst[2] = make_float4(rec[8], rec[9], rec[10], rec[11]);
        dst[3] = make_float4(rec[12], rec[13], rec[14], rec[15]);
        emit(t, rec);
    }
    if (model.kc_variant != HS_KC_ABDUCTION && col) {  // (uniform over the CTA)
        // interpenetration of different fingers: the collision proxies relative to
        // the wrist (distances do not see its translation), then every pair of
        // proxies on different fingers, summed in fixed point (order-independent)
        const int n = model.n_proxies;
        for (int i = t; i < n; i += blockDim.x) {
            const DevProxy& X = col->proxies[i];
            const float* R = bR[X.bone];
            const float* O = bP[X.bone];
            float c[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                c[k] = fmaf(R[3 * k], X.local[0], fmaf(R[3 * k + 1], X.local[1], fmaf(R[3 * k + 2], X.local[2], O[k])));
            sh.pc[i] = make_float4(c[0], c[1], c[2], X.radius);
        }
        if (t == 0) sh.pen_fix = 0ull;
        __syncthreads();
        unsigned long long acc = 0ull;
        for (int k = t; k < model.n_pairs; k += blockDim.x) {  // the host listed the pairs to visit
            const uint32_t ij = col->pairs[k];
            const float4 a = sh.pc[ij & 0xffu], b = sh.pc[ij >> 8];
            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)), rr = a.w + b.w;
            if (d2 < rr * rr) {  // (the root only for the pairs that touch)
                const float pen = rr - sqrtf(d2);
                if (pen > 0.f) acc += (unsigned long long)__float2ll_rn(pen * kPenFix);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((t & 31) == 0 && acc) atomicAdd(&sh.pen_fix, acc);
        __syncthreads();
    }
    if (t == 32) {
        // kc(h): pairs (index, middle), (middle, ring), (ring, pinky) of MP_z
        float k = fmaxf(q[15] - q[11], 0.f) + fmaxf(q[19] - q[15], 0.f) + fmaxf(q[23] - q[19], 0.f);
        if (model.kc_variant == HS_KC_PEN) k = 0.f;
        if (model.kc_variant != HS_KC_ABDUCTION)
            k = fmaf(model.pen_weight, __ull2float_rn(sh.pen_fix) * (1.f / kPenFix), k);
        *kc = bad ? __int_as_float(0x7fc00000) : k;
        if (bad) set_status(status, HS_DEV_NONFINITE_POSE);
    }
}

}  // namespace hs
