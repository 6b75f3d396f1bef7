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

#include "hs_args.cuh"

namespace hs {

struct FkShared {
    DevModel model;
    float q[kNdof];
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

__device__ __forceinline__ int clamp_i16(float v)
{
    return (int)fminf(fmaxf(v, -32767.0f), 32767.0f);
}

// one coalesced copy of the model (a by-value launch parameter) into shared
// memory; later accesses use thread-dependent bone / primitive indices
__device__ __forceinline__ void fk_load_model(FkShared& sh, const DevModel& mp)
{
    // only the used part: header and limits, then the n_prims primitives and n_bones bones
    const uint32_t* srcw = reinterpret_cast<const uint32_t*>(&mp);
    uint32_t* dstw = reinterpret_cast<uint32_t*>(&sh.model);
    constexpr int head = (int)(offsetof(DevModel, prims) / 4);
    const int prim_end = head + mp.n_prims * (int)(sizeof(DevPrimDesc) / 4);
    constexpr int bones0 = (int)(offsetof(DevModel, bones) / 4);
    const int bone_words = mp.n_bones * (int)(sizeof(DevBone) / 4);
    for (int i = threadIdx.x; i < prim_end; i += blockDim.x) dstw[i] = srcw[i];
    for (int i = threadIdx.x; i < bone_words; i += blockDim.x) dstw[bones0 + i] = srcw[bones0 + i];
}

// FK of the raw pose `pose` [26] (global or shared memory): writes the particle's
// n_prims records to prims [n_prims][4] and kc.  cam = (fx, fy, cx, cy).  Every
// thread of the 64-thread CTA must call it (it synchronises the CTA).
__device__ __forceinline__ void fk_particle(FkShared& sh, const float* pose, float4 cam, float4* prims, float* kc,
                                            uint32_t* status)
{
    const DevModel& model = sh.model;
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
        q[t] = fminf(fmaxf(v, model.lo[t]), model.hi[t]);
    }
    __syncthreads();

    // local rotation of each bone
    if (t < model.n_bones) {
        float R[9];
        if (t == 0) {
            // palm: diag(1,-1,-1) * Rz(q5) Ry(q4) Rx(q3)
            float sx, cx, sy, cy, sz, cz;
            sincosf(q[3], &sx, &cx);
            sincosf(q[4], &sy, &cy);
            sincosf(q[5], &sz, &cz);
            const float Rz[9] = {cz, -sz, 0.f, sz, cz, 0.f, 0.f, 0.f, 1.f};
            const float Ry[9] = {cy, 0.f, sy, 0.f, 1.f, 0.f, -sy, 0.f, cy};
            const float Rx[9] = {1.f, 0.f, 0.f, 0.f, cx, -sx, 0.f, sx, cx};
            float T[9];
            mat3_mul(Rz, Ry, T);
            mat3_mul(T, Rx, R);
#pragma unroll
            for (int k = 3; k < 9; ++k) R[k] = -R[k];
        } else {
            const DevBone& B = model.bones[t];
            float sz = 0.f, cz = 1.f, sx = 0.f, cx = 1.f;
            if (B.dof_z >= 0) sincosf(q[B.dof_z], &sz, &cz);
            if (B.dof_x >= 0) sincosf(q[B.dof_x], &sx, &cx);
            const float ZX[9] = {cz, -sz * cx, sz * sx, sz, cz * cx, -cz * sx, 0.f, sx, cx};  // Rz Rx
            mat3_mul(B.rest, ZX, R);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) lR[t][k] = R[k];
    }
    __syncthreads();
    if (t == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) bR[0][k] = lR[0][k];
        bP[0][0] = 0.f;  // positions relative to the wrist; its translation is added once per primitive
        bP[0][1] = 0.f;
        bP[0][2] = 0.f;
    }
    __syncthreads();
    for (int lvl = 1; lvl <= model.max_depth; ++lvl) {
        if (t < model.n_bones && t > 0 && model.bones[t].depth == lvl) {
            const DevBone& B = model.bones[t];
            const float* Rp = bR[B.parent];
            float R[9];
            mat3_mul(Rp, lR[t], R);
#pragma unroll
            for (int k = 0; k < 9; ++k) bR[t][k] = R[k];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                bP[t][i] = fmaf(Rp[3 * i], B.off[0], fmaf(Rp[3 * i + 1], B.off[1], fmaf(Rp[3 * i + 2], B.off[2], bP[B.parent][i])));
        }
        __syncthreads();
    }

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
        // box half extents e (local x, y, z)
        float e[3];
        if (cone) {
            const float grow = 1.f + fabsf(D.dims[3]);
            e[0] = D.dims[0] * grow; e[1] = D.dims[2]; e[2] = D.dims[1] * grow;
        } else {
            e[0] = D.dims[0]; e[1] = D.dims[1]; e[2] = D.dims[2];
        }
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
        // conservative pixel box from the 8 projected corners of the local box
        float amin = FLT_MAX, amax = -FLT_MAX, bmin = FLT_MAX, bmax = -FLT_MAX;
        bool behind = false;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float sx = (c & 1) ? e[0] : -e[0], sy = (c & 2) ? e[1] : -e[1], sz = (c & 4) ? e[2] : -e[2];
            const float X = fmaf(R[0], sx, fmaf(R[1], sy, fmaf(R[2], sz, C[0])));
            const float Y = fmaf(R[3], sx, fmaf(R[4], sy, fmaf(R[5], sz, C[1])));
            const float Z = fmaf(R[6], sx, fmaf(R[7], sy, fmaf(R[8], sz, C[2])));
            behind |= !(Z >= 1.0f);
            const float iz = rcp_approx(Z);  // the box keeps a 1-pixel margin
            amin = fminf(amin, X * iz);
            amax = fmaxf(amax, X * iz);
            bmin = fminf(bmin, Y * iz);
            bmax = fmaxf(bmax, Y * iz);
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
    }
    if (t == 32) {
        // kc(h): pairs (index, middle), (middle, ring), (ring, pinky) of MP_z
        const float k = fmaxf(q[15] - q[11], 0.f) + fmaxf(q[19] - q[15], 0.f) + fmaxf(q[23] - q[19], 0.f);
        *kc = bad ? __int_as_float(0x7fc00000) : k;
        if (bad) set_status(status, HS_DEV_NONFINITE_POSE);
    }
}

}  // namespace hs
