// api.cu -- the extern "C" boundary of libhandscore.so (include/handscore.h).
//
// Every entry point validates its arguments on the host and returns a
// negative status before touching the GPU; only then does it launch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <mutex>

#include "hs_args.cuh"

namespace hs {

// ---- the device status word ----------------------------------------------------
static __device__ uint32_t g_status;
constexpr int kMaxDevices = 64;
static uint32_t* g_status_ptr[kMaxDevices];
static std::mutex g_mutex;

// device address of g_status on the current device (looked up once per device)
static int status_ptr(uint32_t** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_status_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return HS_ERR_CUDA;
        g_status_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_status_ptr[dev];
    return HS_OK;
}

// ---- TMA descriptor encoding (driver entry point, no link-time libcuda) ----------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static int encode_tile_map(CUtensorMap* map, const void* base, CUtensorMapDataType type, int esz, int W, int H,
                           int pitch)
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return HS_ERR_CUDA;
    (void)esz;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {16, 4};  // one TMA box = one 16 x 4 work unit
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(map, type, 2, const_cast<void*>(base), dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HS_OK : HS_ERR_CUDA;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
static bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

static int validate_obs(const HsObs* o)
{
    if (!o || !o->depth || !o->skin || !o->stats) return HS_ERR_ARG;
    if (o->depth_type != HS_DEPTH_U16 && o->depth_type != HS_DEPTH_F32) return HS_ERR_ARG;
    if (o->W < 1 || o->H < 1 || o->W > HS_MAX_ROI || o->H > HS_MAX_ROI) return HS_ERR_SIZE;
    const int esz = o->depth_type == HS_DEPTH_F32 ? 4 : 2;
    if (!aligned16(o->depth) || !aligned16(o->skin)) return HS_ERR_ALIGN;
    if (o->depth_pitch % 16 != 0 || o->skin_pitch % 16 != 0) return HS_ERR_ALIGN;
    if (o->depth_pitch < o->W * esz || o->skin_pitch < o->W) return HS_ERR_SIZE;
    return HS_OK;
}

static int validate_cam(const HsCamera* c)
{
    if (!c) return HS_ERR_ARG;
    if (!finite_pos(c->fx) || !finite_pos(c->fy) || !std::isfinite(c->cx) || !std::isfinite(c->cy))
        return HS_ERR_ARG;
    return HS_OK;
}

constexpr int kMaxK = 16;             // default cap of CTAs per particle in the render
constexpr int kMaxCtasPerParticle = 64;
constexpr int kTargetCtas = 148 * 6;  // one resident wave of the unit and strip kernels (6 CTAs of 4 warps per SM)

}  // namespace hs

int hs_render_variant(const HsScoreParams* p, int P)
{
    if (!p || p->variant < 0 || p->variant >= HS_RENDER_VARIANTS || P < 0) return HS_ERR_ARG;
    if (p->variant != HS_RENDER_AUTO) return p->variant;
    // many particles per call: the tile kernel (pixel-exact work, throughput);
    // fewer than one wave of CTAs: the unit kernel (shorter critical path)
    return P >= hs::kTargetCtas ? HS_RENDER_TILES_64x32 : HS_RENDER_UNITS;
}

namespace hs {

static int validate_score_params(const HsScoreParams* p)
{
    if (!p) return HS_ERR_ARG;
    if (!std::isfinite(p->d_m) || !std::isfinite(p->d_M) || !std::isfinite(p->lambda) ||
        !std::isfinite(p->lambda_k) || p->d_m < 0.f || p->d_M < 0.f || p->d_M >= 127.f)
        return HS_ERR_ARG;
    if (p->variant < 0 || p->variant >= HS_RENDER_VARIANTS) return HS_ERR_ARG;
    if (p->ctas_per_particle < 0 || p->ctas_per_particle > kMaxCtasPerParticle) return HS_ERR_ARG;
    return HS_OK;
}

// the render kernel and its CTAs per particle for a call over P particles
static cudaError_t launch_render(const HsScoreParams& prm, const CUtensorMap& tm_depth, const CUtensorMap& tm_skin,
                                 RenderArgs& a, cudaStream_t s)
{
    const int variant = hs_render_variant(&prm, a.P);
    // default: about one resident wave in total (any K is correct; it only
    // changes how a particle's work is dealt)
    int K = prm.ctas_per_particle;
    if (K == 0) {
        K = kTargetCtas / a.P;  // rounded down: K * P never exceeds one wave
        if (K > kMaxK) K = kMaxK;
        if (K < 1) K = 1;
    }
    a.K = K;
    a.d_m = prm.d_m;
    a.d_M = prm.d_M;
    a.lambda = prm.lambda;
    a.lambda_k = prm.lambda_k;
    if (variant == HS_RENDER_UNITS) return launch_render_score(tm_depth, tm_skin, a, s);
    if (variant >= HS_RENDER_STRIPS_8x16 && variant <= HS_RENDER_PERSISTENT_8x32)
        return launch_render_strips(variant, tm_depth, tm_skin, a, s);
    return launch_render_tiles(variant, tm_depth, tm_skin, a, s);
}

}  // namespace hs

using namespace hs;

struct HsModel {
    DevModel dev;
    Limits lim;
    int proxies;  // collision proxies the model has (dev holds at most kMaxProxies of them)
    int pairs;    // and pairs of them the penetration test visits (dev holds at most kMaxPairs)
};

struct HsBatch {
    int S, P_total, P_max, max_H;
    BatchDev dev;          // device views / particle-to-swarm table (inside the caller's buffer)
    const int32_t* order;  // device [P_total]: the render's CTA rows, largest ROI first
};

namespace {
__global__ void zero_stats_kernel(const BatchDev b)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < b.S) {
        b.views[s].stats[0] = 0u;
        b.views[s].stats[1] = 0u;
    }
}

size_t table_bytes(long long P_total) { return ((size_t)P_total * 4 + 255) / 256 * 256; }

// [256-byte header][S views][particle -> swarm table][render order]
size_t batch_bytes(int S, long long P_total)
{
    return 256 + (size_t)S * sizeof(SwarmView) + 2 * table_bytes(P_total);
}
}  // namespace

extern "C" {

int hs_version(void) { return 100; }

const char* hs_status_string(int s)
{
    switch (s) {
    case HS_OK: return "ok";
    case HS_ERR_ARG: return "invalid argument";
    case HS_ERR_ALIGN: return "misaligned pointer or pitch";
    case HS_ERR_SIZE: return "size out of range";
    case HS_ERR_TIMEOUT: return "device wait timed out";
    case HS_ERR_NOT_IMPL: return "not implemented";
    case HS_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

int hs_model_create(const HsModelDesc* d, HsModel** out)
{
    if (!d || !out || !d->bones || !d->prims) return HS_ERR_ARG;
    if (d->n_bones < 1 || d->n_bones > HS_MAX_BONES || d->n_prims < 1 || d->n_prims > HS_MAX_PRIMS)
        return HS_ERR_SIZE;
    HsModel* m = static_cast<HsModel*>(std::calloc(1, sizeof(HsModel)));
    if (!m) return HS_ERR_ARG;
    DevModel& dm = m->dev;
    dm.n_bones = d->n_bones;
    dm.n_prims = d->n_prims;
    int bad = 0;
    for (int k = 0; k < HS_NDOF; ++k) {
        if (!std::isfinite(d->lo[k]) || !std::isfinite(d->hi[k]) || d->lo[k] > d->hi[k]) bad = 1;
        dm.lo[k] = m->lim.lo[k] = d->lo[k];
        dm.hi[k] = m->lim.hi[k] = d->hi[k];
    }
    int max_depth = 0;
    for (int b = 0; b < d->n_bones; ++b) {
        const HsBoneDesc& B = d->bones[b];
        DevBone& o = dm.bones[b];
        o.parent = b == 0 ? -1 : B.parent;
        o.dof_z = B.dof_z;
        o.dof_x = B.dof_x;
        if (b > 0 && (B.parent < 0 || B.parent >= b)) bad = 1;
        if (B.dof_z < -1 || B.dof_z >= HS_NDOF || B.dof_x < -1 || B.dof_x >= HS_NDOF) bad = 1;
        o.depth = b == 0 ? 0 : dm.bones[B.parent < 0 || B.parent >= b ? 0 : B.parent].depth + 1;
        if (o.depth > max_depth) max_depth = o.depth;
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(B.offset[i]) || !std::isfinite(B.rest[i])) bad = 1;
            o.off[i] = B.offset[i];
        }
        // rest rotation Rz(rz) Ry(ry) Rx(rx), row-major, built in double
        const double cx = std::cos(B.rest[0]), sx = std::sin(B.rest[0]);
        const double cy = std::cos(B.rest[1]), sy = std::sin(B.rest[1]);
        const double cz = std::cos(B.rest[2]), sz = std::sin(B.rest[2]);
        const double R[9] = {cz * cy, cz * sy * sx - sz * cx, cz * sy * cx + sz * sx,
                             sz * cy, sz * sy * sx + cz * cx, sz * sy * cx - cz * sx,
                             -sy,     cy * sx,                cy * cx};
        for (int i = 0; i < 9; ++i) o.rest[i] = (float)R[i];
    }
    if (!bad && max_depth > HS_MAX_DEPTH) return HS_ERR_SIZE;
    for (int b = 0; !bad && b < d->n_bones; ++b) {  // the path from the palm, for FK's one-pass chains
        DevBone& o = dm.bones[b];
        for (int k = 0; k < kMaxChain; ++k) o.anc[k] = 0;
        for (int k = o.depth, a = b; k >= 0; --k, a = dm.bones[a].parent) o.anc[k] = (int8_t)a;
    }
    dm.max_depth = max_depth;
    for (int k = 0; k < d->n_prims; ++k) {
        const HsPrimDesc& P = d->prims[k];
        DevPrimDesc& o = dm.prims[k];
        o.bone = P.bone;
        o.kind = P.kind;
        if (P.bone < 0 || P.bone >= d->n_bones) bad = 1;
        if (P.kind != HS_PRIM_ELLIPSOID && P.kind != HS_PRIM_ECONE) bad = 1;
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(P.center[i])) bad = 1;
            o.center[i] = P.center[i];
        }
        for (int i = 0; i < 4; ++i) o.dims[i] = P.dims[i];
        if (!finite_pos(P.dims[0]) || !finite_pos(P.dims[1]) || !finite_pos(P.dims[2])) bad = 1;
        if (P.kind == HS_PRIM_ECONE && !(std::fabs(P.dims[3]) < 1.f)) bad = 1;
        // local scale (x, y, z): ellipsoid semi-axes; cone (ax, hl, az)
        const float sc[3] = {P.dims[0], P.kind == HS_PRIM_ECONE ? P.dims[2] : P.dims[1],
                             P.kind == HS_PRIM_ECONE ? P.dims[1] : P.dims[2]};
        for (int i = 0; i < 3; ++i) o.inv_s[i] = 1.f / sc[i];
        o.caps = 3;
    }
    if (bad) {
        std::free(m);
        return HS_ERR_ARG;
    }
    // A cone's planar cap is never the nearest surface when an ellipsoid that is
    // rigidly attached at the cap centre contains the cap disc: every ray through
    // the disc enters that ellipsoid first (or at the disc rim, at equal depth).
    // Such caps are skipped by the renderer; the rendered depth is unchanged.
    for (int k = 0; k < d->n_prims; ++k) {
        DevPrimDesc& c = dm.prims[k];
        if (c.kind != HS_PRIM_ECONE) continue;
        for (int side = 0; side < 2; ++side) {
            const float sgn = side ? 1.f : -1.f;
            const float w = 1.f + sgn * c.dims[3];
            const float rx = c.dims[0] * w, rz = c.dims[1] * w;
            const float cc[3] = {c.center[0], c.center[1] + sgn * c.dims[2], c.center[2]};
            bool covered = false;
            for (int e = 0; e < d->n_prims && !covered; ++e) {
                const DevPrimDesc& q = dm.prims[e];
                if (q.kind != HS_PRIM_ELLIPSOID) continue;
                const float tol = 1e-5f;  // relative slack on the radii only
                const bool big = q.dims[0] >= rx * (1.f - tol) && q.dims[2] >= rz * (1.f - tol);
                if (q.bone == c.bone && q.center[0] == cc[0] && q.center[1] == cc[1] && q.center[2] == cc[2] && big)
                    covered = true;
                // a sphere at the origin of a child bone whose origin is the cap centre
                const bool sphere = q.dims[0] == q.dims[1] && q.dims[1] == q.dims[2];
                if (sphere && q.bone > 0 && dm.bones[q.bone].parent == c.bone && q.center[0] == 0.f &&
                    q.center[1] == 0.f && q.center[2] == 0.f) {
                    const float* off = dm.bones[q.bone].off;
                    if (off[0] == cc[0] && off[1] == cc[1] && off[2] == cc[2] && q.dims[0] >= std::fmax(rx, rz) * (1.f - tol))
                        covered = true;
                }
            }
            if (covered) c.caps &= ~(1 << side);
        }
    }
    // collision proxies of the interpenetration test (inscribed spheres), and
    // the finger of each bone: the palm's child on its path to the palm
    int finger[HS_MAX_BONES];
    int n_fingers = 0;
    finger[0] = -1;
    for (int b = 1; b < d->n_bones; ++b) finger[b] = d->bones[b].parent == 0 ? n_fingers++ : finger[d->bones[b].parent];
    int np = 0;
    auto add_proxy = [&](int bone, float x, float y, float z, float r) {
        const int fixed = bone > 0 && d->bones[bone].parent == 0 && x == 0.f && y == 0.f && z == 0.f;
        if (np < kMaxProxies) dm.proxies[np] = DevProxy{{x, y, z}, r, bone, finger[bone], fixed};
        ++np;
    };
    for (int k = 0; k < d->n_prims; ++k) {
        const HsPrimDesc& P = d->prims[k];
        if (P.kind == HS_PRIM_ELLIPSOID) {
            add_proxy(P.bone, P.center[0], P.center[1], P.center[2],
                      std::min(P.dims[0], std::min(P.dims[1], P.dims[2])));
        } else {  // on the axis (local y) at -hl/2, 0, +hl/2: the largest sphere
                  // inside the circular cone of section rho (1 + kappa y / hl) there
            const double hl = P.dims[2], rho = std::min(P.dims[0], P.dims[1]), kap = P.dims[3];
            for (int i = -1; i <= 1; ++i) {
                const double y = 0.5 * i * hl;
                const double side = rho * (1.0 + kap * y / hl) / std::sqrt(1.0 + (rho * kap / hl) * (rho * kap / hl));
                add_proxy(P.bone, P.center[0], P.center[1] + (float)y, P.center[2],
                          (float)std::min(side, hl - std::fabs(y)));
            }
        }
    }
    m->proxies = np;
    // the pairs the test visits: different fingers, not both fixed to the palm
    int npairs = 0;
    for (int i = 0; i < std::min(np, kMaxProxies); ++i)
        for (int j = i + 1; j < std::min(np, kMaxProxies); ++j) {
            const DevProxy &a = dm.proxies[i], &b = dm.proxies[j];
            if (a.finger < 0 || b.finger < 0 || a.finger == b.finger || (a.fixed && b.fixed)) continue;
            if (npairs < kMaxPairs) dm.pairs[npairs] = (uint16_t)(i | (j << 8));
            ++npairs;
        }
    m->pairs = npairs;
    dm.n_proxies = 0;  // the paper's kc needs none
    dm.n_pairs = 0;
    dm.kc_variant = HS_KC_ABDUCTION;
    dm.pen_weight = 0.f;
    *out = m;
    return HS_OK;
}

int hs_model_set_kc(HsModel* model, const HsKcParams* kc)
{
    if (!model || !kc) return HS_ERR_ARG;
    if (kc->variant != HS_KC_ABDUCTION && kc->variant != HS_KC_ABD_PEN && kc->variant != HS_KC_PEN) return HS_ERR_ARG;
    if (!std::isfinite(kc->pen_weight) || kc->pen_weight < 0.f) return HS_ERR_ARG;
    const bool pen = kc->variant != HS_KC_ABDUCTION;
    if (pen && (model->proxies > kMaxProxies || model->pairs > kMaxPairs)) return HS_ERR_SIZE;
    model->dev.kc_variant = kc->variant;
    model->dev.pen_weight = kc->pen_weight;
    model->dev.n_proxies = pen ? model->proxies : 0;
    model->dev.n_pairs = pen ? model->pairs : 0;
    return HS_OK;
}

int hs_model_destroy(HsModel* m)
{
    if (!m) return HS_ERR_ARG;
    std::free(m);
    return HS_OK;
}

int hs_workspace_size(int P, size_t* bytes)
{
    if (!bytes) return HS_ERR_ARG;
    if (P < 0 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    // per particle a 32-byte slot, then the persistent launch's control block
    *bytes = ((size_t)P * sizeof(HsParticleWork) + sizeof(RenderCtl) + 255) / 256 * 256;
    return HS_OK;
}

int hs_workspace_reset(void* ws, size_t bytes, hs_stream_t stream)
{
    if (!ws && bytes) return HS_ERR_ARG;
    if (!bytes) return HS_OK;
    return cudaMemsetAsync(ws, 0, bytes, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int hs_obs_prepare(const HsObs* obs, hs_stream_t stream)
{
    int rc = validate_obs(obs);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(obs->stats, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return HS_ERR_CUDA;
    if (launch_obs_stats(static_cast<const unsigned char*>(obs->depth), obs->depth_pitch,
                         obs->depth_type == HS_DEPTH_F32, obs->skin, obs->skin_pitch, obs->W, obs->H, obs->stats,
                         s) != cudaSuccess)
        return HS_ERR_CUDA;
    return HS_OK;
}

int pose_fk(const HsModel* model, const float* poses, int P, const HsCamera* cam, HsPrim* prims, float* kc,
            hs_stream_t stream)
{
    if (!model || !poses || !prims || !kc) return HS_ERR_ARG;
    int rc = validate_cam(cam);
    if (rc) return rc;
    if (P < 0 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    if (P == 0) return HS_OK;
    FkArgs a = {};
    a.poses = poses;
    a.P = P;
    a.fx = cam->fx;
    a.fy = cam->fy;
    a.cx = cam->cx;
    a.cy = cam->cy;
    a.prims = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    if ((rc = status_ptr(&a.status))) return rc;
    return launch_fk(model->dev, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int render_score_batch(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims,
                       const float* kc, int P, const HsScoreParams* params, void* workspace, size_t workspace_bytes,
                       float* E, HsParts* parts, float* dbg_depth, uint8_t* dbg_mask, hs_stream_t stream)
{
    if (!model || !prims || !kc || !params || !E) return HS_ERR_ARG;
    if ((dbg_depth == nullptr) != (dbg_mask == nullptr)) return HS_ERR_ARG;
    int rc = validate_obs(obs);
    if (rc) return rc;
    if ((rc = validate_cam(cam))) return rc;
    if ((rc = validate_score_params(params))) return rc;
    if (P < 0 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    if (!aligned16(prims) || (workspace && !aligned16(workspace))) return HS_ERR_ALIGN;
    size_t need = 0;
    hs_workspace_size(P, &need);
    if (P > 0 && (!workspace || workspace_bytes < need)) return HS_ERR_SIZE;
    if (P == 0) return HS_OK;

    cudaStream_t s = (cudaStream_t)stream;
    const bool f32 = obs->depth_type == HS_DEPTH_F32;
    CUtensorMap tm_depth, tm_skin;
    if ((rc = encode_tile_map(&tm_depth, obs->depth, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                              f32 ? 4 : 2, obs->W, obs->H, obs->depth_pitch)))
        return rc;
    if ((rc = encode_tile_map(&tm_skin, obs->skin, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, obs->W, obs->H, obs->skin_pitch)))
        return rc;
    if (dbg_depth) {
        const size_t n = (size_t)P * obs->W * obs->H;
        if (cudaMemsetAsync(dbg_depth, 0, n * sizeof(float), s) != cudaSuccess ||
            cudaMemsetAsync(dbg_mask, 0, n, s) != cudaSuccess)
            return HS_ERR_CUDA;
    }
    RenderArgs a = {};
    a.prims = reinterpret_cast<const float4*>(prims);
    a.kc = kc;
    a.P = P;
    a.n_prims = model->dev.n_prims;
    a.W = obs->W;
    a.H = obs->H;
    // ray of pixel (u, v): ((u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, 1), as one FMA per axis
    a.inv_fx = (float)(1.0 / (double)cam->fx);
    a.inv_fy = (float)(1.0 / (double)cam->fy);
    a.off_x = (float)((0.5 - (double)cam->cx) / (double)cam->fx);
    a.off_y = (float)((0.5 - (double)cam->cy) / (double)cam->fy);
    a.depth_f32 = f32;
    a.stats = obs->stats;
    a.work = static_cast<HsParticleWork*>(workspace);
    a.ctl = reinterpret_cast<RenderCtl*>(a.work + P);
    a.E = E;
    a.parts = parts;
    a.dbg_depth = dbg_depth;
    a.dbg_mask = dbg_mask;
    if ((rc = status_ptr(&a.status))) return rc;
    return launch_render(*params, tm_depth, tm_skin, a, s) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pso_init(const HsModel* model, const HsSwarm* sw, int P, const float* seed_pose, const float* scale,
             uint64_t seed, uint32_t frame, hs_stream_t stream)
{
    if (!model || !sw || !seed_pose || !scale) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E) return HS_ERR_ARG;
    if (P < 1 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    PsoInitArgs a = {};
    a.x = sw->x;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.seed_pose = seed_pose;
    for (int d = 0; d < HS_NDOF; ++d) {
        if (!std::isfinite(scale[d]) || scale[d] < 0.f) return HS_ERR_ARG;
        a.scale[d] = scale[d];
    }
    a.P = P;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.frame = frame;
    return launch_pso_init(model->lim, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pso_step(const HsModel* model, const HsSwarm* sw, int P, const HsPsoParams* prm, uint64_t seed, uint32_t frame,
             uint32_t gen, hs_stream_t stream)
{
    if (!model || !sw || !prm) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E || !sw->E) return HS_ERR_ARG;
    if (P < 1 || P > 4096) return HS_ERR_SIZE;
    const double psi = (double)prm->c1 + (double)prm->c2;
    if (!std::isfinite(psi) || prm->c1 < 0.f || prm->c2 < 0.f || psi <= 4.0) return HS_ERR_ARG;
    if (prm->e_stop != 0.f) return HS_ERR_ARG;  // the stopping rule is the batch step's
    if (prm->mutate_every > 0 && (prm->n_mutate < 0 || prm->n_mutate > P)) return HS_ERR_ARG;
    PsoStepArgs a = {};
    a.x = sw->x;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.E = sw->E;
    a.P = P;
    a.c1 = prm->c1;
    a.c2 = prm->c2;
    // constriction factor of Section III.B
    a.w = (float)(2.0 / std::fabs(2.0 - psi - std::sqrt(psi * psi - 4.0 * psi)));
    a.mutate = prm->mutate_every > 0 && gen % (uint32_t)prm->mutate_every == 0 && prm->n_mutate > 0;
    a.n_mutate = prm->n_mutate;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.frame = frame;
    a.gen = gen;
    return launch_pso_step(model->lim, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pso_step_fk(const HsModel* model, const HsSwarm* sw, float* x_next, int P, const HsPsoParams* prm,
                uint64_t seed, uint32_t frame, uint32_t gen, const HsCamera* cam, HsPrim* prims, float* kc,
                hs_stream_t stream)
{
    if (!model || !sw || !prm || !x_next || !prims || !kc) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E || !sw->E) return HS_ERR_ARG;
    if (x_next == sw->x) return HS_ERR_ARG;  // positions are double-buffered
    int rc = validate_cam(cam);
    if (rc) return rc;
    if (P < 1 || P > HS_FUSED_MAX_PARTICLES) return HS_ERR_SIZE;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    const double psi = (double)prm->c1 + (double)prm->c2;
    if (!std::isfinite(psi) || prm->c1 < 0.f || prm->c2 < 0.f || psi <= 4.0) return HS_ERR_ARG;
    if (prm->e_stop != 0.f) return HS_ERR_ARG;  // the stopping rule is the batch step's
    if (prm->mutate_every > 0 && (prm->n_mutate < 0 || prm->n_mutate > P)) return HS_ERR_ARG;
    PsoFkArgs a = {};
    a.x = sw->x;
    a.x_next = x_next;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.E = sw->E;
    a.P = P;
    a.c1 = prm->c1;
    a.c2 = prm->c2;
    a.w = (float)(2.0 / std::fabs(2.0 - psi - std::sqrt(psi * psi - 4.0 * psi)));
    a.mutate = prm->mutate_every > 0 && gen % (uint32_t)prm->mutate_every == 0 && prm->n_mutate > 0;
    a.n_mutate = prm->n_mutate;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.frame = frame;
    a.gen = gen;
    a.cam = make_float4(cam->fx, cam->fy, cam->cx, cam->cy);
    a.prims = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    if ((rc = status_ptr(&a.status))) return rc;
    return launch_pso_step_fk(model->dev, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// ---- a whole tracking frame in one cooperative launch -------------------------------

int hs_frame_workspace_size(int P, size_t* bytes)
{
    if (!bytes) return HS_ERR_ARG;
    if (P < 1 || P > HS_FRAME_MAX_PARTICLES) return HS_ERR_SIZE;
    *bytes = sizeof(FrameCtl) + 3 * (size_t)P * sizeof(FrameSums);
    return HS_OK;
}

int hs_frame_capacity(int* ctas)
{
    if (!ctas) return HS_ERR_ARG;
    return track_frame_capacity(ctas) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int track_frame(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsSwarm* sw, float* x_next, int P,
                int gens, const HsScoreParams* score, const HsPsoParams* prm, const float* seed_pose,
                const float* scale, uint64_t seed, uint32_t frame, int ctas, void* workspace,
                size_t workspace_bytes, HsPrim* prims, float* kc, hs_stream_t stream)
{
    if (!model || !sw || !x_next || !score || !prm || !seed_pose || !scale || !kc) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E || !sw->E) return HS_ERR_ARG;
    if (x_next == sw->x || gens < 0) return HS_ERR_ARG;
    int rc = validate_obs(obs);
    if (rc) return rc;
    if ((rc = validate_cam(cam))) return rc;
    if ((rc = validate_score_params(score))) return rc;
    if (P < 1 || P > HS_FRAME_MAX_PARTICLES) return HS_ERR_SIZE;
    if (ctas < 0) return HS_ERR_ARG;
    const double psi = (double)prm->c1 + (double)prm->c2;
    if (!std::isfinite(psi) || prm->c1 < 0.f || prm->c2 < 0.f || psi <= 4.0) return HS_ERR_ARG;
    if (prm->e_stop != 0.f) return HS_ERR_ARG;  // the stopping rule is the batch step's
    if (prm->mutate_every > 0 && (prm->n_mutate < 0 || prm->n_mutate > P)) return HS_ERR_ARG;
    if (!workspace || (prims && !aligned16(prims)) || !aligned16(workspace)) return workspace ? HS_ERR_ALIGN : HS_ERR_ARG;
    size_t need = 0;
    hs_frame_workspace_size(P, &need);
    if (workspace_bytes < need) return HS_ERR_SIZE;
    FrameArgs a = {};
    for (int d = 0; d < HS_NDOF; ++d) {
        if (!std::isfinite(scale[d]) || scale[d] < 0.f) return HS_ERR_ARG;
        a.scale[d] = scale[d];
    }
    int cap = 0;
    if (track_frame_capacity(&cap) != cudaSuccess) return HS_ERR_CUDA;
    const int nb = ctas ? ctas : std::min(cap, 8 * P);
    if (nb < P || nb > cap) return HS_ERR_SIZE;

    cudaStream_t s = (cudaStream_t)stream;
    const bool f32 = obs->depth_type == HS_DEPTH_F32;
    CUtensorMap tm_depth, tm_skin;
    if ((rc = encode_tile_map(&tm_depth, obs->depth, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                              f32 ? 4 : 2, obs->W, obs->H, obs->depth_pitch)))
        return rc;
    if ((rc = encode_tile_map(&tm_skin, obs->skin, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, obs->W, obs->H, obs->skin_pitch)))
        return rc;
    a.W = obs->W;
    a.H = obs->H;
    a.depth_f32 = f32;
    // rays and projection exactly as render_score_batch and pso_step_fk form them
    a.inv_fx = (float)(1.0 / (double)cam->fx);
    a.inv_fy = (float)(1.0 / (double)cam->fy);
    a.off_x = (float)((0.5 - (double)cam->cx) / (double)cam->fx);
    a.off_y = (float)((0.5 - (double)cam->cy) / (double)cam->fy);
    a.cam = make_float4(cam->fx, cam->fy, cam->cx, cam->cy);
    a.depth = static_cast<const unsigned char*>(obs->depth);
    a.skin = obs->skin;
    a.depth_pitch = obs->depth_pitch;
    a.skin_pitch = obs->skin_pitch;
    a.stats = obs->stats;
    a.d_m = score->d_m;
    a.d_M = score->d_M;
    a.lambda = score->lambda;
    a.lambda_k = score->lambda_k;
    a.xbuf[0] = sw->x;
    a.xbuf[1] = x_next;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.E = const_cast<float*>(sw->E);
    a.prims_out = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    a.seed_pose = seed_pose;
    a.c1 = prm->c1;
    a.c2 = prm->c2;
    a.w = (float)(2.0 / std::fabs(2.0 - psi - std::sqrt(psi * psi - 4.0 * psi)));
    a.mutate_every = prm->mutate_every;
    a.n_mutate = prm->n_mutate;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.frame = frame;
    a.P = P;
    a.gens = gens;
    a.ctl = static_cast<FrameCtl*>(workspace);
    a.sums = reinterpret_cast<FrameSums*>(static_cast<unsigned char*>(workspace) + sizeof(FrameCtl));
    if ((rc = status_ptr(&a.status))) return rc;
    // the frame's observation totals start from zero (as hs_obs_prepare)
    if (cudaMemsetAsync(obs->stats, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return HS_ERR_CUDA;
    return launch_track_frame(model->dev, tm_depth, tm_skin, a, nb, s) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// ---- the smoothed objective and its gradient ---------------------------------------

static int soft_common(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims, int P,
                       const HsScoreParams* params, const HsSoftParams* sp, SoftArgs& a)
{
    if (!model || !prims || !params || !sp) return HS_ERR_ARG;
    int rc = validate_obs(obs);
    if (rc) return rc;
    if ((rc = validate_cam(cam))) return rc;
    if ((rc = validate_score_params(params))) return rc;
    if (!(sp->tau_px > 0.f && sp->tau_px <= 8.f) || !(sp->tau_mm > 0.f && sp->tau_mm <= 10.f)) return HS_ERR_ARG;
    if (sp->ctas_per_particle < 0 || sp->ctas_per_particle > kMaxCtasPerParticle) return HS_ERR_ARG;
    if (P < 0 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    a = SoftArgs{};
    a.prims = reinterpret_cast<const float4*>(prims);
    a.P = P;
    a.n_prims = model->dev.n_prims;
    // 0: the launcher picks one resident wave of the kernel in total (these calls
    // serve few particles; the forward and backward kernels differ in occupancy)
    a.K = sp->ctas_per_particle;
    a.W = obs->W;
    a.H = obs->H;
    a.inv_fx = (float)(1.0 / (double)cam->fx);
    a.inv_fy = (float)(1.0 / (double)cam->fy);
    a.off_x = (float)((0.5 - (double)cam->cx) / (double)cam->fx);
    a.off_y = (float)((0.5 - (double)cam->cy) / (double)cam->fy);
    a.fx = cam->fx;
    a.fy = cam->fy;
    a.d_m = params->d_m;
    a.d_M = params->d_M;
    a.lambda = params->lambda;
    a.lambda_k = params->lambda_k;
    a.tau = sp->tau_px;
    a.tau_mm = sp->tau_mm;
    a.depth = static_cast<const unsigned char*>(obs->depth);
    a.skin = obs->skin;
    a.depth_pitch = obs->depth_pitch;
    a.skin_pitch = obs->skin_pitch;
    a.depth_f32 = obs->depth_type == HS_DEPTH_F32;
    a.stats = obs->stats;
    return HS_OK;
}

int soft_score(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims, const float* kc,
               int P, const HsScoreParams* params, const HsSoftParams* soft, void* workspace,
               size_t workspace_bytes, float* E_s, float* sums, hs_stream_t stream)
{
    SoftArgs a;
    int rc = soft_common(model, obs, cam, prims, P, params, soft, a);
    if (rc) return rc;
    if (!kc || !E_s) return HS_ERR_ARG;
    if (workspace && !aligned16(workspace)) return HS_ERR_ALIGN;
    size_t need = 0;
    hs_workspace_size(P, &need);
    if (P > 0 && (!workspace || workspace_bytes < need)) return HS_ERR_SIZE;
    if (P == 0) return HS_OK;
    a.kc = kc;
    a.work = static_cast<SoftWork*>(workspace);
    a.E = E_s;
    a.sums = sums;
    return launch_soft(false, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int soft_score_backward(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims, int P,
                        const HsScoreParams* params, const HsSoftParams* soft, const float* sums, int64_t* adj,
                        hs_stream_t stream)
{
    SoftArgs a;
    int rc = soft_common(model, obs, cam, prims, P, params, soft, a);
    if (rc) return rc;
    if (!sums || !adj) return HS_ERR_ARG;
    if (P == 0) return HS_OK;
    a.sums = const_cast<float*>(sums);
    a.adj = reinterpret_cast<long long*>(adj);
    return launch_soft(true, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pose_grad(const HsModel* model, const float* poses, int P, const HsCamera* cam, const HsScoreParams* params,
              HsPrim* prims, float* kc, int64_t* adj, float* grad, hs_stream_t stream)
{
    if (!model || !poses || !params || !prims || !kc || !adj || !grad) return HS_ERR_ARG;
    int rc = validate_cam(cam);
    if (rc) return rc;
    if ((rc = validate_score_params(params))) return rc;
    if (P < 0 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    if (P == 0) return HS_OK;
    GradArgs a = {};
    a.poses = poses;
    a.P = P;
    a.fx = cam->fx;
    a.fy = cam->fy;
    a.cx = cam->cx;
    a.cy = cam->cy;
    a.lambda_k = params->lambda_k;
    a.prims = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    a.adj = reinterpret_cast<long long*>(adj);
    a.grad = grad;
    if ((rc = status_ptr(&a.status))) return rc;
    return launch_pose_grad(model->dev, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// ---- gradient polish ----------------------------------------------------------------

int polish_select(const float* E, int P, int k, int32_t* sel, hs_stream_t stream)
{
    if (!E || !sel) return HS_ERR_ARG;
    if (P < 1 || P > HS_MAX_PARTICLES || k < 1 || k > HS_POLISH_MAX || k > P) return HS_ERR_SIZE;
    return launch_select_best(E, P, k, sel, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int polish_gather(const float* x, const float* E, const int32_t* sel, int k, float* x_sel, float* E_sel,
                  hs_stream_t stream)
{
    if (!x || !E || !sel || !x_sel || !E_sel) return HS_ERR_ARG;
    if (k < 1 || k > HS_POLISH_MAX) return HS_ERR_SIZE;
    return launch_gather(x, E, sel, k, x_sel, E_sel, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int polish_step(const HsModel* model, float* x_sel, const float* grad, int k, float eta, const float* scale,
                hs_stream_t stream)
{
    if (!model || !x_sel || !grad || !scale) return HS_ERR_ARG;
    if (k < 1 || k > HS_POLISH_MAX) return HS_ERR_SIZE;
    if (!std::isfinite(eta) || eta < 0.f) return HS_ERR_ARG;
    PolishStep st = {};
    st.eta = eta;
    for (int d = 0; d < HS_NDOF; ++d) {
        if (!std::isfinite(scale[d]) || scale[d] <= 0.f) return HS_ERR_ARG;
        st.scale[d] = scale[d];
        st.lo[d] = model->lim.lo[d];
        st.hi[d] = model->lim.hi[d];
    }
    return launch_polish_step(x_sel, grad, k, st, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int polish_keep_better(float* x, float* E, const int32_t* sel, int k, const float* x_sel, const float* E_old,
                       const float* E_new, hs_stream_t stream)
{
    if (!x || !E || !sel || !x_sel || !E_old || !E_new) return HS_ERR_ARG;
    if (k < 1 || k > HS_POLISH_MAX) return HS_ERR_SIZE;
    return launch_keep_better(x, E, sel, k, x_sel, E_old, E_new, (cudaStream_t)stream) == cudaSuccess ? HS_OK
                                                                                                  : HS_ERR_CUDA;
}

// ---- batches of independent swarms ------------------------------------------------

int hs_batch_buffer_size(const HsSwarmDesc* sw, int S, size_t* bytes)
{
    if (!sw || !bytes) return HS_ERR_ARG;
    if (S < 1 || S > HS_MAX_SWARMS) return HS_ERR_SIZE;
    long long total = 0;
    for (int s = 0; s < S; ++s) {
        if (sw[s].P < 1 || sw[s].P > HS_FUSED_MAX_PARTICLES) return HS_ERR_SIZE;
        total += sw[s].P;
    }
    if (total > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    *bytes = batch_bytes(S, total);
    return HS_OK;
}

int hs_batch_create(const HsModel* model, const HsSwarmDesc* sw, int S, void* buffer, size_t bytes,
                    hs_stream_t stream, HsBatch** out)
{
    if (!model || !sw || !buffer || !out) return HS_ERR_ARG;
    size_t need = 0;
    int rc = hs_batch_buffer_size(sw, S, &need);
    if (rc) return rc;
    if (bytes < need) return HS_ERR_SIZE;
    if ((reinterpret_cast<uintptr_t>(buffer) & 255u) != 0) return HS_ERR_ALIGN;
    for (int s = 0; s < S; ++s) {
        if ((rc = validate_obs(&sw[s].obs))) return rc;
        if ((rc = validate_cam(&sw[s].cam))) return rc;
        if (sw[s].n_mutate < 0 || sw[s].n_mutate > sw[s].P) return HS_ERR_ARG;
    }
    // host image of the buffer
    unsigned char* img = static_cast<unsigned char*>(std::calloc(1, need));
    if (!img) return HS_ERR_ARG;
    SwarmView* views = reinterpret_cast<SwarmView*>(img + 256);
    int32_t* sid = reinterpret_cast<int32_t*>(img + 256 + (size_t)S * sizeof(SwarmView));
    long long P_all = 0;
    for (int s = 0; s < S; ++s) P_all += sw[s].P;
    int32_t* order = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(sid) + table_bytes(P_all));
    int off = 0, P_max = 0, max_H = 0;
    for (int s = 0; s < S && rc == HS_OK; ++s) {
        const HsObs& o = sw[s].obs;
        const HsCamera& c = sw[s].cam;
        SwarmView& v = views[s];
        const bool f32 = o.depth_type == HS_DEPTH_F32;
        rc = encode_tile_map(&v.tm_depth, o.depth, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                             f32 ? 4 : 2, o.W, o.H, o.depth_pitch);
        if (rc == HS_OK)
            rc = encode_tile_map(&v.tm_skin, o.skin, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, o.W, o.H, o.skin_pitch);
        v.W = o.W;
        v.H = o.H;
        v.depth_f32 = f32;
        v.P = sw[s].P;
        v.offset = off;
        v.n_mutate = sw[s].n_mutate;
        v.depth_pitch = o.depth_pitch;
        v.skin_pitch = o.skin_pitch;
        v.inv_fx = (float)(1.0 / (double)c.fx);
        v.inv_fy = (float)(1.0 / (double)c.fy);
        v.off_x = (float)((0.5 - (double)c.cx) / (double)c.fx);
        v.off_y = (float)((0.5 - (double)c.cy) / (double)c.fy);
        v.fx = c.fx;
        v.fy = c.fy;
        v.cx = c.cx;
        v.cy = c.cy;
        v.depth = static_cast<const unsigned char*>(o.depth);
        v.skin = o.skin;
        v.stats = o.stats;
        v.key0 = (uint32_t)sw[s].seed;
        v.key1 = (uint32_t)(sw[s].seed >> 32);
        for (int i = 0; i < sw[s].P; ++i) sid[off + i] = s;
        off += sw[s].P;
        if (sw[s].P > P_max) P_max = sw[s].P;
        if (o.H > max_H) max_H = o.H;
    }
    // render order: swarms by decreasing ROI area (stable), each swarm's particles in
    // turn; CTAs start in this order, so the largest pieces of work go first
    if (rc == HS_OK) {
        std::vector<int> by_area(S);
        for (int s = 0; s < S; ++s) by_area[s] = s;
        std::stable_sort(by_area.begin(), by_area.end(), [&](int x, int y) {
            return (long long)views[x].W * views[x].H > (long long)views[y].W * views[y].H;
        });
        int k = 0;
        for (int s : by_area)
            for (int i = 0; i < views[s].P; ++i) order[k++] = views[s].offset + i;
    }
    if (rc == HS_OK && cudaMemcpyAsync(buffer, img, need, cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
        rc = HS_ERR_CUDA;
    if (rc == HS_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = HS_ERR_CUDA;
    std::free(img);
    if (rc) return rc;
    HsBatch* b = static_cast<HsBatch*>(std::calloc(1, sizeof(HsBatch)));
    if (!b) return HS_ERR_ARG;
    b->S = S;
    b->P_total = off;
    b->P_max = P_max;
    b->max_H = max_H;
    unsigned char* dev = static_cast<unsigned char*>(buffer);
    b->dev.S = S;
    b->dev.P_total = off;
    b->dev.views = reinterpret_cast<const SwarmView*>(dev + 256);
    b->dev.sid = reinterpret_cast<const int32_t*>(dev + 256 + (size_t)S * sizeof(SwarmView));
    b->order = reinterpret_cast<const int32_t*>(dev + 256 + (size_t)S * sizeof(SwarmView) + table_bytes(off));
    *out = b;
    return HS_OK;
}

int hs_batch_destroy(HsBatch* b)
{
    if (!b) return HS_ERR_ARG;
    std::free(b);
    return HS_OK;
}

int hs_batch_particles(const HsBatch* b, int* P_total)
{
    if (!b || !P_total) return HS_ERR_ARG;
    *P_total = b->P_total;
    return HS_OK;
}

int hs_obs_prepare_multi(const HsBatch* b, hs_stream_t stream)
{
    if (!b) return HS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    zero_stats_kernel<<<(b->S + 127) / 128, 128, 0, s>>>(b->dev);
    if (cudaGetLastError() != cudaSuccess) return HS_ERR_CUDA;
    return launch_obs_stats_multi(b->dev, b->max_H, s) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pose_fk_multi(const HsModel* model, const HsBatch* b, const float* poses, HsPrim* prims, float* kc,
                  hs_stream_t stream)
{
    if (!model || !b || !poses || !prims || !kc) return HS_ERR_ARG;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    FkArgs a = {};
    a.poses = poses;
    a.P = b->P_total;
    a.fx = a.fy = 1.f;
    a.prims = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    a.batch = b->dev;
    int rc = status_ptr(&a.status);
    if (rc) return rc;
    return launch_fk(model->dev, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int render_score_multi(const HsModel* model, const HsBatch* b, const HsPrim* prims, const float* kc,
                       const HsScoreParams* params, void* workspace, size_t workspace_bytes, float* E, HsParts* parts,
                       hs_stream_t stream)
{
    if (!model || !b || !prims || !kc || !params || !E || !workspace) return HS_ERR_ARG;
    int rc = validate_score_params(params);
    if (rc) return rc;
    if (!aligned16(prims) || !aligned16(workspace)) return HS_ERR_ALIGN;
    size_t need = 0;
    hs_workspace_size(b->P_total, &need);
    if (workspace_bytes < need) return HS_ERR_SIZE;
    RenderArgs a = {};
    a.prims = reinterpret_cast<const float4*>(prims);
    a.kc = kc;
    a.P = b->P_total;
    a.n_prims = model->dev.n_prims;
    a.work = static_cast<HsParticleWork*>(workspace);
    a.ctl = reinterpret_cast<RenderCtl*>(a.work + b->P_total);
    a.E = E;
    a.parts = parts;
    a.batch = b->dev;
    a.order = b->order;
    if ((rc = status_ptr(&a.status))) return rc;
    CUtensorMap unused = {};  // the maps come from the batch views
    return launch_render(*params, unused, unused, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pso_init_multi(const HsModel* model, const HsBatch* b, const HsSwarm* sw, const float* seed_poses,
                   const float* scale, uint32_t frame, hs_stream_t stream)
{
    if (!model || !b || !sw || !seed_poses || !scale) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E) return HS_ERR_ARG;
    PsoInitArgs a = {};
    a.x = sw->x;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.seed_pose = seed_poses;
    for (int d = 0; d < HS_NDOF; ++d) {
        if (!std::isfinite(scale[d]) || scale[d] < 0.f) return HS_ERR_ARG;
        a.scale[d] = scale[d];
    }
    a.P = b->P_total;
    a.frame = frame;
    a.batch = b->dev;
    return launch_pso_init(model->lim, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int pso_step_fk_multi(const HsModel* model, const HsBatch* b, const HsSwarm* sw, float* x_next,
                      const HsPsoParams* prm, uint32_t frame, uint32_t gen, HsPrim* prims, float* kc,
                      hs_stream_t stream)
{
    if (!model || !b || !sw || !prm || !x_next || !prims || !kc) return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E || !sw->E) return HS_ERR_ARG;
    if (x_next == sw->x) return HS_ERR_ARG;
    if (!aligned16(prims)) return HS_ERR_ALIGN;
    const double psi = (double)prm->c1 + (double)prm->c2;
    if (!std::isfinite(psi) || prm->c1 < 0.f || prm->c2 < 0.f || psi <= 4.0) return HS_ERR_ARG;
    if (!(prm->e_stop >= 0.f) || !std::isfinite(prm->e_stop)) return HS_ERR_ARG;
    PsoFkArgs a = {};
    a.x = sw->x;
    a.x_next = x_next;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.E = sw->E;
    a.P = b->P_max;  // shared memory for the largest swarm; each CTA uses its own swarm's size
    a.c1 = prm->c1;
    a.c2 = prm->c2;
    a.w = (float)(2.0 / std::fabs(2.0 - psi - std::sqrt(psi * psi - 4.0 * psi)));
    a.mutate = prm->mutate_every > 0 && gen % (uint32_t)prm->mutate_every == 0;
    a.frame = frame;
    a.gen = gen;
    a.e_stop = prm->e_stop;
    a.prims = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    a.batch = b->dev;
    int rc = status_ptr(&a.status);
    if (rc) return rc;
    return launch_pso_step_fk(model->dev, a, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// ---- a whole frame of every swarm of a batch in one cooperative launch ----------------

static size_t frame_multi_done_bytes(int S) { return ((size_t)S * 4 + 127) / 128 * 128; }

int hs_frame_multi_workspace_size(const HsBatch* b, size_t* bytes)
{
    if (!b || !bytes) return HS_ERR_ARG;
    *bytes = sizeof(FrameMultiCtl) + frame_multi_done_bytes(b->S) + 2 * (size_t)b->P_total * sizeof(float);
    return HS_OK;
}

int hs_frame_multi_capacity(const HsModel* model, const HsBatch* b, int* ctas)
{
    if (!ctas) return HS_ERR_ARG;
    const int P_max = b ? b->P_max : HS_FRAME_MAX_PARTICLES;
    if (P_max > HS_FRAME_MAX_PARTICLES) return HS_ERR_SIZE;
    const bool collide = model && frame_multi_needs_collide(model->dev);
    const int n_prims = model ? model->dev.n_prims : HS_MAX_PRIMS;
    return track_frame_multi_capacity(ctas, P_max, n_prims, collide) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

int track_frame_multi(const HsModel* model, const HsBatch* b, const HsSwarm* sw, float* x_next, int gens,
                      const HsScoreParams* score, const HsPsoParams* prm, const float* seed_poses,
                      const float* scale, uint32_t frame, int ctas, void* workspace, size_t workspace_bytes,
                      HsPrim* prims, float* kc, hs_stream_t stream)
{
    if (!model || !b || !sw || !x_next || !score || !prm || !seed_poses || !scale || !prims || !kc)
        return HS_ERR_ARG;
    if (!sw->x || !sw->v || !sw->pbest || !sw->pbest_E || !sw->gbest || !sw->gbest_E || !sw->E) return HS_ERR_ARG;
    if (x_next == sw->x || gens < 0 || ctas < 0) return HS_ERR_ARG;
    int rc = validate_score_params(score);
    if (rc) return rc;
    const double psi = (double)prm->c1 + (double)prm->c2;
    if (!std::isfinite(psi) || prm->c1 < 0.f || prm->c2 < 0.f || psi <= 4.0) return HS_ERR_ARG;
    if (prm->e_stop != 0.f) return HS_ERR_ARG;  // the stopping rule is the step-by-step batch calls'
    if (b->P_max > HS_FRAME_MAX_PARTICLES) return HS_ERR_SIZE;
    if ((long long)(gens + 1) * b->P_total > INT_MAX) return HS_ERR_SIZE;  // the task counter's range
    if (!workspace) return HS_ERR_ARG;
    if (!aligned16(prims) || !aligned16(workspace)) return HS_ERR_ALIGN;
    size_t need = 0;
    hs_frame_multi_workspace_size(b, &need);
    if (workspace_bytes < need) return HS_ERR_SIZE;
    FrameMultiArgs a = {};
    for (int d = 0; d < HS_NDOF; ++d) {
        if (!std::isfinite(scale[d]) || scale[d] < 0.f) return HS_ERR_ARG;
        a.scale[d] = scale[d];
    }
    int cap = 0;
    if (track_frame_multi_capacity(&cap, b->P_max, model->dev.n_prims, frame_multi_needs_collide(model->dev)) !=
        cudaSuccess)
        return HS_ERR_CUDA;  // for this batch's swarms and this model's kernel
    const int nb = ctas ? ctas : cap;
    if (nb < 1 || nb > cap) return HS_ERR_SIZE;
    a.batch = b->dev;
    a.order = b->order;
    a.d_m = score->d_m;
    a.d_M = score->d_M;
    a.lambda = score->lambda;
    a.lambda_k = score->lambda_k;
    a.xbuf[0] = sw->x;
    a.xbuf[1] = x_next;
    a.v = sw->v;
    a.pbest = sw->pbest;
    a.pbest_E = sw->pbest_E;
    a.gbest = sw->gbest;
    a.gbest_E = sw->gbest_E;
    a.E = const_cast<float*>(sw->E);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    a.ctl = reinterpret_cast<FrameMultiCtl*>(ws);
    a.done = reinterpret_cast<uint32_t*>(ws + sizeof(FrameMultiCtl));
    a.Ebuf = reinterpret_cast<float*>(ws + sizeof(FrameMultiCtl) + frame_multi_done_bytes(b->S));
    a.prims_out = reinterpret_cast<float4*>(prims);
    a.kc = kc;
    a.seed_poses = seed_poses;
    a.c1 = prm->c1;
    a.c2 = prm->c2;
    a.w = (float)(2.0 / std::fabs(2.0 - psi - std::sqrt(psi * psi - 4.0 * psi)));
    a.mutate_every = prm->mutate_every;
    a.frame = frame;
    a.gens = gens;
    a.P_max = b->P_max;
    if ((rc = status_ptr(&a.status))) return rc;
    // the frame's observation totals (as hs_obs_prepare_multi), then the frame
    if ((rc = hs_obs_prepare_multi(b, stream))) return rc;
    return launch_track_frame_multi(model->dev, a, nb, (cudaStream_t)stream) == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// ---- render autotuning -------------------------------------------------------------

}  // extern "C"

namespace {
constexpr int kTuneCtas[HS_TUNE_CTAS] = {0, 1, 2, 3, 4, 6, 8, 16, 32};  // 0: the automatic choice

// Times every (kernel, CTAs per particle) candidate of one render call and keeps
// the fastest.  Each candidate's `reps` calls are captured into a CUDA graph on
// a private stream (so host-side set-up does not pace them, as in a tracker's
// graph) after one eager call, and the graph is launched once untimed and once
// between two CUDA events.
// launch(params, stream) issues one call.
template <class Launch>
int autotune(HsScoreParams* params, int P, int reps, float* times_us, cudaStream_t stream, Launch&& launch)
{
    if (reps < 1 || reps > 1000) return HS_ERR_ARG;
    if (times_us)
        for (int i = 0; i < HS_RENDER_VARIANTS * HS_TUNE_CTAS; ++i) times_us[i] = -1.f;
    cudaStream_t cs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HS_OK;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess)
        rc = HS_ERR_CUDA;
    HsScoreParams best = *params;
    float best_us = INFINITY;
    for (int v = HS_RENDER_UNITS; v < HS_RENDER_VARIANTS && rc == HS_OK; ++v) {
        for (int c = 0; c < HS_TUNE_CTAS && rc == HS_OK; ++c) {
            // more CTAs per particle only while the launch stays within a few waves
            if (kTuneCtas[c] > 1 && (long long)kTuneCtas[c] * P > 4LL * kTargetCtas) break;
            // the persistent launches deal whole particles: no CTAs-per-particle choice
            if (c > 0 && (v == HS_RENDER_PERSISTENT_8x16 || v == HS_RENDER_PERSISTENT_8x32)) break;
            HsScoreParams cand = *params;
            cand.variant = v;
            cand.ctas_per_particle = kTuneCtas[c];
            // one eager call first: lazy set-up (module loading, symbol lookups,
            // the shared-memory opt-in) must not happen during capture
            if ((rc = launch(cand, cs)) != HS_OK) break;
            if (cudaStreamSynchronize(cs) != cudaSuccess) {
                rc = HS_ERR_CUDA;
                break;
            }
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = HS_ERR_CUDA;
                break;
            }
            int lrc = HS_OK;
            for (int r = 0; r < reps && lrc == HS_OK; ++r) lrc = launch(cand, cs);
            const cudaError_t ec = cudaStreamEndCapture(cs, &g);
            if (lrc != HS_OK || ec != cudaSuccess) rc = lrc != HS_OK ? lrc : HS_ERR_CUDA;
            if (rc == HS_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) rc = HS_ERR_CUDA;
            float ms = 0.f;
            if (rc == HS_OK &&
                (cudaGraphLaunch(ge, cs) != cudaSuccess || cudaEventRecord(e0, cs) != cudaSuccess ||
                 cudaGraphLaunch(ge, cs) != cudaSuccess || cudaEventRecord(e1, cs) != cudaSuccess ||
                 cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = HS_ERR_CUDA;
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (rc != HS_OK) break;
            const float us = ms * 1e3f / (float)reps;
            if (times_us) times_us[v * HS_TUNE_CTAS + c] = us;
            if (us < best_us) {
                best_us = us;
                best = cand;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cs) cudaStreamDestroy(cs);
    if (rc == HS_OK) *params = best;
    return rc;
}
}  // namespace

extern "C" {

int render_score_batch_autotune(const HsModel* model, const HsObs* obs, const HsCamera* cam, const HsPrim* prims,
                                const float* kc, int P, HsScoreParams* params, void* workspace,
                                size_t workspace_bytes, float* E, int reps, float* times_us, hs_stream_t stream)
{
    if (!params) return HS_ERR_ARG;
    // every argument is checked by a call that launches nothing
    int rc = render_score_batch(model, obs, cam, prims, kc, 0, params, workspace, workspace_bytes, E, nullptr,
                                nullptr, nullptr, stream);
    if (rc) return rc;
    if (P < 1 || P > HS_MAX_PARTICLES) return HS_ERR_SIZE;
    return autotune(params, P, reps, times_us, (cudaStream_t)stream, [&](const HsScoreParams& c, cudaStream_t cs) {
        return render_score_batch(model, obs, cam, prims, kc, P, &c, workspace, workspace_bytes, E, nullptr, nullptr,
                                  nullptr, (hs_stream_t)cs);
    });
}

int render_score_multi_autotune(const HsModel* model, const HsBatch* batch, const HsPrim* prims, const float* kc,
                                HsScoreParams* params, void* workspace, size_t workspace_bytes, float* E, int reps,
                                float* times_us, hs_stream_t stream)
{
    if (!model || !batch || !params) return HS_ERR_ARG;
    int rc = validate_score_params(params);
    if (rc) return rc;
    return autotune(params, batch->P_total, reps, times_us, (cudaStream_t)stream,
                    [&](const HsScoreParams& c, cudaStream_t cs) {
                        return render_score_multi(model, batch, prims, kc, &c, workspace, workspace_bytes, E, nullptr,
                                                  (hs_stream_t)cs);
                    });
}

int hs_get_device_status(uint32_t* out, int clear)
{
    if (!out) return HS_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return HS_ERR_CUDA;
    if (cudaMemcpyFromSymbol(out, g_status, sizeof(uint32_t)) != cudaSuccess) return HS_ERR_CUDA;
    if (clear) {
        const uint32_t z = 0;
        if (cudaMemcpyToSymbol(g_status, &z, sizeof(uint32_t)) != cudaSuccess) return HS_ERR_CUDA;
    }
    return HS_OK;
}

}  // extern "C"
