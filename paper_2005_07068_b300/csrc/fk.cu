// fk.cu -- batched forward kinematics (Eq. 1-3, Section II.A; Tables 1-2):
// 64 threads per particle, the body in hs_fk.cuh.
#include <algorithm>

#include "hs_fk.cuh"

namespace hs {

// M: DevModelCore for the paper's kc (a smaller launch parameter), DevModel
// when a kc variant needs the collision data.  Each CTA takes particles p =
// blockIdx.x, + gridDim.x, ... (at most the resident CTAs are launched, so the
// model is copied into shared memory once per CTA, not once per particle).
template <class M>
__global__ void __launch_bounds__(64, 8) fk_kernel(const __grid_constant__ M model_param, const FkArgs a)
{
    __shared__ FkShared sh;
    __shared__ CollideSmem<M> s_col;
    fk_load_model(sh, model_param);
    const CollideShared* col = collide_load(s_col, model_param);
    for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
        float4 cam = make_float4(a.fx, a.fy, a.cx, a.cy);
        if (a.batch.views) {  // the camera of this particle's swarm
            const SwarmView& v = a.batch.views[a.batch.sid[p]];
            cam = make_float4(v.fx, v.fy, v.cx, v.cy);
        }
        fk_particle(sh, col, a.poses + (size_t)p * kNdof, cam,
                    a.prims + (size_t)p * model_param.n_prims * 4, a.kc + p, a.status);
        __syncthreads();  // this particle's shared state is no longer read
    }
}

template <class M>
static cudaError_t launch_fk_as(const M& model, const FkArgs& args, cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0, grid = args.P;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk_kernel<M>, 64, 0) == cudaSuccess && sms * per_sm > 0)
        grid = std::min(args.P, sms * per_sm);
    fk_kernel<M><<<grid, 64, 0, stream>>>(model, args);
    return cudaGetLastError();
}

cudaError_t launch_fk(const DevModel& model, const FkArgs& args, cudaStream_t stream)
{
    if (model.kc_variant == HS_KC_ABDUCTION) return launch_fk_as(static_cast<const DevModelCore&>(model), args, stream);
    return launch_fk_as(model, args, stream);
}

}  // namespace hs
