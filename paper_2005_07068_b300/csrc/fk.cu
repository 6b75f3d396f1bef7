// fk.cu -- batched forward kinematics (Eq. 1-3, Section II.A; Tables 1-2):
// one 64-thread CTA per particle, the body in hs_fk.cuh.
#include "hs_fk.cuh"

namespace hs {

// M: DevModelCore for the paper's kc (a smaller launch parameter), DevModel
// when a kc variant needs the collision data
template <class M>
__global__ void __launch_bounds__(64) fk_kernel(const __grid_constant__ M model_param, const FkArgs a)
{
    __shared__ FkShared sh;
    fk_load_model(sh, model_param);
    const int p = blockIdx.x;
    float4 cam = make_float4(a.fx, a.fy, a.cx, a.cy);
    if (a.batch.views) {  // the camera of this particle's swarm
        const SwarmView& v = a.batch.views[a.batch.sid[p]];
        cam = make_float4(v.fx, v.fy, v.cx, v.cy);
    }
    fk_particle(sh, collide_data(model_param), a.poses + (size_t)p * kNdof, cam, a.prims + (size_t)p * model_param.n_prims * 4, a.kc + p,
                a.status);
}

cudaError_t launch_fk(const DevModel& model, const FkArgs& args, cudaStream_t stream)
{
    if (model.kc_variant == HS_KC_ABDUCTION)
        fk_kernel<DevModelCore><<<args.P, 64, 0, stream>>>(static_cast<const DevModelCore&>(model), args);
    else
        fk_kernel<DevModel><<<args.P, 64, 0, stream>>>(model, args);
    return cudaGetLastError();
}

}  // namespace hs
