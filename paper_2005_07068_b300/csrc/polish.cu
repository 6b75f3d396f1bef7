// polish.cu -- the gradient polish of the best particles (the hybrid of PSO
// with descent on the smoothed objective E_s).
//
// Once a generation's objectives E are known, the k best particles (lowest E,
// lower index on ties) are copied out, take a few normalised descent steps on
// E_s (soft_score, soft_score_backward, pose_grad), and are scored again with
// the exact objective E; each keeps its polished pose only if that lowered
// its E.  The swarm update (Eq. 6-7) then proceeds as in plain PSO.
#include "hs_args.cuh"

namespace hs {

// rank of particle i among the P objectives (ascending, lower index first on
// ties, NaN last); the k best write their index into sel
__global__ void __launch_bounds__(256) select_best_kernel(const float* E, int P, int k, int32_t* sel)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float ei = E[i];
    const bool ni = !(ei == ei);
    int rank = 0;
    for (int j = 0; j < P; ++j) {
        const float ej = E[j];
        const bool nj = !(ej == ej);
        const bool before = ni ? (!nj || j < i) : (!nj && (ej < ei || (ej == ei && j < i)));
        rank += before && j != i;
    }
    if (rank < k) sel[rank] = i;
}

// x_sel[r] = x[sel[r]], E_sel[r] = E[sel[r]]
__global__ void __launch_bounds__(64) gather_kernel(const float* x, const float* E, const int32_t* sel, int k,
                                                    float* x_sel, float* E_sel)
{
    const int r = blockIdx.x, t = threadIdx.x;
    if (r >= k) return;
    const int i = sel[r];
    if (t < kNdof) x_sel[(size_t)r * kNdof + t] = x[(size_t)i * kNdof + t];
    if (t == 0) E_sel[r] = E[i];
}

// one normalised descent step per particle: x <- clamp(x - eta S^2 g / |S g|)
// (S = per-parameter scale; the step moves eta in scaled units)
__global__ void __launch_bounds__(64) polish_step_kernel(float* x, const float* grad, int k, PolishStep st)
{
    const int r = blockIdx.x, t = threadIdx.x;
    __shared__ float red[2];
    float sg = 0.f;
    if (t < kNdof) {
        const float v = st.scale[t] * grad[(size_t)r * kNdof + t];
        sg = v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
    if ((t & 31) == 0) red[t >> 5] = sg;
    __syncthreads();
    const float norm = sqrtf(red[0] + red[1]);
    if (t < kNdof && r < k && norm > 0.f && isfinite(norm)) {
        const float d = st.eta * st.scale[t] * st.scale[t] * grad[(size_t)r * kNdof + t] / norm;
        const float xv = x[(size_t)r * kNdof + t] - d;
        x[(size_t)r * kNdof + t] = fminf(fmaxf(xv, st.lo[t]), st.hi[t]);
    }
}

// keep the polished pose where it lowered E: x[sel[r]] = x_sel[r], E[sel[r]] = E_new[r]
__global__ void __launch_bounds__(64) keep_better_kernel(float* x, float* E, const int32_t* sel, int k,
                                                         const float* x_sel, const float* E_old, const float* E_new)
{
    const int r = blockIdx.x, t = threadIdx.x;
    if (r >= k) return;
    const float en = E_new[r];
    if (!(en < E_old[r])) return;  // not better (or NaN): the particle keeps its pose
    const int i = sel[r];
    if (t < kNdof) x[(size_t)i * kNdof + t] = x_sel[(size_t)r * kNdof + t];
    if (t == 0) E[i] = en;
}

cudaError_t launch_select_best(const float* E, int P, int k, int32_t* sel, cudaStream_t s)
{
    select_best_kernel<<<(P + 255) / 256, 256, 0, s>>>(E, P, k, sel);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float* x, const float* E, const int32_t* sel, int k, float* x_sel, float* E_sel,
                          cudaStream_t s)
{
    gather_kernel<<<k, 64, 0, s>>>(x, E, sel, k, x_sel, E_sel);
    return cudaGetLastError();
}

cudaError_t launch_polish_step(float* x, const float* grad, int k, const PolishStep& st, cudaStream_t s)
{
    polish_step_kernel<<<k, 64, 0, s>>>(x, grad, k, st);
    return cudaGetLastError();
}

cudaError_t launch_keep_better(float* x, float* E, const int32_t* sel, int k, const float* x_sel, const float* E_old,
                               const float* E_new, cudaStream_t s)
{
    keep_better_kernel<<<k, 64, 0, s>>>(x, E, sel, k, x_sel, E_old, E_new);
    return cudaGetLastError();
}

}  // namespace hs
