// Instantiations and launchers of the private step kernel (lbm_step_private.cuh)
// for the five storage formats.
#include "lbm_handle.cuh"
#include "lbm_step_private.cuh"

namespace gb300lbm {
namespace {

template <typename S, int BX, int D>
cudaError_t launch_private(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs,
                          cudaStream_t st) {
    using Plan = PrivatePlan<S, BX / 32, D>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(step_private_kernel<S, BX, D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Plan::kBytes);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    Grid g = make_grid(h, 0, h->p.ny);
    g.strips = tn.strips;
    dim3 grid((h->p.nx + BX - 1) / BX, tn.strips);
    step_private_kernel<S, BX, D><<<grid, BX, Plan::kBytes, st>>>(
        h->pmap[src], h->plmap, at_col0<S>(h->fbase[1 - src]), h->rows,
        h->dprm, acc, obs, g);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_prec(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    if (tn.bx == 64) {
        if (tn.depth >= 2) return launch_private<S, 64, 2>(h, src, tn, acc, obs, st);
        return launch_private<S, 64, 1>(h, src, tn, acc, obs, st);
    }
    if (tn.depth >= 2) return launch_private<S, 128, 2>(h, src, tn, acc, obs, st);
    return launch_private<S, 128, 1>(h, src, tn, acc, obs, st);
}

template <typename S>
int occupancy_prec(int bx, int depth) {
    if (bx == 64)
        return depth >= 2 ? occupancy_of(step_private_kernel<S, 64, 2>, 64, PrivatePlan<S, 2, 2>::kBytes)
                          : occupancy_of(step_private_kernel<S, 64, 1>, 64, PrivatePlan<S, 2, 1>::kBytes);
    return depth >= 2 ? occupancy_of(step_private_kernel<S, 128, 2>, 128, PrivatePlan<S, 4, 2>::kBytes)
                      : occupancy_of(step_private_kernel<S, 128, 1>, 128, PrivatePlan<S, 4, 1>::kBytes);
}

}  // namespace

cudaError_t launch_private_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    switch (h->p.precision) {
        case LBM_FP64: return launch_prec<double>(h, src, tn, acc, obs, st);
        case LBM_FP32: return launch_prec<float>(h, src, tn, acc, obs, st);
        case LBM_FP32C: return launch_prec<f32c>(h, src, tn, acc, obs, st);
        case LBM_FP16S: return launch_prec<__half>(h, src, tn, acc, obs, st);
        default: return launch_prec<__nv_bfloat16>(h, src, tn, acc, obs, st);
    }
}

int occupancy_private(int prec, int bx, int depth) {
    switch (prec) {
        case LBM_FP64: return occupancy_prec<double>(bx, depth);
        case LBM_FP32: return occupancy_prec<float>(bx, depth);
        case LBM_FP32C: return occupancy_prec<f32c>(bx, depth);
        case LBM_FP16S: return occupancy_prec<__half>(bx, depth);
        default: return occupancy_prec<__nv_bfloat16>(bx, depth);
    }
}

}  // namespace gb300lbm
