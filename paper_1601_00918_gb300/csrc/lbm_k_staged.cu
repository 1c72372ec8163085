// Instantiations and launchers of the staged step kernel (lbm_step_tma.cuh)
// for the five storage formats.
#include "lbm_handle.cuh"
#include "lbm_step_tma.cuh"

namespace gb300lbm {
namespace {

template <typename S, int BX, int D, int kReg>
cudaError_t launch_staged_reg(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs,
                              cudaStream_t st) {
    using Plan = StagedPlan<S, BX, D>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(step_staged_kernel<S, BX, D, kReg>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Plan::kBytes);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    Grid g = make_grid(h, 0, h->p.ny);
    g.strips = tn.strips;
    g.strip_rows = tn.strip_abs ? (h->p.ny + tn.strips - 1) / tn.strips : 0;
    dim3 grid((h->p.nx + BX - 1) / BX, tn.strips);
    step_staged_kernel<S, BX, D, kReg><<<grid, BX, Plan::kBytes, st>>>(
        h->smap[src][BX == 64 ? 0 : 1], h->lmap[BX == 64 ? 0 : 1], at_col0<S>(h->fbase[1 - src]), h->rows,
        h->dprm, acc, obs, g);
    return cudaGetLastError();
}

// The collision is fixed per handle (lbm_params.collision): one kernel per
// collision, without the other's branch.
template <typename S, int BX, int D>
cudaError_t launch_staged(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs,
                          cudaStream_t st) {
    if (h->p.collision == 1) return launch_staged_reg<S, BX, D, 1>(h, src, tn, acc, obs, st);
    return launch_staged_reg<S, BX, D, 0>(h, src, tn, acc, obs, st);
}

template <typename S>
cudaError_t launch_prec(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    if (tn.bx == 64) {
        if (tn.depth >= 2) return launch_staged<S, 64, 2>(h, src, tn, acc, obs, st);
        return launch_staged<S, 64, 1>(h, src, tn, acc, obs, st);
    }
    if (tn.depth >= 2) return launch_staged<S, 128, 2>(h, src, tn, acc, obs, st);
    return launch_staged<S, 128, 1>(h, src, tn, acc, obs, st);
}

template <typename S, int BX, int D>
int occupancy_one() {
    return occupancy_of(step_staged_kernel<S, BX, D, 0>, BX, StagedPlan<S, BX, D>::kBytes);
}

template <typename S>
int occupancy_prec(int bx, int depth) {
    if (bx == 64)
        return depth >= 2 ? occupancy_one<S, 64, 2>() : occupancy_one<S, 64, 1>();
    return depth >= 2 ? occupancy_one<S, 128, 2>() : occupancy_one<S, 128, 1>();
}

}  // namespace

cudaError_t launch_staged_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    switch (h->p.precision) {
        case LBM_FP64: return launch_prec<double>(h, src, tn, acc, obs, st);
        case LBM_FP32: return launch_prec<float>(h, src, tn, acc, obs, st);
        case LBM_FP32C: return launch_prec<f32c>(h, src, tn, acc, obs, st);
        case LBM_FP16S: return launch_prec<__half>(h, src, tn, acc, obs, st);
        default: return launch_prec<__nv_bfloat16>(h, src, tn, acc, obs, st);
    }
}

int occupancy_staged(int prec, int bx, int depth) {
    switch (prec) {
        case LBM_FP64: return occupancy_prec<double>(bx, depth);
        case LBM_FP32: return occupancy_prec<float>(bx, depth);
        case LBM_FP32C: return occupancy_prec<f32c>(bx, depth);
        case LBM_FP16S: return occupancy_prec<__half>(bx, depth);
        default: return occupancy_prec<__nv_bfloat16>(bx, depth);
    }
}

}  // namespace gb300lbm
