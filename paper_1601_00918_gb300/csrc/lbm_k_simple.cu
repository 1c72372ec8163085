// Instantiations and launchers of the simple step kernel, the fields pass and
// the persistent multi-step kernel (lbm_step.cuh) for the five storage
// formats.
#include "lbm_handle.cuh"
#include "lbm_step.cuh"

namespace gb300lbm {
namespace {

template <typename S>
cudaError_t launch_simple_t(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    Grid g = make_grid(h, 0, h->p.ny);
    g.rows_per_block = tn.rpb;
    dim3 grid(h->ncb, (h->p.ny + tn.rpb - 1) / tn.rpb);
    step_simple_kernel<S, kBX, false><<<grid, kBX, 0, st>>>(
        at_col0<S>(h->fbase[src]), at_col0<S>(h->fbase[1 - src]), h->links + kGhost, h->dprm, acc, obs,
        nullptr, g);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_fields_t(lbm_t* h, double* out, int rb, int re) {
    Grid g = make_grid(h, rb, re);
    g.rows_per_block = 8;
    dim3 grid(h->ncb, (re - rb + 7) / 8);
    step_simple_kernel<S, kBX, true><<<grid, kBX, 0, h->stream>>>(
        at_col0<S>(h->fbase[h->cur]), nullptr, h->links + kGhost, h->dprm, h->dacc, h->dobs, out, g);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_persist_t(lbm_t* h, int nsteps) {
    Grid g = make_grid(h, 0, h->p.ny);
    g.rows_per_block = h->persist_rpb;
    S* f0 = at_col0<S>(h->fbase[0]);
    S* f1 = at_col0<S>(h->fbase[1]);
    const uint16_t* lk = h->links + kGhost;
    int parity = h->cur;
    void* args[] = {(void*)&f0, (void*)&f1, (void*)&lk, (void*)&h->dprm, (void*)&h->dacc, (void*)&h->dobs,
                    (void*)&g, (void*)&nsteps, (void*)&parity};
    return cudaLaunchCooperativeKernel((const void*)step_persist_kernel<S, kBX>, dim3(h->persist_ctas), dim3(kBX),
                                       args, 0, h->stream);
}

template <typename S>
int persist_occupancy() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_persist_kernel<S, kBX>, kBX, 0) != cudaSuccess) return 0;
    return n;
}

}  // namespace

cudaError_t launch_simple_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    switch (h->p.precision) {
        case LBM_FP64: return launch_simple_t<double>(h, src, tn, acc, obs, st);
        case LBM_FP32: return launch_simple_t<float>(h, src, tn, acc, obs, st);
        case LBM_FP32C: return launch_simple_t<f32c>(h, src, tn, acc, obs, st);
        case LBM_FP16S: return launch_simple_t<__half>(h, src, tn, acc, obs, st);
        default: return launch_simple_t<__nv_bfloat16>(h, src, tn, acc, obs, st);
    }
}

cudaError_t launch_fields(lbm_t* h, double* out, int rb, int re) {
    switch (h->p.precision) {
        case LBM_FP64: return launch_fields_t<double>(h, out, rb, re);
        case LBM_FP32: return launch_fields_t<float>(h, out, rb, re);
        case LBM_FP32C: return launch_fields_t<f32c>(h, out, rb, re);
        case LBM_FP16S: return launch_fields_t<__half>(h, out, rb, re);
        default: return launch_fields_t<__nv_bfloat16>(h, out, rb, re);
    }
}

cudaError_t launch_persist(lbm_t* h, int nsteps) {
    switch (h->p.precision) {
        case LBM_FP64: return launch_persist_t<double>(h, nsteps);
        case LBM_FP32: return launch_persist_t<float>(h, nsteps);
        case LBM_FP32C: return launch_persist_t<f32c>(h, nsteps);
        case LBM_FP16S: return launch_persist_t<__half>(h, nsteps);
        default: return launch_persist_t<__nv_bfloat16>(h, nsteps);
    }
}

int persist_occupancy_of(int prec) {
    switch (prec) {
        case LBM_FP64: return persist_occupancy<double>();
        case LBM_FP32: return persist_occupancy<float>();
        case LBM_FP32C: return persist_occupancy<f32c>();
        case LBM_FP16S: return persist_occupancy<__half>();
        default: return persist_occupancy<__nv_bfloat16>();
    }
}

}  // namespace gb300lbm
