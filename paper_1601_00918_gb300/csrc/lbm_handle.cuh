// The single-grid handle (struct lbm_t of include/lbm.h) and the launchers of
// its step kernels.  The runtime (lbm_capi.cu) owns the handle; every family
// of step kernels is instantiated in a translation unit of its own
// (lbm_k_staged.cu, lbm_k_warp.cu, lbm_k_private.cu, lbm_k_simple.cu), so the
// five storage formats of each family compile in parallel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/lbm.h"
#include "lbm_common.cuh"

namespace gb300lbm {

constexpr int kBX = 128;         // columns per CTA of the simple kernel
constexpr int kRowBlock = 64;    // column granularity of the fluid-row table
constexpr int kGraphSteps = 32;  // steps per captured graph (even: parity is kept)

struct Tuned {
    int variant = 1;   // 1 simple, 2 staged, 3 pipelined, 4 private
    int depth = 2;     // staged: rows issued ahead of the three in use (1 or 2)
    int rpb = 16;      // simple: rows per CTA strip
    int strips = 1;    // staged: strips per column block
    int bx = 128;      // staged: columns per CTA (64 or 128)
    int strip_abs = 0; // staged: strips at absolute rows (Grid::strip_rows)
};

}  // namespace gb300lbm

struct lbm_t {
    lbm_params p{};
    int pitch = 0;
    int ncb = 0;                  // 128-column blocks
    int nrb = 0;                  // 64-column blocks of the fluid-row table
    size_t elem = 0;              // bytes per stored population
    size_t buf_bytes = 0;         // one population buffer
    void* arena = nullptr;
    bool own_arena = false;
    char* fbase[2] = {nullptr, nullptr};   // buffer starts (storage column 0)
    int cur = 0;                  // fbase[cur] holds the current stored state
    uint16_t* links = nullptr;    // storage column 0 of row 0
    int2* rows = nullptr;
    gb300lbm::StepParams* dprm = nullptr;
    gb300lbm::ObsAccum* dacc = nullptr;
    gb300lbm::ObsState* dobs = nullptr;
    gb300lbm::ObsAccum* tacc = nullptr;     // autotuning scratch
    gb300lbm::ObsState* tobs = nullptr;
    gb300lbm::StepParams hprm{};
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;       // private stream for graph capture
    CUtensorMap fmap[2][2];       // [buffer][box width 64 + 16 or 128 + 16] (pipelined kernel)
    CUtensorMap lmap[2];          // link words, box width 64 + 16 or 128 + 16
    CUtensorMap smap[2][2];       // [buffer][64 or 128 columns] windows of the staged kernel
    CUtensorMap pmap[2];          // [buffer] per-warp windows of the private kernel
    CUtensorMap plmap;
    bool maps_ok = false;
    gb300lbm::Tuned tune;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t fluid_nodes = 0;
    // persistent multi-step launches (small grids): 0 undecided, 1 used, -1 not used
    int persist = 0;
    int persist_rpb = 8;          // rows per tile of the persistent march
    int persist_ctas = 0;         // resident CTAs of one cooperative launch
    std::string err;
};

namespace gb300lbm {

inline Grid make_grid(const lbm_t* h, int row_begin, int row_end) {
    Grid g;
    g.nx = h->p.nx;
    g.ny = h->p.ny;
    g.pitch = h->pitch;
    g.periodic_x = h->p.periodic_x;
    g.rows_per_block = h->tune.rpb;
    g.row_begin = row_begin;
    g.row_end = row_end;
    g.strips = h->tune.strips;
    g.strip_rows = 0;
    return g;
}

template <typename S>
S* at_col0(char* base) {
    return (S*)base + kGhost;
}

// One step fin = fbase[src] -> fbase[1 - src] with launch configuration tn,
// observables reduced into acc / finalised into obs; the family is tn.variant
// and the storage format h->p.precision.
cudaError_t launch_staged_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st);
cudaError_t launch_pipelined_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs,
                                 cudaStream_t st);
cudaError_t launch_private_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st);
cudaError_t launch_simple_any(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st);
// Macroscopic fields of fbase[cur], rows [rb, re), into out (device).
cudaError_t launch_fields(lbm_t* h, double* out, int rb, int re);
// nsteps steps in one cooperative launch (h->persist_ctas CTAs).
cudaError_t launch_persist(lbm_t* h, int nsteps);

// Resident CTAs per SM of one configuration of a family (0: cannot launch).
int occupancy_staged(int prec, int bx, int depth);
int occupancy_pipelined(int prec, int bx, int depth);
int occupancy_private(int prec, int bx, int depth);
int persist_occupancy_of(int prec);

// Resident CTAs per SM of `kernel` with `threads` threads and `smem` bytes of
// dynamic shared memory (0 if it cannot launch).
template <typename K>
int occupancy_of(K kernel, int threads, int smem) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace gb300lbm
