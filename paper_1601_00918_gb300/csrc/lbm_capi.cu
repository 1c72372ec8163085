// Runtime and C ABI (include/lbm.h) of the two-component D2Q9 library.
//
// A handle owns, in one device arena (allocated here or supplied by the
// caller):
//   - two population buffers A/B (ping-pong), layout
//     f[species][direction][y][pitch] with 8 ghost columns on each side of
//     every row (see lbm_common.cuh), pitch a multiple of 32 elements;
//   - a 16-bit link word per node (bit i: the pull source x - c_i is solid,
//     bit 15: the node is solid), same row layout;
//   - the fluid row range of every 128-column block (the staged kernel
//     marches only over rows that hold fluid in its columns);
//   - the device parameter block, the per-step reduction accumulators and
//     the finalised observables (plus a spare pair used while autotuning).
// Steps run as one kernel launch each; runs of 32 steps are replayed from a
// captured CUDA graph.  The step kernel and its launch shape are picked by
// timing candidates on the handle's own data (autotuner, cached per grid
// shape, precision and periodicity).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_handle.cuh"
#include "lbm_step.cuh"
#include "lbm_step_private.cuh"
#include "lbm_setup.cuh"

using namespace gb300lbm;

namespace {

thread_local std::string g_create_err;

int fail(lbm_t* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_err = buf;
    return code;
}

#define CUDA_TRY(h, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

size_t elem_size(int prec) {
    switch (prec) {
        case LBM_FP64: return 8;
        case LBM_FP32:
        case LBM_FP32C: return 4;
        case LBM_FP16S:
        case LBM_BF16S: return 2;
        default: return 0;
    }
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// planes per buffer: 18 populations, plus the two density planes of the
// 16-bit node-shifted formats
int planes_of(int prec) { return (prec == LBM_FP16S || prec == LBM_BF16S) ? 20 : 18; }

struct Layout {
    int pitch, ncb, nrb;
    size_t buf, links, rows, prm, acc, obs, total;
};

bool layout_of(const lbm_params* p, Layout* L) {
    const size_t es = elem_size(p->precision);
    if (es == 0 || p->nx < 1 || p->ny < 1) return false;
    if (p->nx > (1 << 24) || p->ny > (1 << 24)) return false;
    L->pitch = (p->nx + 2 * kGhost + 31) / 32 * 32;
    L->ncb = (p->nx + kBX - 1) / kBX;
    L->nrb = (p->nx + kRowBlock - 1) / kRowBlock;
    const size_t plane = (size_t)p->ny * L->pitch;
    const size_t np = (size_t)planes_of(p->precision);
    // kernel indices are 32-bit: all planes must stay below 2^31 elements
    if (plane * np >= (size_t(1) << 31)) return false;
    L->buf = align256(plane * np * es);
    L->links = align256(plane * sizeof(uint16_t));
    L->rows = align256((size_t)L->nrb * sizeof(int2));
    L->prm = align256(sizeof(StepParams));
    L->acc = align256(sizeof(ObsAccum));
    L->obs = align256(sizeof(ObsState));
    L->total = 2 * L->buf + L->links + L->rows + L->prm + 2 * L->acc + 2 * L->obs;
    return true;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
cudaError_t launch_step(lbm_t* h, int src, const Tuned& tn, ObsAccum* acc, ObsState* obs, cudaStream_t st) {
    switch (tn.variant) {
        case 2: return launch_staged_any(h, src, tn, acc, obs, st);
        case 3: return launch_pipelined_any(h, src, tn, acc, obs, st);
        case 4: return launch_private_any(h, src, tn, acc, obs, st);
        default: return launch_simple_any(h, src, tn, acc, obs, st);
    }
}

// ---------------------------------------------------------------------------
// tensor maps for the staged kernel
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

bool make_maps(lbm_t* h) {
    auto fn = encode_fn();
    if (!fn) return false;
    CUtensorMapDataType dt;
    switch (h->p.precision) {
        case LBM_FP64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
        case LBM_FP32:
        case LBM_FP32C: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
        case LBM_FP16S: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        default: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    }
    const cuuint32_t np = (cuuint32_t)planes_of(h->p.precision);
    for (int k = 0; k < 2; k++) {
        const cuuint32_t W = (k ? 128 : 64) + 2 * kGhost;
        for (int b = 0; b < 2; b++) {
            cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny, np};
            cuuint64_t strides[2] = {(cuuint64_t)h->pitch * h->elem, (cuuint64_t)h->p.ny * h->pitch * h->elem};
            cuuint32_t box[3] = {W, 1, np};
            cuuint32_t es[3] = {1, 1, 1};
            if (fn(&h->fmap[b][k], dt, 3, h->fbase[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
        cuuint64_t dims[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny};
        cuuint64_t strides[1] = {(cuuint64_t)h->pitch * 2};
        cuuint32_t box[2] = {W, 1};
        cuuint32_t es[2] = {1, 1};
        if (fn(&h->lmap[k], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h->links, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    // windows of the staged kernel (StagedPlan: block width + twice the lead)
    for (int k = 0; k < 2; k++) {
        cuuint32_t W = 0;
        switch (h->p.precision) {
            case LBM_FP64: W = k ? StagedPlan<double, 128, 1>::kW : StagedPlan<double, 64, 1>::kW; break;
            case LBM_FP32:
            case LBM_FP32C: W = k ? StagedPlan<float, 128, 1>::kW : StagedPlan<float, 64, 1>::kW; break;
            default: W = k ? StagedPlan<__half, 128, 1>::kW : StagedPlan<__half, 64, 1>::kW; break;
        }
        for (int b = 0; b < 2; b++) {
            cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny, np};
            cuuint64_t strides[2] = {(cuuint64_t)h->pitch * h->elem, (cuuint64_t)h->p.ny * h->pitch * h->elem};
            cuuint32_t box[3] = {W, 1, np};
            cuuint32_t es[3] = {1, 1, 1};
            if (fn(&h->smap[b][k], dt, 3, h->fbase[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
    }
    // per-warp windows of the private kernel (PrivatePlan: the width depends
    // on the element size only)
    {
        cuuint32_t W = 0;
        switch (h->p.precision) {
            case LBM_FP64: W = PrivatePlan<double, 1, 1>::kW; break;
            case LBM_FP32:
            case LBM_FP32C: W = PrivatePlan<float, 1, 1>::kW; break;
            default: W = PrivatePlan<__half, 1, 1>::kW; break;
        }
        for (int b = 0; b < 2; b++) {
            cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny, np};
            cuuint64_t strides[2] = {(cuuint64_t)h->pitch * h->elem, (cuuint64_t)h->p.ny * h->pitch * h->elem};
            cuuint32_t box[3] = {W, 1, np};
            cuuint32_t es[3] = {1, 1, 1};
            if (fn(&h->pmap[b], dt, 3, h->fbase[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
        cuuint64_t dims[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny};
        cuuint64_t strides[1] = {(cuuint64_t)h->pitch * 2};
        cuuint32_t box[2] = {(cuuint32_t)PrivatePlan<float, 1, 1>::kLW, 1};
        cuuint32_t es[2] = {1, 1};
        if (fn(&h->plmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h->links, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int64_t>, Tuned> g_tune_cache;

int sms_of_device() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

int occupancy(const lbm_t* h, int var, int bx, int depth) {
    if (var == 2) return occupancy_staged(h->p.precision, bx, depth);
    if (var == 3) return occupancy_pipelined(h->p.precision, bx, depth);
    return occupancy_private(h->p.precision, bx, depth);
}

std::vector<Tuned> candidates(const lbm_t* h) {
    std::vector<Tuned> out;
    const int sms = sms_of_device();
    const int ny = h->p.ny;
    const int req = h->p.variant;
    // the persistent variant (5) keeps a simple-kernel configuration for the
    // single launches the library still makes
    if (req == 0 || req == 1 || req == 5) {
        for (int ctas_per_sm : {4, 8, 16}) {
            Tuned t;
            t.variant = 1;
            t.rpb = (int)std::max<int64_t>(4, std::min<int64_t>(ny, (int64_t)h->ncb * ny / (sms * ctas_per_sm)));
            out.push_back(t);
        }
    }
    for (int var : {2, 3, 4}) {
        if (!((req == 0 || req == var) && h->maps_ok)) continue;
        for (int bx : {64, 128}) {
            const int ncols = (h->p.nx + bx - 1) / bx;
            for (int depth : {1, 2}) {
                // strips for 1 to 4 full waves of the CTAs this configuration keeps resident
                const int per_sm = occupancy(h, var, bx, depth);
                if (per_sm < 1) continue;
                // staged: also strips at absolute rows, up to 5 (their clipped
                // strips are shorter, so more of them fit the same waves)
                for (int waves : {1, 2, 3, 4, 5}) {
                    for (int abs_rows : {0, 1}) {
                        if (abs_rows && var != 2) continue;
                        if (!abs_rows && waves > 4) continue;
                        Tuned t;
                        t.variant = var;
                        t.bx = bx;
                        t.depth = depth;
                        t.strip_abs = abs_rows;
                        const int resident = sms * per_sm;
                        t.strips = std::max(1, std::min(ny, waves * resident / std::max(1, ncols)));
                        out.push_back(t);
                    }
                }
            }
        }
    }
    std::vector<Tuned> u;
    for (auto& t : out) {
        bool dup = false;
        for (auto& v : u)
            dup |= v.variant == t.variant && v.depth == t.depth && v.rpb == t.rpb && v.strips == t.strips &&
                   v.bx == t.bx && v.strip_abs == t.strip_abs;
        if (!dup) u.push_back(t);
    }
    return u;
}

// GB300LBM_TUNE="staged,<cols per CTA>,<rows ahead: 1 or 2>,<strips>[,abs]"
// (",abs": strips at absolute rows; likewise "pipelined,..." and
// "private,..." without it) or "simple,<rows per strip>"
// pins the launch configuration (no timing); used to profile one
// configuration.
bool tune_from_env(lbm_t* h) {
    const char* e = getenv("GB300LBM_TUNE");
    if (!e || !*e) return false;
    Tuned t;
    int a = 0, b = 0, c = 0;
    int v = 0, n = 0;
    if (sscanf(e, "staged,%d,%d,%d%n", &a, &b, &c, &n) == 3) {
        v = 2;
        t.strip_abs = strcmp(e + n, ",abs") == 0;
    }
    else if (sscanf(e, "pipelined,%d,%d,%d", &a, &b, &c) == 3) v = 3;
    else if (sscanf(e, "private,%d,%d,%d", &a, &b, &c) == 3) v = 4;
    if (v && (a == 64 || a == 128) && (b == 1 || b == 2) && c >= 1 && h->maps_ok) {
        t.variant = v;
        t.bx = a;
        t.depth = b;
        t.strips = std::min(c, h->p.ny);
    } else if (sscanf(e, "simple,%d", &a) == 1 && a >= 1) {
        t.variant = 1;
        t.rpb = std::min(a, h->p.ny);
    } else {
        return false;
    }
    h->tune = t;
    return true;
}

int autotune(lbm_t* h) {
    if (tune_from_env(h)) return LBM_OK;
    auto key = std::make_tuple(h->p.nx, h->p.ny, h->p.precision, h->p.periodic_x, h->p.variant, h->fluid_nodes);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->tune = it->second;
            return LBM_OK;
        }
    }
    std::vector<Tuned> cand = candidates(h);
    if (cand.empty()) return fail(nullptr, LBM_ECUDA, "no step kernel available (tensor maps failed)");
    Tuned best = cand[0];
    if (cand.size() > 1) {
        cudaEvent_t e0, e1;
        CUDA_TRY(nullptr, cudaEventCreate(&e0));
        CUDA_TRY(nullptr, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        // candidates step from the current buffer into the other one, with
        // scratch accumulators: the stored state and the observables are untouched
        for (const Tuned& t : cand) {
            CUDA_TRY(nullptr, cudaMemsetAsync(h->tacc, 0, sizeof(ObsAccum), h->stream));
            CUDA_TRY(nullptr, cudaMemsetAsync(h->tobs, 0, sizeof(ObsState), h->stream));
            CUDA_TRY(nullptr, launch_step(h, h->cur, t, h->tacc, h->tobs, h->stream));
            // a candidate whose bounded waits gave up is not a candidate
            int tflag = 0;
            CUDA_TRY(nullptr, cudaMemcpyAsync(&tflag, &h->tobs->timeout_flag, sizeof(int), cudaMemcpyDeviceToHost,
                                              h->stream));
            CUDA_TRY(nullptr, cudaStreamSynchronize(h->stream));
            if (tflag) continue;
            CUDA_TRY(nullptr, cudaEventRecord(e0, h->stream));
            for (int k = 0; k < 3; k++) CUDA_TRY(nullptr, launch_step(h, h->cur, t, h->tacc, h->tobs, h->stream));
            CUDA_TRY(nullptr, cudaEventRecord(e1, h->stream));
            CUDA_TRY(nullptr, cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_TRY(nullptr, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    h->tune = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// misc host helpers
// ---------------------------------------------------------------------------
double to_double(const void* base, size_t k, int prec) {
    switch (prec) {
        case LBM_FP64: return ((const double*)base)[k];
        case LBM_FP32:
        case LBM_FP32C: return ((const float*)base)[k];
        case LBM_FP16S: return __half2float(((const __half*)base)[k]);
        default: return __bfloat162float(((const __nv_bfloat16*)base)[k]);
    }
}

void from_double(void* base, size_t k, int prec, double v) {
    switch (prec) {
        case LBM_FP64: ((double*)base)[k] = v; break;
        case LBM_FP32:
        case LBM_FP32C: ((float*)base)[k] = (float)v; break;
        case LBM_FP16S: ((__half*)base)[k] = __float2half_rn((float)v); break;
        default: ((__nv_bfloat16*)base)[k] = __float2bfloat16_rn((float)v); break;
    }
}

// FP32 lattice weights as the device uses them (1/36 one ulp low: the nine
// sum to exactly 1 in FP32)
float host_wf(int i) {
    if (i == 0) return 4.0f / 9.0f;
    if (i <= 4) return 1.0f / 9.0f;
    uint32_t bits = 0x3CE38E38u;
    float w;
    memcpy(&w, &bits, sizeof w);
    return w;
}

int validate(const lbm_params* p, const uint8_t* mask) {
    if (!p) return fail(nullptr, LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(nullptr, LBM_EINVAL, "nx, ny must be >= 1");
    if (elem_size(p->precision) == 0) return fail(nullptr, LBM_EINVAL, "unknown precision %d", p->precision);
    if (p->eq_order != 2 && p->eq_order != 3) return fail(nullptr, LBM_EINVAL, "eq_order must be 2 or 3");
    if (p->variant < 0 || p->variant > 5) return fail(nullptr, LBM_EINVAL, "variant must be 0, 1, 2, 3, 4 or 5");
    if (p->collision != 0 && p->collision != 1) return fail(nullptr, LBM_EINVAL, "collision must be 0 or 1");
    for (int a = 0; a < 2; a++)
        if (!(p->tau[a] > 0.5) || !std::isfinite(p->tau[a]))
            return fail(nullptr, LBM_EINVAL, "tau[%d] must be finite and exceed 1/2", a);
    if (!std::isfinite(p->G) || !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]) ||
        !std::isfinite(p->rho_wall[0]) || !std::isfinite(p->rho_wall[1]))
        return fail(nullptr, LBM_EINVAL, "G, g and rho_wall must be finite");
    Layout L;
    if (!layout_of(p, &L)) return fail(nullptr, LBM_EINVAL, "grid %d x %d too large", p->nx, p->ny);
    if (mask) {
        const int nx = p->nx, ny = p->ny;
        if (!p->periodic_x)
            for (int y = 0; y < ny; y++)
                if (!mask[(size_t)y * nx] || !mask[(size_t)y * nx + nx - 1])
                    return fail(nullptr, LBM_EINVAL, "x is not periodic but column 0 or nx-1 has fluid");
        if (!p->periodic_y)
            for (int x = 0; x < nx; x++)
                if (!mask[x] || !mask[(size_t)(ny - 1) * nx + x])
                    return fail(nullptr, LBM_EINVAL, "y is not periodic but row 0 or ny-1 has fluid");
    }
    return LBM_OK;
}

void fill_params(lbm_t* h) {
    StepParams& s = h->hprm;
    for (int a = 0; a < 2; a++) {
        s.nu[a] = (h->p.tau[a] - 0.5) / 3.0;
        s.rho_wall[a] = h->p.rho_wall[a];
        s.g[a] = h->p.g[a];
    }
    s.G = h->p.G;
    s.k3 = h->p.eq_order >= 3 ? 4.5 : 0.0;
    s.reg = h->p.collision == 1 ? 1.0 : 0.0;
}

void drop_graphs(lbm_t* h) {
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Capture kGraphSteps launches starting from buffer `src` on the private
// capture stream.
int build_graph(lbm_t* h, int src) {
    cudaGraph_t g = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    int s = src;
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; k++) {
        le = launch_step(h, s, h->tune, h->dacc, h->dobs, h->capture);
        s = 1 - s;
    }
    cudaError_t ce = cudaStreamEndCapture(h->capture, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, LBM_ECUDA, "graph capture failed: %s",
                    cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&h->graph[src], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(h, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    return LBM_OK;
}

}  // namespace

// Wait self-test: one thread waits, through the same bounded mbarrier wait
// the step kernels use, on a barrier that nothing ever arrives at, and
// records whether the wait gave up (it must).
__global__ void wait_selftest_kernel(int* out) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    out[0] = mbar_wait(&bar, 0u) ? 0 : 1;
}

namespace {

constexpr int64_t kPersistMaxFluid = int64_t(1) << 21;   // grids the persistent path is tried on
constexpr int kPersistChunk = 4096;                      // steps per cooperative launch


// Tiles of `rpb` rows for the persistent march, and a cooperative grid no
// larger than what is resident.
void set_persist_tiles(lbm_t* h, int rpb, int resident) {
    h->persist_rpb = std::max(1, std::min(rpb, h->p.ny));
    const int ntiles = h->ncb * ((h->p.ny + h->persist_rpb - 1) / h->persist_rpb);
    h->persist_ctas = std::min(ntiles, resident);
}

// Whether this handle steps with the persistent launch, and with which tile
// height.  With enough steps at hand, after one untimed launch of each path
// (the graph's upload and the lazy loading of the cooperative kernel's
// module are not part of a step), it times 32 steps through the captured
// graph (unless variant 5 forces the persistent launch) and 16 steps of the
// persistent launch for tiles of 1, 2, 4 and 8 rows, and keeps the fastest;
// every timed launch advances the simulation by an even number of steps (the
// marches give the same bits up to the order of a few sums).  Otherwise
// (variant 5 and fewer steps) it takes 4-row tiles, or enough rows for one
// wave of resident CTAs.  *left is reduced by the steps taken.
int decide_persist(lbm_t* h, int64_t* left) {
    int dev = 0, coop = 0, sms = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = persist_occupancy_of(h->p.precision);
    cudaGetLastError();
    const bool forced = h->p.variant == 5;
    if (!coop || occ < 1) {
        if (forced) return fail(h, LBM_ECUDA, "cooperative launches are not available");
        h->persist = -1;
        return LBM_OK;
    }
    const int resident = occ * sms;
    const int64_t rows = (int64_t)h->ncb * h->p.ny;
    const int rpb_wave = (int)std::max<int64_t>(4, (rows + resident - 1) / resident);
    constexpr int kCand[4] = {1, 2, 4, 8};
    constexpr int kTimed = 16;
    const int64_t need = (forced ? 0 : 2 * kGraphSteps) + 2 + 4 * kTimed;
    if (forced && *left < need) {
        set_persist_tiles(h, rpb_wave, resident);
        h->persist = 1;
        return LBM_OK;
    }
    if (!forced && !h->graph[h->cur]) {
        int rc = build_graph(h, h->cur);
        if (rc) return rc;
    }
    if (!forced) CUDA_TRY(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
    set_persist_tiles(h, kCand[0], resident);
    CUDA_TRY(h, launch_persist(h, 2));
    cudaEvent_t ev[6];
    for (auto& e : ev) CUDA_TRY(h, cudaEventCreate(&e));
    CUDA_TRY(h, cudaEventRecord(ev[0], h->stream));
    if (!forced) CUDA_TRY(h, cudaGraphLaunch(h->graph[h->cur], h->stream));   // 32 steps: the parity is unchanged
    CUDA_TRY(h, cudaEventRecord(ev[1], h->stream));
    for (int c = 0; c < 4; c++) {
        set_persist_tiles(h, kCand[c], resident);
        CUDA_TRY(h, launch_persist(h, kTimed));
        CUDA_TRY(h, cudaEventRecord(ev[2 + c], h->stream));
    }
    CUDA_TRY(h, cudaEventSynchronize(ev[5]));
    float t_graph = 0.f;
    CUDA_TRY(h, cudaEventElapsedTime(&t_graph, ev[0], ev[1]));
    float best = 0.f;
    int best_rpb = kCand[0];
    for (int c = 0; c < 4; c++) {
        float t = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&t, ev[1 + c], ev[2 + c]));
        if (c == 0 || t < best) {
            best = t;
            best_rpb = kCand[c];
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    *left -= need;
    set_persist_tiles(h, best_rpb, resident);
    h->persist = (forced || best / kTimed < t_graph / kGraphSteps) ? 1 : -1;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_workspace_size(const lbm_params* p, size_t* bytes) {
    if (!p || !bytes) return fail(nullptr, LBM_EINVAL, "NULL argument");
    Layout L;
    if (!layout_of(p, &L)) return fail(nullptr, LBM_EINVAL, "bad size or precision");
    *bytes = L.total;
    return LBM_OK;
}

int lbm_create(const uint8_t* mask, const double* rho_init, const lbm_params* p, lbm_t** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mask || !rho_init) return fail(nullptr, LBM_EINVAL, "mask and rho_init are required");
    int rc = validate(p, mask);
    if (rc) return rc;
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;

    // the fluid-node count, the fluid row range of every column block and
    // the check of the initial densities come from one device pass below
    Layout L;
    layout_of(p, &L);
    const std::vector<int2> rows(L.nrb, int2{ny, -1});

    lbm_t* h = new (std::nothrow) lbm_t();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    h->p = *p;
    h->stream = (cudaStream_t)p->cuda_stream;
    h->pitch = L.pitch;
    h->ncb = L.ncb;
    h->nrb = L.nrb;
    h->elem = elem_size(p->precision);
    h->buf_bytes = L.buf;

    if (p->workspace) {
        if (p->workspace_bytes < L.total || ((uintptr_t)p->workspace & 255)) {
            delete h;
            return fail(nullptr, LBM_ENOMEM, "workspace smaller than %zu bytes or not 256-byte aligned", L.total);
        }
        h->arena = p->workspace;
    } else {
        cudaError_t e = cudaMalloc(&h->arena, L.total);
        if (e != cudaSuccess) {
            delete h;
            return fail(nullptr, LBM_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
        }
        h->own_arena = true;
    }
    char* base = (char*)h->arena;
    size_t off = 0;
    h->fbase[0] = base + off;
    off += L.buf;
    h->fbase[1] = base + off;
    off += L.buf;
    h->links = (uint16_t*)(base + off);
    off += L.links;
    h->rows = (int2*)(base + off);
    off += L.rows;
    h->dprm = (StepParams*)(base + off);
    off += L.prm;
    h->dacc = (ObsAccum*)(base + off);
    off += L.acc;
    h->tacc = (ObsAccum*)(base + off);
    off += L.acc;
    h->dobs = (ObsState*)(base + off);
    off += L.obs;
    h->tobs = (ObsState*)(base + off);

    fill_params(h);

    auto bail = [&](int code) {
        std::string msg = g_create_err;
        lbm_destroy(h);
        g_create_err = msg;
        return code;
    };
#define CREATE_TRY(call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            fail(nullptr, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));             \
            return bail(LBM_ECUDA);                                                               \
        }                                                                                         \
    } while (0)
    CREATE_TRY(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking));
    // stage rho_init (FP64) and the mask in buffer B, build links, init A
    const size_t rho_bytes = n * 2 * sizeof(double);
    char* stage = h->fbase[1];
    double* d_rho = (double*)stage;
    uint8_t* d_mask = (uint8_t*)(stage + align256(rho_bytes));
    CREATE_TRY(cudaMemcpyAsync(d_rho, rho_init, rho_bytes, cudaMemcpyHostToDevice, h->stream));
    CREATE_TRY(cudaMemcpyAsync(d_mask, mask, n, cudaMemcpyHostToDevice, h->stream));
    CREATE_TRY(cudaMemcpyAsync(h->rows, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    // scan counters after the staged mask (the staging area is free until B is filled)
    unsigned long long* d_nfluid = (unsigned long long*)(stage + align256(rho_bytes) + align256(n));
    int* d_bad = (int*)(d_nfluid + 1);
    CREATE_TRY(cudaMemsetAsync(d_nfluid, 0, 16, h->stream));
    scan_kernel<<<dim3((nx + 255) / 256, ny), 256, 0, h->stream>>>(d_mask, d_rho, nx, ny, h->rows, d_nfluid, d_bad);
    CREATE_TRY(cudaGetLastError());
    struct {
        unsigned long long nfluid;
        int bad, pad;
    } scan{};
    CREATE_TRY(cudaMemcpyAsync(&scan, d_nfluid, 16, cudaMemcpyDeviceToHost, h->stream));
    CREATE_TRY(cudaStreamSynchronize(h->stream));
    if (scan.bad) {
        fail(nullptr, LBM_EINVAL, "rho_init must be finite, >= 0, with positive total at fluid nodes");
        return bail(LBM_EINVAL);
    }
    h->fluid_nodes = (int64_t)scan.nfluid;
    CREATE_TRY(cudaMemsetAsync(h->dacc, 0, 2 * L.acc, h->stream));
    CREATE_TRY(cudaMemsetAsync(h->dobs, 0, 2 * L.obs, h->stream));
    CREATE_TRY(cudaMemcpyAsync(h->dprm, &h->hprm, sizeof(StepParams), cudaMemcpyHostToDevice, h->stream));
    dim3 blk(256), grd((h->pitch + 255) / 256, ny);
    links_kernel<<<grd, blk, 0, h->stream>>>(d_mask, h->links, nx, ny, h->pitch, p->periodic_x);
    const int px = p->periodic_x;
    switch (p->precision) {
        case LBM_FP64: init_kernel<double><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (double*)h->fbase[0], nx, ny, h->pitch, px); break;
        case LBM_FP32: init_kernel<float><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (float*)h->fbase[0], nx, ny, h->pitch, px); break;
        case LBM_FP32C: init_kernel<f32c><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (f32c*)h->fbase[0], nx, ny, h->pitch, px); break;
        case LBM_FP16S: init_kernel<__half><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (__half*)h->fbase[0], nx, ny, h->pitch, px); break;
        default: init_kernel<__nv_bfloat16><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (__nv_bfloat16*)h->fbase[0], nx, ny, h->pitch, px); break;
    }
    CREATE_TRY(cudaGetLastError());
    // B holds the same zeros at solid nodes, padding and unused ghosts as A
    CREATE_TRY(cudaMemcpyAsync(h->fbase[1], h->fbase[0], L.buf, cudaMemcpyDeviceToDevice, h->stream));
    CREATE_TRY(cudaStreamSynchronize(h->stream));
#undef CREATE_TRY
    h->maps_ok = make_maps(h);
    h->cur = 0;
    if (p->variant >= 2 && !h->maps_ok) {
        fail(nullptr, LBM_ECUDA, "tensor-map encoding failed: the staged kernel is unavailable");
        return bail(LBM_ECUDA);
    }
    rc = autotune(h);
    if (rc) return bail(rc);
    *out = h;
    return LBM_OK;
}

int lbm_step(lbm_t* h, int64_t nsteps) {
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
    int64_t left = nsteps;
    // small grids: many steps per cooperative launch, when that beats one
    // graph node per step (decided once per handle by timing both: 130
    // steps in all)
    if (h->persist == 0 && ((h->p.variant == 0 && left >= 160 && h->fluid_nodes <= kPersistMaxFluid) ||
                            h->p.variant == 5)) {
        int rc = decide_persist(h, &left);
        if (rc) return rc;
    }
    if (h->persist == 1) {
        while (left > 0) {
            const int n = (int)std::min<int64_t>(left, kPersistChunk);
            CUDA_TRY(h, launch_persist(h, n));
            if (n & 1) h->cur = 1 - h->cur;
            left -= n;
        }
        return LBM_OK;
    }
    if (left >= kGraphSteps) {
        if (!h->graph[h->cur]) {
            int rc = build_graph(h, h->cur);
            if (rc) return rc;
        }
        while (left >= kGraphSteps) {
            CUDA_TRY(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
            left -= kGraphSteps;   // an even number of steps: the parity is unchanged
        }
    }
    for (; left > 0; left--) {
        CUDA_TRY(h, launch_step(h, h->cur, h->tune, h->dacc, h->dobs, h->stream));
        h->cur = 1 - h->cur;
    }
    return LBM_OK;
}

int lbm_observables(lbm_t* h, lbm_obs* out) {
    if (!h || !out) return fail(h, LBM_EINVAL, "NULL argument");
    ObsState s;
    CUDA_TRY(h, cudaMemcpyAsync(&s, h->dobs, sizeof s, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    out->mass[0] = s.mass[0];
    out->mass[1] = s.mass[1];
    out->oil_mom_x = s.px;
    out->oil_disp_x = s.disp;
    out->max_u = s.umax;
    out->step = s.step;
    out->nan_flag = s.nan_flag;
    out->timeout_flag = s.timeout_flag;
    if (s.timeout_flag) return fail(h, LBM_ETIMEOUT, "a bounded device wait gave up");
    if (s.nan_flag) return fail(h, LBM_EUNSTABLE, "a fluid node reached a NaN or negative density");
    return LBM_OK;
}

int lbm_get_fields(lbm_t* h, double* rho, double* u, double* pr) {
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    const int nx = h->p.nx, ny = h->p.ny;
    const size_t n = (size_t)nx * ny;
    // fields of a window of rows are written to the free buffer, 5 doubles a node
    const int max_rows = (int)std::min<size_t>(ny, h->buf_bytes / (5 * sizeof(double) * nx));
    if (max_rows < 1) return fail(h, LBM_EINVAL, "grid row too long for the staging buffer");
    double* stage = (double*)h->fbase[1 - h->cur];
    // the window's five planes (rho^o, rho^w, u_x, u_y, p) go straight into
    // the caller's arrays: a single window when the grid fits the buffer,
    // then rho and u are one copy each (their two planes are adjacent)
    for (int y0 = 0; y0 < ny; y0 += max_rows) {
        const int y1 = std::min(ny, y0 + max_rows);
        const size_t cnt = (size_t)nx * (y1 - y0);
        const size_t o = (size_t)y0 * nx;
        const size_t b = cnt * sizeof(double);
        CUDA_TRY(h, launch_fields(h, stage, y0, y1));
        double* dst[5] = {rho ? rho + o : nullptr, rho ? rho + n + o : nullptr, u ? u + o : nullptr,
                          u ? u + n + o : nullptr, pr ? pr + o : nullptr};
        for (int k = 0; k < 5; k++) {
            if (!dst[k]) continue;
            if (cnt == n && k % 2 == 0 && k < 4 && dst[k + 1]) {
                CUDA_TRY(h, cudaMemcpyAsync(dst[k], stage + k * cnt, 2 * b, cudaMemcpyDeviceToHost, h->stream));
                k++;
                continue;
            }
            CUDA_TRY(h, cudaMemcpyAsync(dst[k], stage + k * cnt, b, cudaMemcpyDeviceToHost, h->stream));
        }
        // the next window overwrites the staging planes
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

int lbm_set_body_force(lbm_t* h, double gx, double gy) {
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (!std::isfinite(gx) || !std::isfinite(gy)) return fail(h, LBM_EINVAL, "g must be finite");
    h->p.g[0] = gx;
    h->p.g[1] = gy;
    h->hprm.g[0] = gx;
    h->hprm.g[1] = gy;
    CUDA_TRY(h, cudaMemcpyAsync(h->dprm, &h->hprm, sizeof(StepParams), cudaMemcpyHostToDevice, h->stream));
    // the host copy must stay valid until the copy ran
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_save(lbm_t* h, double* f) {
    if (!h || !f) return fail(h, LBM_EINVAL, "NULL argument");
    const int nx = h->p.nx, ny = h->p.ny, pitch = h->pitch, prec = h->p.precision;
    const size_t plane = (size_t)ny * pitch;
    const bool shifted = planes_of(prec) == 20;
    std::vector<char> raw(h->buf_bytes);
    std::vector<uint16_t> lk(plane);
    CUDA_TRY(h, cudaMemcpyAsync(raw.data(), h->fbase[h->cur], h->buf_bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(lk.data(), h->links, lk.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            const size_t node = (size_t)y * pitch + kGhost + x;
            const bool solid = lk[node] & (1u << kSolidBit);
            for (int a = 0; a < 2; a++) {
                const float rh = shifted ? (float)to_double(raw.data(), (18 + a) * plane + node, prec) : 0.f;
                for (int i = 0; i < 9; i++) {
                    const double s = to_double(raw.data(), (a * 9 + i) * plane + node, prec);
                    // the device decode: s + w_i rhohat as one fused multiply-add in FP32
                    const double v = shifted ? (double)std::fma(host_wf(i), rh, (float)s) : s;
                    f[((size_t)(a * 9 + i) * ny + y) * nx + x] = solid ? 0.0 : v;
                }
            }
        }
    return LBM_OK;
}

int lbm_load(lbm_t* h, const double* f) {
    if (!h || !f) return fail(h, LBM_EINVAL, "NULL argument");
    const int nx = h->p.nx, ny = h->p.ny, pitch = h->pitch, prec = h->p.precision;
    const size_t plane = (size_t)ny * pitch;
    const bool shifted = planes_of(prec) == 20;
    std::vector<uint16_t> lk(plane);
    CUDA_TRY(h, cudaMemcpyAsync(lk.data(), h->links, lk.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    std::vector<char> raw(h->buf_bytes, 0);
    for (int y = 0; y < ny; y++)
        for (int sc = 0; sc < pitch; sc++) {
            // storage column sc holds logical column x, or a periodic image
            int x = sc - kGhost;
            if (x < 0 || x >= nx) {
                if (!h->p.periodic_x || x < -kGhost || x >= nx + kGhost) continue;
                x = ((x % nx) + nx) % nx;
            }
            if (lk[(size_t)y * pitch + kGhost + x] & (1u << kSolidBit)) continue;
            const size_t node = (size_t)y * pitch + sc;
            for (int a = 0; a < 2; a++) {
                float rh = 0.f;
                if (shifted) {
                    double r = 0.0;
                    for (int i = 0; i < 9; i++) r += f[((size_t)(a * 9 + i) * ny + y) * nx + x];
                    from_double(raw.data(), (18 + a) * plane + node, prec, r);
                    rh = (float)to_double(raw.data(), (18 + a) * plane + node, prec);
                }
                for (int i = 0; i < 9; i++) {
                    const double v = f[((size_t)(a * 9 + i) * ny + y) * nx + x];
                    from_double(raw.data(), (a * 9 + i) * plane + node, prec,
                                shifted ? (double)std::fma(-host_wf(i), rh, (float)v) : v);
                }
            }
        }
    CUDA_TRY(h, cudaMemcpyAsync(h->fbase[h->cur], raw.data(), h->buf_bytes, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->dacc, 0, sizeof(ObsAccum), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->dobs, 0, sizeof(ObsState), h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_kernel_info(const lbm_t* h, int32_t info[5]) {
    if (!h || !info) return fail(nullptr, LBM_EINVAL, "NULL argument");
    if (h->persist == 1) {
        info[0] = 5;
        info[1] = 0;
        info[2] = h->persist_rpb;
        info[3] = h->persist_ctas;
        info[4] = 0;
        return LBM_OK;
    }
    info[0] = h->tune.variant;
    info[1] = h->tune.variant >= 2 ? h->tune.depth : 0;
    info[2] = h->tune.variant == 1 ? h->tune.rpb : h->tune.bx;
    info[3] = h->tune.variant >= 2 ? h->tune.strips : 0;
    info[4] = h->tune.variant == 2 ? h->tune.strip_abs : 0;
    return LBM_OK;
}

void lbm_destroy(lbm_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    drop_graphs(h);
    if (h->capture) cudaStreamDestroy(h->capture);
    if (h->own_arena && h->arena) cudaFree(h->arena);
    delete h;
}

const char* lbm_last_error(const lbm_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int lbm_wait_selftest(void* cuda_stream, double* seconds) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int* d = nullptr;
    CUDA_TRY(nullptr, cudaMalloc(&d, sizeof(int)));
    int flag = -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    wait_selftest_kernel<<<1, 1, 0, st>>>(d);
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "wait self-test: %s", cudaGetErrorString(e));
    if (seconds) *seconds = ms * 1e-3;
    if (flag == 1) return fail(nullptr, LBM_ETIMEOUT, "wait self-test: the bounded wait gave up (as it should)");
    return fail(nullptr, LBM_ECUDA, "wait self-test: a wait on a barrier nothing arrives at completed");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free step
//
// For callers that cannot allocate device memory: code running while a CUDA
// graph is being captured (cudaMalloc is not allowed there), real-time loops
// that must not allocate, or plug-ins whose device memory is owned by a host
// framework's allocator.  The caller passes device inputs and outputs; the
// step's scratch (link words, parameters, reduction accumulators) lives in
// one fixed device array of this file.
// ---------------------------------------------------------------------------
namespace {

// Largest lattice the allocation-free entry point accepts (nx * ny).
constexpr int kNoAllocMaxNodes = 1 << 21;
// Scratch layout: [StepParams | ObsAccum | ObsState | link words (uint16)].
constexpr size_t kNoAllocHead = 1024;
constexpr size_t kNoAllocBytes = kNoAllocHead + sizeof(uint16_t) * (size_t)kNoAllocMaxNodes;

// The scratch of lbm_step_noalloc: a fixed device array that every GPU which
// loads the library holds until the process exits (4 MiB + 1 KiB).  In host
// code this name is only a host-side stand-in; its device address is taken
// with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

static_assert(sizeof(StepParams) + sizeof(ObsAccum) + sizeof(ObsState) <= kNoAllocHead, "scratch head");

// Link words of a dense [ny][nx] lattice (no ghost columns), plus the
// parameters and cleared accumulators, into the scratch.  Rows are visited
// grid-stride in y, so any admitted shape launches with gridDim.y <= 65535.
__global__ void noalloc_prepare_kernel(const uint8_t* __restrict__ mask, unsigned char* __restrict__ scratch, int nx,
                                       int ny, StepParams prm) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x == 0 && blockIdx.y == 0) {
        *(StepParams*)scratch = prm;
        ObsAccum* acc = (ObsAccum*)(scratch + sizeof(StepParams));
        ObsState* obs = (ObsState*)(scratch + sizeof(StepParams) + sizeof(ObsAccum));
        memset(acc, 0, sizeof(ObsAccum));
        memset(obs, 0, sizeof(ObsState));
    }
    if (x >= nx) return;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        unsigned w = mask[y * nx + x] ? (1u << kSolidBit) : 0u;
        for (int i = 1; i < 9; i++) {
            int sx = x - d2q9_cx(i), sy = y - d2q9_cy(i);
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            if (mask[sy * nx + sx]) w |= 1u << i;
        }
        ((uint16_t*)(scratch + kNoAllocHead))[y * nx + x] = uint16_t(w);
    }
}

__global__ void noalloc_obs_kernel(const unsigned char* __restrict__ scratch, lbm_obs* __restrict__ out) {
    const ObsState* s = (const ObsState*)(scratch + sizeof(StepParams) + sizeof(ObsAccum));
    out->mass[0] = s->mass[0];
    out->mass[1] = s->mass[1];
    out->oil_mom_x = s->px;
    out->oil_disp_x = s->disp;
    out->max_u = s->umax;
    out->step = s->step;
    out->nan_flag = s->nan_flag;
    out->timeout_flag = s->timeout_flag;
}

}  // namespace

extern "C" int lbm_step_noalloc(const uint8_t* mask, const float* f_in, float* f_out, lbm_obs* obs,
                                const lbm_params* p) {
    if (!mask || !f_in || !f_out || !p) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: NULL argument");
    if (p->precision != LBM_FP32) return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: precision must be LBM_FP32");
    if (p->nx < 1 || p->ny < 1 || (int64_t)p->nx * p->ny > kNoAllocMaxNodes)
        return fail(nullptr, LBM_EINVAL, "lbm_step_noalloc: nx * ny must be in [1, %d] (got %d x %d)",
                    kNoAllocMaxNodes, p->nx, p->ny);
    if (p->eq_order != 2 && p->eq_order != 3) return fail(nullptr, LBM_EINVAL, "eq_order must be 2 or 3");
    if (p->collision != 0 && p->collision != 1) return fail(nullptr, LBM_EINVAL, "collision must be 0 or 1");
    for (int a = 0; a < 2; a++)
        if (!(p->tau[a] > 0.5) || !std::isfinite(p->tau[a]))
            return fail(nullptr, LBM_EINVAL, "tau[%d] must be finite and exceed 1/2", a);
    if (!std::isfinite(p->G) || !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]) ||
        !std::isfinite(p->rho_wall[0]) || !std::isfinite(p->rho_wall[1]))
        return fail(nullptr, LBM_EINVAL, "G, g and rho_wall must be finite");
    int dev = 0;
    CUDA_TRY(nullptr, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, LBM_EINVAL, "device %d out of range", dev);
    unsigned char* scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(nullptr, LBM_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (unsigned char*)ptr;
        }
        scratch = g_noalloc_ptr[dev];
    }
    const int nx = p->nx, ny = p->ny;
    cudaStream_t st = (cudaStream_t)p->cuda_stream;
    StepParams prm{};
    for (int a = 0; a < 2; a++) {
        prm.nu[a] = (p->tau[a] - 0.5) / 3.0;
        prm.rho_wall[a] = p->rho_wall[a];
        prm.g[a] = p->g[a];
    }
    prm.G = p->G;
    prm.k3 = p->eq_order >= 3 ? 4.5 : 0.0;
    prm.reg = p->collision == 1 ? 1.0 : 0.0;
    noalloc_prepare_kernel<<<dim3((nx + 127) / 128, std::min(ny, 65535)), 128, 0, st>>>(mask, scratch, nx, ny, prm);
    CUDA_TRY(nullptr, cudaGetLastError());
    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.pitch = nx;            // dense rows, no ghost columns
    g.periodic_x = 0;        // no ghost images to write (pulls still wrap)
    // rows per CTA strip: 32 (fewer on short grids), more when ny / 32
    // would exceed the 65535 limit of gridDim.y
    g.rows_per_block = std::max(std::max(4, std::min(ny, 32)), (ny + 65534) / 65535);
    g.row_begin = 0;
    g.row_end = ny;
    g.strips = 1;
    dim3 grid((nx + kBX - 1) / kBX, (ny + g.rows_per_block - 1) / g.rows_per_block);
    step_simple_kernel<float, kBX, false><<<grid, kBX, 0, st>>>(
        f_in, f_out, (const uint16_t*)(scratch + kNoAllocHead), (const StepParams*)scratch,
        (ObsAccum*)(scratch + sizeof(StepParams)), (ObsState*)(scratch + sizeof(StepParams) + sizeof(ObsAccum)),
        nullptr, g);
    CUDA_TRY(nullptr, cudaGetLastError());
    if (obs) {
        noalloc_obs_kernel<<<1, 1, 0, st>>>(scratch, obs);
        CUDA_TRY(nullptr, cudaGetLastError());
    }
    return LBM_OK;
}
