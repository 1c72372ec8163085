// Batched instances and the device-side critical-pressure bisection.
//
// Many independent channels of uneven size step together: every instance's
// grid is cut into tiles (128 columns x a strip of rows) and ONE launch per
// step covers the concatenated tile list of all still-active instances; the
// kernel boundary is the step barrier, and runs of steps are replayed from a
// captured CUDA graph.  Each CTA reduces its observables into its own
// instance's FP64 accumulators, and the last CTA of an instance integrates
// that instance's oil displacement.
//
// The bisection of Section 3.4's critical body force (the slug starts to
// move once g exceeds g_crit) runs on the device in FP64: after each probe
// window of t_obs steps a one-thread-per-instance kernel classifies the slug
// as moving (|oil displacement over the window| > the instance's threshold)
// or static, updates the instance's bracket [g_lo, g_hi] (first checking
// that g_hi moves and g_lo does not, doubling / halving the bracket when
// either check fails), and sets the next probe at the geometric midpoint.
// Every probe restarts from the state equilibrated at g = 0 (a device
// snapshot), so probes are independent.  The host only launches graphs and
// reads one counter per window.
//
// Layout: three regions (A, B, snapshot) of the arena, each holding every
// instance's population buffer at the same offset; link words in a fourth
// region.  Buffer layout per instance as in lbm_common.cuh.
//
// Step kernels: FP32 and the 16-bit formats run the staged march of the
// single-grid library (lbm_step_tma.cuh: rows moved to shared memory by the
// Tensor Memory Accelerator) over a list of (instance, 128-column block,
// strip of rows) tiles that holds only the rows with fluid; each instance has
// its own tensor maps in device memory.  FP64 (arithmetic-bound) runs the
// register-pull march over 128 x ~32 tiles.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_setup.cuh"
#include "lbm_step.cuh"
#include "lbm_step_tma.cuh"

using namespace gb300lbm;

namespace {

constexpr int kTileX = 128;
constexpr int kBatchGraphSteps = 16;   // even: the parity is kept across a replay

enum : int { kCheckHi = 0, kCheckLo = 1, kBisect = 2, kDone = 3 };

// One tile of the staged batch kernel: rows [y0, y1) of the 128 columns
// starting at x0 of instance inst, marched in direction dir.
struct BatchTile {
    int inst, x0, y0, y1, dir, pad[3];
};

// Staged tiles of a whole batch for one strip height R.
struct TileSet {
    int R = 0;
    std::vector<BatchTile> tiles;
    std::vector<int> t0, nt;      // first tile and tile count of every instance
};

// Per-instance device record.
struct BatchInst {
    int nx, ny, pitch, periodic_x;
    int ncb, rpb, strips;         // register-pull tiles: ncb column blocks x strips of rpb rows
    int tile0, ntiles;            // first tile and tile count (of the kernel in use)
    int active;                   // steps run only for active instances
    long long off;                // element offset of the instance buffer in each region
    long long loff;               // element offset of its link words
    StepParams prm;
    ObsAccum acc;
    ObsState obs;
    // bisection (FP64)
    double g_lo, g_hi, g_probe, disp_thr;
    int state, probes, status, pad;
};

thread_local std::string g_batch_err;

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

int planes_for(int prec) { return (prec == LBM_FP16S || prec == LBM_BF16S) ? 20 : 18; }

size_t esize(int prec) {
    switch (prec) {
        case LBM_FP64: return 8;
        case LBM_FP32:
        case LBM_FP32C: return 4;
        case LBM_FP16S:
        case LBM_BF16S: return 2;
        default: return 0;
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kTileX) batch_step_kernel(BatchInst* __restrict__ inst,
                                                            const int* __restrict__ tile_inst, S* __restrict__ fa,
                                                            S* __restrict__ fb, const uint16_t* __restrict__ links,
                                                            int parity) {
    using R = typename Codec<S>::R;
    __shared__ pair_t<R> s_rho[4][kTileX + 2];
    const int ti = blockIdx.x;
    const int i = tile_inst[ti];
    BatchInst* I = inst + i;
    if (!I->active) return;                          // uniform over the CTA
    const int nx = I->nx, ny = I->ny, pitch = I->pitch;
    const int local = ti - I->tile0;
    const int cb = local % I->ncb, st = local / I->ncb;
    const int x0 = cb * kTileX;
    const int y0 = st * I->rpb;
    const int y1 = min(y0 + I->rpb, ny);
    const S* fin = (parity ? fb : fa) + I->off + kGhost;
    S* fout = (parity ? fa : fb) + I->off + kGhost;
    NodeParams<R> P;
    P.load(&I->prm);
    ObsLocal<R> ob;
    march_simple<S, kTileX, false>(fin, fout, links + I->loff + kGhost, P, nullptr, nx, ny, pitch, I->periodic_x,
                                   x0, y0, y1, 0, 0, ob, s_rho);
    reduce_observables<R, kTileX>(ob, &I->acc, &I->obs, false, (unsigned)I->ntiles);
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
    // the maps were written by a copy from the host before the launch; make
    // them visible to the tensor-map proxy before the first copy uses them
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}

// Staged step of the batch: one CTA per tile.  maps holds three tensor maps
// per instance (populations of region A, of region B, link words).
template <typename S>
__global__ void __launch_bounds__(kTileX, sizeof(S) == 8 ? 4 : 5)
    batch_staged_kernel(BatchInst* __restrict__ inst, const BatchTile* __restrict__ tiles, const CUtensorMap* maps,
                        S* __restrict__ fa, S* __restrict__ fb, int parity) {
    using R = typename Codec<S>::R;
    const BatchTile tl = tiles[blockIdx.x];
    BatchInst* I = inst + tl.inst;
    if (!I->active) return;                          // uniform over the CTA
    const CUtensorMap* m = maps + 3 * tl.inst;
    if (threadIdx.x == 0) {
        tensormap_acquire(m + parity);
        tensormap_acquire(m + 2);
    }
    S* fout = (parity ? fa : fb) + I->off + kGhost;
    ObsLocal<R> ob;
    // the instance's collision, uniform over the CTA: one march without the
    // other collision's branch for each
    const bool timed_out =
        I->prm.reg != 0.0
            ? staged_march<S, kTileX, 1, 1>(m + parity, m + 2, fout, &I->prm, I->nx, I->ny, I->pitch, I->periodic_x,
                                            tl.x0, tl.y0, tl.y1, tl.dir, ob)
            : staged_march<S, kTileX, 1, 0>(m + parity, m + 2, fout, &I->prm, I->nx, I->ny, I->pitch, I->periodic_x,
                                            tl.x0, tl.y0, tl.y1, tl.dir, ob);
    reduce_observables<R, kTileX>(ob, &I->acc, &I->obs, timed_out, (unsigned)I->ntiles);
}

// Start of a probe window: probe value by state, reset the window's
// displacement.  One thread per instance.
__global__ void probe_begin_kernel(BatchInst* __restrict__ inst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    BatchInst* I = inst + i;
    if (!I->active) return;
    double g;
    if (I->state == kCheckHi) g = I->g_hi;
    else if (I->state == kCheckLo) g = I->g_lo;
    else g = sqrt(I->g_lo * I->g_hi);
    I->g_probe = g;
    I->prm.g[0] = g;
    I->obs.disp = 0.0;
}

// End of a probe window: classify, update the bracket, count the instances
// still active.
__global__ void probe_decide_kernel(BatchInst* __restrict__ inst, int n, double rel_bracket, int max_probes,
                                    int* __restrict__ n_active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    BatchInst* I = inst + i;
    if (!I->active) return;
    I->probes += 1;
    if (I->obs.nan_flag || I->obs.timeout_flag) {     // unstable, or a bounded wait gave up
        I->status = I->obs.nan_flag ? 2 : 3;
        I->state = kDone;
        I->active = 0;
        return;
    }
    const bool moving = fabs(I->obs.disp) > I->disp_thr;
    const double g = I->g_probe;
    switch (I->state) {
        case kCheckHi:
            if (moving) I->state = kCheckLo;
            else {
                I->g_lo = I->g_hi;                    // g_hi was static: expand upwards
                I->g_hi = 2.0 * I->g_hi;
            }
            break;
        case kCheckLo:
            if (!moving) I->state = kBisect;
            else {
                I->g_hi = I->g_lo;                    // g_lo moved: expand downwards
                I->g_lo = 0.5 * I->g_lo;
            }
            break;
        default:
            if (moving) I->g_hi = g;
            else I->g_lo = g;
            break;
    }
    if (I->state == kBisect && (I->g_hi - I->g_lo) <= rel_bracket * I->g_hi) {
        I->state = kDone;
        I->status = 0;
        I->active = 0;
    } else if (I->probes >= max_probes) {
        I->state = kDone;
        I->status = 1;
        I->active = 0;
    } else {
        atomicAdd(n_active, 1);
    }
}

template <typename S>
cudaError_t launch_batch_step(S* fa, S* fb, BatchInst* inst, const int* tiles, const uint16_t* links, int ntiles,
                              int parity, cudaStream_t st) {
    batch_step_kernel<S><<<ntiles, kTileX, 0, st>>>(inst, tiles, fa, fb, links, parity);
    return cudaGetLastError();
}

// Shared-memory limit of the staged batch kernel, set once per format (at
// create time, outside any stream capture).
template <typename S>
cudaError_t staged_attr() {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(batch_staged_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    StagedPlan<S, kTileX, 1>::kBytes);
    });
    return attr;
}

cudaError_t staged_attr_for(int prec) {
    if (prec == LBM_FP32) return staged_attr<float>();
    if (prec == LBM_FP32C) return staged_attr<f32c>();
    if (prec == LBM_FP16S) return staged_attr<__half>();
    return staged_attr<__nv_bfloat16>();
}

template <typename S>
cudaError_t launch_batch_staged(S* fa, S* fb, BatchInst* inst, const BatchTile* tiles, const CUtensorMap* maps,
                                int ntiles, int parity, cudaStream_t st) {
    batch_staged_kernel<S><<<ntiles, kTileX, StagedPlan<S, kTileX, 1>::kBytes, st>>>(inst, tiles, maps, fa, fb,
                                                                                     parity);
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 batch_encode_fn() {
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

// Window width (columns) of the staged march for a storage format.
int staged_window(int prec) {
    switch (prec) {
        case LBM_FP32:
        case LBM_FP32C: return StagedPlan<float, kTileX, 1>::kW;
        default: return StagedPlan<__half, kTileX, 1>::kW;
    }
}

// The three tensor maps of instance I (populations in regions A and B, link
// words); false if the driver refuses one.
bool encode_instance_maps(CUtensorMap* out, const BatchInst& I, int prec, size_t es, int np, char* fa, char* fb,
                          uint16_t* links) {
    auto fn = batch_encode_fn();
    if (!fn) return false;
    const CUtensorMapDataType dt = (prec == LBM_FP32 || prec == LBM_FP32C) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : prec == LBM_FP16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    char* base[2] = {fa + I.off * es, fb + I.off * es};
    for (int r = 0; r < 2; r++) {
        cuuint64_t dims[3] = {(cuuint64_t)I.pitch, (cuuint64_t)I.ny, (cuuint64_t)np};
        cuuint64_t strides[2] = {(cuuint64_t)I.pitch * es, (cuuint64_t)I.ny * I.pitch * es};
        cuuint32_t box[3] = {(cuuint32_t)staged_window(prec), 1, (cuuint32_t)np};
        cuuint32_t el[3] = {1, 1, 1};
        if (fn(&out[r], dt, 3, base[r], dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    cuuint64_t dims[2] = {(cuuint64_t)I.pitch, (cuuint64_t)I.ny};
    cuuint64_t strides[1] = {(cuuint64_t)I.pitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)StagedPlan<float, kTileX, 1>::kLW, 1};
    cuuint32_t el[2] = {1, 1};
    return fn(&out[2], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, links + I.loff, dims, strides, box, el,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// First and last row with fluid in every 128-column block of a mask (lo =
// ny, hi = -1 for a block without fluid).
void block_rows(const uint8_t* mask, int nx, int ny, std::vector<int>& lo, std::vector<int>& hi) {
    const int ncb = (nx + kTileX - 1) / kTileX;
    lo.assign(ncb, ny);
    hi.assign(ncb, -1);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
            if (!mask[(size_t)y * nx + x]) {
                const int cb = x / kTileX;
                lo[cb] = std::min(lo[cb], y);
                hi[cb] = std::max(hi[cb], y);
            }
}

// Staged tiles of one instance: for every 128-column block the rows with
// fluid, cut into strips at the same absolute rows [s R, (s + 1) R) in every
// block (neighbouring blocks, adjacent in launch order, then share their
// window columns through L2); odd strips march upwards.  An instance with no
// fluid still gets one empty tile, so that its observables are reduced.
void staged_tiles(const std::vector<int>& lo, const std::vector<int>& hi, int ny, int inst, int R,
                  std::vector<BatchTile>& out) {
    const int ncb = (int)lo.size();
    const size_t before = out.size();
    for (int s = 0; s * R < ny; s++)
        for (int cb = 0; cb < ncb; cb++) {
            const int y0 = std::max(lo[cb], s * R), y1 = std::min(hi[cb] + 1, (s + 1) * R);
            if (y0 < y1) out.push_back(BatchTile{inst, cb * kTileX, y0, y1, (s & 1) ? -1 : 1, {0, 0, 0}});
        }
    if (out.size() == before) out.push_back(BatchTile{inst, 0, 0, 0, 1, {0, 0, 0}});
}

}  // namespace

struct lbm_batch_t {
    int n = 0;
    int prec = 0;
    size_t es = 0;
    size_t region_elems = 0;      // elements of one region (all instances)
    void* arena = nullptr;
    char* fa = nullptr;
    char* fb = nullptr;
    char* snap = nullptr;
    uint16_t* links = nullptr;
    BatchInst* dinst = nullptr;
    int* dtiles = nullptr;        // register-pull kernel: instance of each tile
    BatchTile* dstiles = nullptr; // staged kernel: tiles
    CUtensorMap* dmaps = nullptr; // staged kernel: three maps per instance
    bool staged = false;
    int strip_rows = 0;           // staged kernel: rows per strip
    int* dcount = nullptr;
    int* hcount = nullptr;        // pinned
    int ntiles = 0;
    int parity = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<BatchInst> hinst;
    std::string err;
};

namespace {

int batch_fail(lbm_batch_t* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_err = buf;
    return code;
}

#define BTRY(b, call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return batch_fail((b), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

cudaError_t step_once(lbm_batch_t* b, int parity, cudaStream_t st) {
    if (b->staged) {
        if (b->prec == LBM_FP32)
            return launch_batch_staged<float>((float*)b->fa, (float*)b->fb, b->dinst, b->dstiles, b->dmaps,
                                              b->ntiles, parity, st);
        if (b->prec == LBM_FP32C)
            return launch_batch_staged<f32c>((f32c*)b->fa, (f32c*)b->fb, b->dinst, b->dstiles, b->dmaps,
                                             b->ntiles, parity, st);
        if (b->prec == LBM_FP16S)
            return launch_batch_staged<__half>((__half*)b->fa, (__half*)b->fb, b->dinst, b->dstiles, b->dmaps,
                                               b->ntiles, parity, st);
        return launch_batch_staged<__nv_bfloat16>((__nv_bfloat16*)b->fa, (__nv_bfloat16*)b->fb, b->dinst,
                                                  b->dstiles, b->dmaps, b->ntiles, parity, st);
    }
    switch (b->prec) {
        case LBM_FP64: return launch_batch_step<double>((double*)b->fa, (double*)b->fb, b->dinst, b->dtiles, b->links, b->ntiles, parity, st);
        case LBM_FP32: return launch_batch_step<float>((float*)b->fa, (float*)b->fb, b->dinst, b->dtiles, b->links, b->ntiles, parity, st);
        case LBM_FP32C: return launch_batch_step<f32c>((f32c*)b->fa, (f32c*)b->fb, b->dinst, b->dtiles, b->links, b->ntiles, parity, st);
        case LBM_FP16S: return launch_batch_step<__half>((__half*)b->fa, (__half*)b->fb, b->dinst, b->dtiles, b->links, b->ntiles, parity, st);
        default: return launch_batch_step<__nv_bfloat16>((__nv_bfloat16*)b->fa, (__nv_bfloat16*)b->fb, b->dinst, b->dtiles, b->links, b->ntiles, parity, st);
    }
}

int build_batch_graph(lbm_batch_t* b, int parity) {
    cudaGraph_t g = nullptr;
    BTRY(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    int p = parity;
    for (int k = 0; k < kBatchGraphSteps && le == cudaSuccess; k++) {
        le = step_once(b, p, b->capture);
        p = 1 - p;
    }
    cudaError_t ce = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return batch_fail(b, LBM_ECUDA, "batch graph capture failed: %s",
                          cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return batch_fail(b, LBM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(ie));
    return LBM_OK;
}

template <typename S>
void launch_init(const lbm_instance& in, const BatchInst& I, char* fa, const uint16_t* links, const double* d_rho,
                 cudaStream_t st) {
    dim3 blk(256), grd((I.pitch + 255) / 256, I.ny);
    init_kernel<S><<<grd, blk, 0, st>>>(d_rho, links + I.loff, (S*)fa + I.off, in.nx, in.ny, I.pitch, in.periodic_x);
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_instance* inst, int32_t n, int32_t precision, int32_t eq_order, void* stream,
                     lbm_batch_t** out) {
    if (!out) return batch_fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!inst || n < 1) return batch_fail(nullptr, LBM_EINVAL, "need n >= 1 instances");
    const size_t es = esize(precision);
    if (es == 0) return batch_fail(nullptr, LBM_EINVAL, "unknown precision %d", precision);
    if (eq_order != 2 && eq_order != 3) return batch_fail(nullptr, LBM_EINVAL, "eq_order must be 2 or 3");
    const int np = planes_for(precision);

    lbm_batch_t* b = new (std::nothrow) lbm_batch_t();
    if (!b) return batch_fail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->n = n;
    b->prec = precision;
    b->es = es;
    b->stream = (cudaStream_t)stream;
    b->hinst.resize(n);

    // per-instance layout and validation
    size_t off = 0, loff = 0;
    int tiles = 0;
    size_t max_stage = 0;
    for (int i = 0; i < n; i++) {
        const lbm_instance& in = inst[i];
        BatchInst& I = b->hinst[i];
        memset(&I, 0, sizeof I);
        if (in.nx < 1 || in.ny < 1 || !in.mask || !in.rho_init) {
            delete b;
            return batch_fail(nullptr, LBM_EINVAL, "instance %d: bad size or NULL mask/rho_init", i);
        }
        if (in.collision != 0 && in.collision != 1) {
            delete b;
            return batch_fail(nullptr, LBM_EINVAL, "instance %d: collision must be 0 or 1", i);
        }
        for (int a = 0; a < 2; a++)
            if (!(in.tau[a] > 0.5)) {
                delete b;
                return batch_fail(nullptr, LBM_EINVAL, "instance %d: tau[%d] must exceed 1/2", i, a);
            }
        const int nx = in.nx, ny = in.ny;
        if (!in.periodic_x)
            for (int y = 0; y < ny; y++)
                if (!in.mask[(size_t)y * nx] || !in.mask[(size_t)y * nx + nx - 1]) {
                    delete b;
                    return batch_fail(nullptr, LBM_EINVAL, "instance %d: x not periodic but boundary fluid", i);
                }
        if (!in.periodic_y)
            for (int x = 0; x < nx; x++)
                if (!in.mask[x] || !in.mask[(size_t)(ny - 1) * nx + x]) {
                    delete b;
                    return batch_fail(nullptr, LBM_EINVAL, "instance %d: y not periodic but boundary fluid", i);
                }
        {
            const size_t nn = (size_t)nx * ny;
            for (size_t k = 0; k < nn; k++) {
                if (in.mask[k]) continue;
                const double a = in.rho_init[k], c = in.rho_init[nn + k];
                if (!(a >= 0.0) || !(c >= 0.0) || !(a + c > 0.0) || !std::isfinite(a + c)) {
                    delete b;
                    return batch_fail(nullptr, LBM_EINVAL,
                                      "instance %d: rho_init must be finite, >= 0, with positive total at fluid "
                                      "nodes", i);
                }
            }
        }
        I.nx = nx;
        I.ny = ny;
        I.pitch = (nx + 2 * kGhost + 31) / 32 * 32;
        I.periodic_x = in.periodic_x;
        I.ncb = (nx + kTileX - 1) / kTileX;
        I.strips = std::max(1, std::min(ny, (ny + 31) / 32));   // strips of ~32 rows
        I.rpb = (ny + I.strips - 1) / I.strips;
        I.strips = (ny + I.rpb - 1) / I.rpb;
        I.tile0 = tiles;
        I.ntiles = I.ncb * I.strips;
        tiles += I.ntiles;
        I.active = 1;
        const size_t plane = (size_t)ny * I.pitch;
        if (plane * np >= (size_t(1) << 31)) {
            delete b;
            return batch_fail(nullptr, LBM_EINVAL, "instance %d too large", i);
        }
        I.off = (long long)off;
        off += a256(plane * np * es) / es;
        I.loff = (long long)loff;
        loff += a256(plane * 2) / 2;
        max_stage = std::max(max_stage, (size_t)nx * ny * 17);
        I.prm.nu[0] = (in.tau[0] - 0.5) / 3.0;
        I.prm.nu[1] = (in.tau[1] - 0.5) / 3.0;
        I.prm.G = in.G;
        I.prm.rho_wall[0] = in.rho_wall[0];
        I.prm.rho_wall[1] = in.rho_wall[1];
        I.prm.g[0] = in.g[0];
        I.prm.g[1] = in.g[1];
        I.prm.k3 = eq_order >= 3 ? 4.5 : 0.0;
        I.prm.reg = in.collision == 1 ? 1.0 : 0.0;
        I.disp_thr = in.disp_threshold;
        I.status = -1;
    }
    b->region_elems = off;
    b->ntiles = tiles;

    // staged tiles (FP32 and the 16-bit formats): strips of R rows.  The
    // candidates are R = 8, 16, 32, 48, 64 and the R whose tiles fill about
    // four waves of resident CTAs; they are timed on the batch itself once
    // its state is set up (GB300LBM_BATCH_ROWS pins one R, no timing)
    std::vector<TileSet> cands;
    if (precision != LBM_FP64) {
        std::vector<std::vector<int>> lo(n), hi(n);
        long long block_rows_total = 0;
        for (int i = 0; i < n; i++) {
            block_rows(inst[i].mask, inst[i].nx, inst[i].ny, lo[i], hi[i]);
            for (size_t k = 0; k < lo[i].size(); k++) block_rows_total += std::max(0, hi[i][k] - lo[i][k] + 1);
        }
        int dev = 0, sms = 148, per_sm = 4;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (precision == LBM_FP32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_staged_kernel<float>, kTileX,
                                                          StagedPlan<float, kTileX, 1>::kBytes);
        else if (precision == LBM_FP32C)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_staged_kernel<f32c>, kTileX,
                                                          StagedPlan<f32c, kTileX, 1>::kBytes);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_staged_kernel<__half>, kTileX,
                                                          StagedPlan<__half, kTileX, 1>::kBytes);
        cudaGetLastError();
        const long long waves4 = 4LL * sms * std::max(1, per_sm);
        std::vector<int> rs = {(int)std::max(8LL, std::min(64LL, block_rows_total / std::max(1LL, waves4))), 8, 16,
                               32, 48, 64};
        if (const char* e = getenv("GB300LBM_BATCH_ROWS")) {
            const int r = atoi(e);
            if (r >= 1) rs = {r};
        }
        for (int R : rs) {
            bool dup = false;
            for (const TileSet& c : cands) dup |= c.R == R;
            if (dup) continue;
            TileSet c;
            c.R = R;
            c.t0.resize(n);
            c.nt.resize(n);
            for (int i = 0; i < n; i++) {
                c.t0[i] = (int)c.tiles.size();
                staged_tiles(lo[i], hi[i], inst[i].ny, i, R, c.tiles);
                c.nt[i] = (int)c.tiles.size() - c.t0[i];
            }
            cands.push_back(std::move(c));
        }
    }
    size_t max_stiles = 0;
    for (const TileSet& c : cands) max_stiles = std::max(max_stiles, c.tiles.size());
    const size_t region = off * es;
    const size_t lbytes = a256(loff * 2);
    const size_t ibytes = a256(sizeof(BatchInst) * n);
    const size_t tbytes = a256(sizeof(int) * tiles);
    const size_t stbytes = a256(sizeof(BatchTile) * max_stiles);
    const size_t mbytes = precision != LBM_FP64 ? a256(sizeof(CUtensorMap) * 3 * n) : 0;
    const size_t total = 3 * region + lbytes + ibytes + tbytes + 256 + stbytes + mbytes;
    cudaError_t e = cudaMalloc(&b->arena, total);
    if (e != cudaSuccess) {
        delete b;
        return batch_fail(nullptr, LBM_ENOMEM, "cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
    }
    char* p = (char*)b->arena;
    b->fa = p;
    b->fb = p + region;
    b->snap = p + 2 * region;
    b->links = (uint16_t*)(p + 3 * region);
    b->dinst = (BatchInst*)(p + 3 * region + lbytes);
    b->dtiles = (int*)(p + 3 * region + lbytes + ibytes);
    b->dcount = (int*)(p + 3 * region + lbytes + ibytes + tbytes);
    b->dstiles = stbytes ? (BatchTile*)(p + 3 * region + lbytes + ibytes + tbytes + 256) : nullptr;
    b->dmaps = mbytes ? (CUtensorMap*)(p + 3 * region + lbytes + ibytes + tbytes + 256 + stbytes) : nullptr;
    auto bail = [&](int code) {
        std::string m = g_batch_err;
        lbm_batch_destroy(b);
        g_batch_err = m;
        return code;
    };
#define CTRY(call)                                                                                 \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            batch_fail(nullptr, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
            return bail(LBM_ECUDA);                                                                \
        }                                                                                          \
    } while (0)
    CTRY(cudaMallocHost(&b->hcount, sizeof(int)));
    CTRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    CTRY(cudaMemsetAsync(b->arena, 0, 3 * region + lbytes, b->stream));
    std::vector<int> tile_inst(tiles);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < b->hinst[i].ntiles; k++) tile_inst[b->hinst[i].tile0 + k] = i;
    CTRY(cudaMemcpyAsync(b->dtiles, tile_inst.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice, b->stream));
    // the staged kernel, unless the driver refuses a tensor map (then every
    // format runs the register-pull kernel)
    if (precision != LBM_FP64) {
        std::vector<CUtensorMap> maps(3 * (size_t)n);
        bool ok = true;
        for (int i = 0; i < n && ok; i++)
            ok = encode_instance_maps(&maps[3 * (size_t)i], b->hinst[i], precision, es, np, b->fa, b->fb, b->links);
        if (ok) {
            CTRY(staged_attr_for(precision));
            CTRY(cudaMemcpyAsync(b->dmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                                 b->stream));
            CTRY(cudaStreamSynchronize(b->stream));
            b->staged = true;
        }
    }
    CTRY(cudaMemcpyAsync(b->dinst, b->hinst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, b->stream));
    // per instance: stage mask + densities in the snapshot region, links, init A
    for (int i = 0; i < n; i++) {
        const lbm_instance& in = inst[i];
        const BatchInst& I = b->hinst[i];
        const size_t nn = (size_t)in.nx * in.ny;
        double* d_rho = (double*)b->snap;
        uint8_t* d_mask = (uint8_t*)(b->snap + a256(nn * 16));
        if (a256(nn * 16) + nn > region) {
            batch_fail(nullptr, LBM_EINVAL, "instance %d larger than the staging region", i);
            return bail(LBM_EINVAL);
        }
        CTRY(cudaMemcpyAsync(d_rho, in.rho_init, nn * 16, cudaMemcpyHostToDevice, b->stream));
        CTRY(cudaMemcpyAsync(d_mask, in.mask, nn, cudaMemcpyHostToDevice, b->stream));
        dim3 blk(256), grd((I.pitch + 255) / 256, in.ny);
        links_kernel<<<grd, blk, 0, b->stream>>>(d_mask, b->links + I.loff, in.nx, in.ny, I.pitch, in.periodic_x);
        switch (precision) {
            case LBM_FP64: launch_init<double>(in, I, b->fa, b->links, d_rho, b->stream); break;
            case LBM_FP32: launch_init<float>(in, I, b->fa, b->links, d_rho, b->stream); break;
            case LBM_FP32C: launch_init<f32c>(in, I, b->fa, b->links, d_rho, b->stream); break;
            case LBM_FP16S: launch_init<__half>(in, I, b->fa, b->links, d_rho, b->stream); break;
            default: launch_init<__nv_bfloat16>(in, I, b->fa, b->links, d_rho, b->stream); break;
        }
        CTRY(cudaGetLastError());
        CTRY(cudaStreamSynchronize(b->stream));   // the staging area is reused by the next instance
    }
    if (b->staged) {
        // time the strip-row candidates: steps A -> B only (A keeps the
        // initial state), then the pristine instance records go back up
        auto use = [&](const TileSet& c, std::vector<BatchInst>& h) -> cudaError_t {
            for (int i = 0; i < n; i++) {
                h[i].tile0 = c.t0[i];
                h[i].ntiles = c.nt[i];
            }
            b->ntiles = (int)c.tiles.size();
            b->strip_rows = c.R;
            cudaError_t e1 = cudaMemcpyAsync(b->dstiles, c.tiles.data(), sizeof(BatchTile) * c.tiles.size(),
                                             cudaMemcpyHostToDevice, b->stream);
            if (e1 == cudaSuccess)
                e1 = cudaMemcpyAsync(b->dinst, h.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, b->stream);
            if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(b->stream);
            return e1;
        };
        size_t best = 0;
        if (cands.size() > 1) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            CTRY(cudaEventCreate(&e0));
            CTRY(cudaEventCreate(&e1));
            float best_ms = 1e30f;
            std::vector<BatchInst> h = b->hinst, back(n);
            cudaError_t te = cudaSuccess;
            for (size_t k = 0; k < cands.size() && te == cudaSuccess; k++) {
                te = use(cands[k], h);
                if (te == cudaSuccess) te = step_once(b, 0, b->stream);
                if (te == cudaSuccess) te = cudaEventRecord(e0, b->stream);
                for (int r = 0; r < 3 && te == cudaSuccess; r++) te = step_once(b, 0, b->stream);
                if (te == cudaSuccess) te = cudaEventRecord(e1, b->stream);
                if (te == cudaSuccess) te = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, e0, e1);
                if (te == cudaSuccess)
                    te = cudaMemcpyAsync(back.data(), b->dinst, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost,
                                         b->stream);
                if (te == cudaSuccess) te = cudaStreamSynchronize(b->stream);
                bool gave_up = false;
                for (int i = 0; i < n; i++) gave_up |= back[i].obs.timeout_flag != 0;
                // a candidate whose bounded waits gave up is not a candidate
                if (te == cudaSuccess && !gave_up && ms < best_ms) {
                    best_ms = ms;
                    best = k;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CTRY(te);
        }
        CTRY(use(cands[best], b->hinst));
    }
    CTRY(cudaMemcpyAsync(b->fb, b->fa, region, cudaMemcpyDeviceToDevice, b->stream));
    CTRY(cudaMemcpyAsync(b->snap, b->fa, region, cudaMemcpyDeviceToDevice, b->stream));
    CTRY(cudaStreamSynchronize(b->stream));
#undef CTRY
    b->parity = 0;
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch_t* b, int64_t nsteps) {
    if (!b) return batch_fail(nullptr, LBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return batch_fail(b, LBM_EINVAL, "nsteps < 0");
    int64_t left = nsteps;
    if (left >= kBatchGraphSteps) {
        if (!b->graph[b->parity]) {
            int rc = build_batch_graph(b, b->parity);
            if (rc) return rc;
        }
        while (left >= kBatchGraphSteps) {
            BTRY(b, cudaGraphLaunch(b->graph[b->parity], b->stream));
            left -= kBatchGraphSteps;
        }
    }
    for (; left > 0; left--) {
        BTRY(b, step_once(b, b->parity, b->stream));
        b->parity = 1 - b->parity;
    }
    return LBM_OK;
}

int lbm_batch_observables(lbm_batch_t* b, lbm_obs* out) {
    if (!b || !out) return batch_fail(b, LBM_EINVAL, "NULL argument");
    std::vector<BatchInst> h(b->n);
    BTRY(b, cudaMemcpyAsync(h.data(), b->dinst, sizeof(BatchInst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    int rc = LBM_OK;
    for (int i = 0; i < b->n; i++) {
        const ObsState& s = h[i].obs;
        out[i].mass[0] = s.mass[0];
        out[i].mass[1] = s.mass[1];
        out[i].oil_mom_x = s.px;
        out[i].oil_disp_x = s.disp;
        out[i].max_u = s.umax;
        out[i].step = s.step;
        out[i].nan_flag = s.nan_flag;
        out[i].timeout_flag = s.timeout_flag;
        if (s.nan_flag && rc == LBM_OK) rc = LBM_EUNSTABLE;
        if (s.timeout_flag && rc == LBM_OK) rc = LBM_ETIMEOUT;
    }
    if (rc == LBM_EUNSTABLE) batch_fail(b, rc, "an instance reached a NaN or negative density");
    else if (rc) batch_fail(b, rc, "a bounded device wait gave up: the state of that step is invalid");
    return rc;
}

int lbm_batch_kernel_info(const lbm_batch_t* b, int32_t info[3]) {
    if (!b || !info) return batch_fail(nullptr, LBM_EINVAL, "NULL argument");
    info[0] = b->staged ? 2 : 1;
    info[1] = b->staged ? b->strip_rows : 0;
    info[2] = b->ntiles;
    return LBM_OK;
}

int lbm_batch_set_body_force(lbm_batch_t* b, const double* gx) {
    if (!b || !gx) return batch_fail(b, LBM_EINVAL, "NULL argument");
    for (int i = 0; i < b->n; i++)
        if (!std::isfinite(gx[i])) return batch_fail(b, LBM_EINVAL, "g of instance %d is not finite", i);
    // patch the g[0] field of every record (a small host round trip)
    std::vector<BatchInst> h(b->n);
    BTRY(b, cudaMemcpyAsync(h.data(), b->dinst, sizeof(BatchInst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; i++) h[i].prm.g[0] = gx[i];
    BTRY(b, cudaMemcpyAsync(b->dinst, h.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_save(lbm_batch_t* b, int32_t i, double* f) {
    if (!b || !f || i < 0 || i >= b->n) return batch_fail(b, LBM_EINVAL, "bad argument");
    const BatchInst& I = b->hinst[i];
    const int np = planes_for(b->prec);
    const size_t plane = (size_t)I.ny * I.pitch;
    std::vector<char> raw(plane * np * b->es);
    std::vector<uint16_t> lk(plane);
    const char* src = (b->parity ? b->fb : b->fa) + (size_t)I.off * b->es;
    BTRY(b, cudaMemcpyAsync(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaMemcpyAsync(lk.data(), b->links + I.loff, plane * 2, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    const bool shifted = np == 20;
    const float w5f = [] {
        uint32_t bits = 0x3CE38E38u;
        float w;
        memcpy(&w, &bits, sizeof w);
        return w;
    }();
    auto wf = [&](int d) { return d == 0 ? 4.0f / 9.0f : (d <= 4 ? 1.0f / 9.0f : w5f); };
    auto get = [&](size_t k) -> double {
        switch (b->prec) {
            case LBM_FP64: return ((const double*)raw.data())[k];
            case LBM_FP32:
            case LBM_FP32C: return ((const float*)raw.data())[k];
            case LBM_FP16S: return __half2float(((const __half*)raw.data())[k]);
            default: return __bfloat162float(((const __nv_bfloat16*)raw.data())[k]);
        }
    };
    for (int y = 0; y < I.ny; y++)
        for (int x = 0; x < I.nx; x++) {
            const size_t node = (size_t)y * I.pitch + kGhost + x;
            const bool solid = lk[node] & (1u << kSolidBit);
            for (int a = 0; a < 2; a++) {
                const float rh = shifted ? (float)get((18 + a) * plane + node) : 0.f;
                for (int d = 0; d < 9; d++) {
                    const double s = get((a * 9 + d) * plane + node);
                    const double v = shifted ? (double)std::fma(wf(d), rh, (float)s) : s;
                    f[((size_t)(a * 9 + d) * I.ny + y) * I.nx + x] = solid ? 0.0 : v;
                }
            }
        }
    return LBM_OK;
}

int lbm_critical_pressure_batch(lbm_batch_t* b, const double* g_lo, const double* g_hi, const lbm_bisect_opts* o,
                                lbm_crit_result* out) {
    if (!b || !g_lo || !g_hi || !o || !out) return batch_fail(b, LBM_EINVAL, "NULL argument");
    if (!(o->rel_bracket > 0.0) || o->t_obs < 1 || o->t_eq < 0 || o->max_probes < 1)
        return batch_fail(b, LBM_EINVAL, "bad bisection options");
    for (int i = 0; i < b->n; i++)
        if (!(g_lo[i] > 0.0) || !(g_hi[i] > g_lo[i]) || !std::isfinite(g_hi[i]))
            return batch_fail(b, LBM_EINVAL, "instance %d: need 0 < g_lo < g_hi < infinity", i);
    const auto t_start = std::chrono::steady_clock::now();
    // reset records: bracket, state machine, observables; everyone active
    std::vector<BatchInst> h(b->n);
    BTRY(b, cudaMemcpyAsync(h.data(), b->dinst, sizeof(BatchInst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; i++) {
        BatchInst& I = h[i];
        I.g_lo = g_lo[i];
        I.g_hi = g_hi[i];
        I.state = o->check_bracket ? kCheckHi : kBisect;
        I.probes = 0;
        I.status = -1;
        I.active = 1;
        I.prm.g[0] = 0.0;                      // equilibrate without driving (Section 3.4)
        memset(&I.acc, 0, sizeof I.acc);
        memset(&I.obs, 0, sizeof I.obs);
    }
    BTRY(b, cudaMemcpyAsync(b->dinst, h.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, b->stream));
    int rc = lbm_batch_step(b, o->t_eq);
    if (rc) return rc;
    // the equilibrated state is the start of every probe
    const size_t region = b->region_elems * b->es;
    BTRY(b, cudaMemcpyAsync(b->snap, b->parity ? b->fb : b->fa, region, cudaMemcpyDeviceToDevice, b->stream));
    const int thr = 128, blocks = (b->n + thr - 1) / thr;
    int active = b->n;
    bool timed_out = false;
    while (active > 0) {
        BTRY(b, cudaMemcpyAsync(b->fa, b->snap, region, cudaMemcpyDeviceToDevice, b->stream));
        b->parity = 0;
        probe_begin_kernel<<<blocks, thr, 0, b->stream>>>(b->dinst, b->n);
        BTRY(b, cudaGetLastError());
        rc = lbm_batch_step(b, o->t_obs);
        if (rc) return rc;
        BTRY(b, cudaMemsetAsync(b->dcount, 0, sizeof(int), b->stream));
        probe_decide_kernel<<<blocks, thr, 0, b->stream>>>(b->dinst, b->n, o->rel_bracket, o->max_probes, b->dcount);
        BTRY(b, cudaGetLastError());
        BTRY(b, cudaMemcpyAsync(b->hcount, b->dcount, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        BTRY(b, cudaStreamSynchronize(b->stream));
        active = *b->hcount;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (active > 0 && o->timeout_s > 0.0 && el > o->timeout_s) {
            timed_out = true;
            break;
        }
    }
    BTRY(b, cudaMemcpyAsync(h.data(), b->dinst, sizeof(BatchInst) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; i++) {
        out[i].g_lo = h[i].g_lo;
        out[i].g_hi = h[i].g_hi;
        out[i].probes = h[i].probes;
        out[i].status = h[i].active ? 3 : h[i].status;   // 3: stopped by the timeout
    }
    if (timed_out) return batch_fail(b, LBM_ETIMEOUT, "bisection stopped by timeout_s with %d active", active);
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_t* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    for (auto& g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->hcount) cudaFreeHost(b->hcount);
    if (b->arena) cudaFree(b->arena);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch_t* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
