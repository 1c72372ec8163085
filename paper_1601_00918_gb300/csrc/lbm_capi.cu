// Runtime and C ABI (include/lbm.h) of the two-component D2Q9 library.
//
// A handle owns: two population buffers A/B (ping-pong, layout
// f[species][direction][y][pitch], x fastest, pitch = nx rounded up to 32
// elements so every row starts 128-byte aligned), a 16-bit link word per node
// (bit i set when the pull source x - c_i is solid, bit 15 when the node itself
// is solid), the device parameter block, the per-step reduction accumulators
// and the finalised observables.  All device memory comes from one arena,
// either allocated here or supplied by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_step.cuh"

using namespace gb300lbm;

struct lbm_t {
    lbm_params p{};
    int pitch = 0;
    size_t elem = 0;              // bytes per stored population
    size_t buf_bytes = 0;         // one population buffer
    void* arena = nullptr;
    bool own_arena = false;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;                  // f[cur] holds the current stored state
    uint16_t* links = nullptr;
    StepParams* dprm = nullptr;
    ObsAccum* dacc = nullptr;
    ObsState* dobs = nullptr;
    StepParams hprm{};
    cudaStream_t stream = nullptr;
    int rows_per_block = 0;
    int64_t fluid_nodes = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

constexpr int kBX = 128;

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
        case LBM_FP32: return 4;
        case LBM_FP16S:
        case LBM_BF16S: return 2;
        default: return 0;
    }
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    int pitch;
    size_t buf, links, prm, acc, obs, total;
};

bool layout_of(const lbm_params* p, Layout* L) {
    const size_t es = elem_size(p->precision);
    if (es == 0 || p->nx < 1 || p->ny < 1) return false;
    L->pitch = (p->nx + 31) / 32 * 32;
    const size_t plane = (size_t)p->ny * L->pitch;
    // kernel indices are 32-bit: all 18 planes must fit below 2^31 elements
    if (plane * 18 >= (size_t(1) << 31)) return false;
    L->buf = align256(plane * 18 * es);
    L->links = align256(plane * sizeof(uint16_t));
    L->prm = align256(sizeof(StepParams));
    L->acc = align256(sizeof(ObsAccum));
    L->obs = align256(sizeof(ObsState));
    L->total = 2 * L->buf + L->links + L->prm + L->acc + L->obs;
    return true;
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------
__global__ void links_kernel(const uint8_t* __restrict__ mask, uint16_t* __restrict__ links, int nx,
                             int ny, int pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= pitch || y >= ny) return;
    if (x >= nx) {
        links[y * pitch + x] = uint16_t(1u << kSolidBit);
        return;
    }
    unsigned w = mask[y * nx + x] ? (1u << kSolidBit) : 0u;
    for (int i = 1; i < 9; i++) {
        int sx = x - d2q9_cx(i), sy = y - d2q9_cy(i);
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        if (mask[sy * nx + sx]) w |= 1u << i;
    }
    links[y * pitch + x] = uint16_t(w);
}

template <typename S>
__global__ void init_kernel(const double* __restrict__ rho, const uint16_t* __restrict__ links,
                            S* __restrict__ f, int nx, int ny, int pitch, double ref0, double ref1) {
    using R = typename Codec<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= pitch || y >= ny) return;
    const int plane = ny * pitch;
    const bool solid = x >= nx || (links[y * pitch + x] & (1u << kSolidBit));
    for (int a = 0; a < 2; a++) {
        const double r = solid ? 0.0 : rho[(size_t)a * nx * ny + (size_t)y * nx + x];
        const double ref = a ? ref1 : ref0;
        for (int i = 0; i < 9; i++) {
            const double w = weight_of<double>(i);
            S* dst = f + (a * 9 + i) * plane + y * pitch + x;
            // solid nodes and padding hold the stored value 0
            if (solid)
                Codec<S>::store(dst, R(0), R(0));
            else
                Codec<S>::store(dst, R(w * r), R(w * ref));
        }
    }
}

template <typename S>
void launch_step(lbm_t* h, const void* fin, void* fout, bool fields, double* out, int row_begin,
                 int row_end) {
    Grid g;
    g.nx = h->p.nx;
    g.ny = h->p.ny;
    g.pitch = h->pitch;
    g.rows_per_block = h->rows_per_block;
    g.row_begin = row_begin;
    g.row_end = row_end;
    dim3 grid((h->p.nx + kBX - 1) / kBX, (row_end - row_begin + g.rows_per_block - 1) / g.rows_per_block);
    if (fields)
        step_kernel<S, kBX, true><<<grid, kBX, 0, h->stream>>>(
            (const S*)fin, (S*)fout, h->links, h->dprm, h->dacc, h->dobs, out, g);
    else
        step_kernel<S, kBX, false><<<grid, kBX, 0, h->stream>>>(
            (const S*)fin, (S*)fout, h->links, h->dprm, h->dacc, h->dobs, out, g);
}

void dispatch_step(lbm_t* h, const void* fin, void* fout, bool fields, double* out, int rb, int re) {
    switch (h->p.precision) {
        case LBM_FP64: launch_step<double>(h, fin, fout, fields, out, rb, re); break;
        case LBM_FP32: launch_step<float>(h, fin, fout, fields, out, rb, re); break;
        case LBM_FP16S: launch_step<__half>(h, fin, fout, fields, out, rb, re); break;
        case LBM_BF16S: launch_step<__nv_bfloat16>(h, fin, fout, fields, out, rb, re); break;
    }
}

// Rows per CTA strip: enough CTAs to fill the 152 SMs several times over,
// but strips long enough that the two halo rows stay a small overhead.
int choose_rows_per_block(int nx, int ny) {
    const int cols = (nx + kBX - 1) / kBX;
    const int target_ctas = 152 * 8;
    int rpb = (int)((int64_t)cols * ny / std::max(target_ctas, 1));
    rpb = std::max(4, std::min(rpb, 128));
    return std::min(rpb, ny);
}

// host conversions for save/load
double to_double(const void* base, size_t k, int prec) {
    switch (prec) {
        case LBM_FP64: return ((const double*)base)[k];
        case LBM_FP32: return ((const float*)base)[k];
        case LBM_FP16S: return __half2float(((const __half*)base)[k]);
        default: return __bfloat162float(((const __nv_bfloat16*)base)[k]);
    }
}

void from_double(void* base, size_t k, int prec, double v) {
    switch (prec) {
        case LBM_FP64: ((double*)base)[k] = v; break;
        case LBM_FP32: ((float*)base)[k] = (float)v; break;
        case LBM_FP16S: ((__half*)base)[k] = __float2half_rn((float)v); break;
        default: ((__nv_bfloat16*)base)[k] = __float2bfloat16_rn((float)v); break;
    }
}

double host_weight(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

int validate(const lbm_params* p, const uint8_t* mask) {
    if (!p) return fail(nullptr, LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(nullptr, LBM_EINVAL, "nx, ny must be >= 1");
    if (elem_size(p->precision) == 0) return fail(nullptr, LBM_EINVAL, "unknown precision %d", p->precision);
    if (p->eq_order != 2 && p->eq_order != 3) return fail(nullptr, LBM_EINVAL, "eq_order must be 2 or 3");
    for (int a = 0; a < 2; a++)
        if (!(p->tau[a] > 0.5)) return fail(nullptr, LBM_EINVAL, "tau[%d] must exceed 1/2", a);
    if (!std::isfinite(p->G) || !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]))
        return fail(nullptr, LBM_EINVAL, "G and g must be finite");
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

    // host checks and the reference densities of the 16-bit storage shift
    double sum[2] = {0.0, 0.0};
    int64_t nfluid = 0;
    for (size_t k = 0; k < n; k++) {
        if (mask[k]) continue;
        const double a = rho_init[k], b = rho_init[n + k];
        if (!(a >= 0.0) || !(b >= 0.0) || !(a + b > 0.0) || !std::isfinite(a + b))
            return fail(nullptr, LBM_EINVAL, "rho_init must be finite, >= 0, with positive total at fluid nodes");
        sum[0] += a;
        sum[1] += b;
        nfluid++;
    }

    lbm_t* h = new (std::nothrow) lbm_t();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    h->p = *p;
    h->stream = (cudaStream_t)p->cuda_stream;
    h->fluid_nodes = nfluid;
    Layout L;
    layout_of(p, &L);
    h->pitch = L.pitch;
    h->elem = elem_size(p->precision);
    h->buf_bytes = L.buf;
    h->rows_per_block = choose_rows_per_block(nx, ny);

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
    h->f[0] = base;
    h->f[1] = base + L.buf;
    h->links = (uint16_t*)(base + 2 * L.buf);
    h->dprm = (StepParams*)(base + 2 * L.buf + L.links);
    h->dacc = (ObsAccum*)(base + 2 * L.buf + L.links + L.prm);
    h->dobs = (ObsState*)(base + 2 * L.buf + L.links + L.prm + L.acc);

    fill_params(h);
    if (p->precision == LBM_FP16S || p->precision == LBM_BF16S) {
        for (int a = 0; a < 2; a++) h->hprm.rho_ref[a] = nfluid ? sum[a] / nfluid : 0.0;
    }

    // stage rho_init (FP64) and the mask in buffer B, build links, init A
    const size_t rho_bytes = n * 2 * sizeof(double);
    char* stage = (char*)h->f[1];
    double* d_rho = (double*)stage;
    uint8_t* d_mask = (uint8_t*)(stage + align256(rho_bytes));
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
    CREATE_TRY(cudaMemcpyAsync(d_rho, rho_init, rho_bytes, cudaMemcpyHostToDevice, h->stream));
    CREATE_TRY(cudaMemcpyAsync(d_mask, mask, n, cudaMemcpyHostToDevice, h->stream));
    CREATE_TRY(cudaMemsetAsync(h->dacc, 0, sizeof(ObsAccum), h->stream));
    CREATE_TRY(cudaMemsetAsync(h->dobs, 0, sizeof(ObsState), h->stream));
    CREATE_TRY(cudaMemcpyAsync(h->dprm, &h->hprm, sizeof(StepParams), cudaMemcpyHostToDevice, h->stream));
    dim3 blk(256), grd((h->pitch + 255) / 256, ny);
    links_kernel<<<grd, blk, 0, h->stream>>>(d_mask, h->links, nx, ny, h->pitch);
    const double r0 = h->hprm.rho_ref[0], r1 = h->hprm.rho_ref[1];
    switch (p->precision) {
        case LBM_FP64: init_kernel<double><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (double*)h->f[0], nx, ny, h->pitch, r0, r1); break;
        case LBM_FP32: init_kernel<float><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (float*)h->f[0], nx, ny, h->pitch, r0, r1); break;
        case LBM_FP16S: init_kernel<__half><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (__half*)h->f[0], nx, ny, h->pitch, r0, r1); break;
        default: init_kernel<__nv_bfloat16><<<grd, blk, 0, h->stream>>>(d_rho, h->links, (__nv_bfloat16*)h->f[0], nx, ny, h->pitch, r0, r1); break;
    }
    CREATE_TRY(cudaGetLastError());
    // B must hold the same zeros at solid nodes and padding as A
    CREATE_TRY(cudaMemcpyAsync(h->f[1], h->f[0], L.buf, cudaMemcpyDeviceToDevice, h->stream));
    CREATE_TRY(cudaStreamSynchronize(h->stream));
#undef CREATE_TRY
    h->cur = 0;
    *out = h;
    return LBM_OK;
}

int lbm_step(lbm_t* h, int64_t nsteps) {
    if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
    for (int64_t s = 0; s < nsteps; s++) {
        dispatch_step(h, h->f[h->cur], h->f[1 - h->cur], false, nullptr, 0, h->p.ny);
        h->cur = 1 - h->cur;
    }
    CUDA_TRY(h, cudaGetLastError());
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
    out->reserved = 0;
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
    double* stage = (double*)h->f[1 - h->cur];
    std::vector<double> tmp;
    for (int y0 = 0; y0 < ny; y0 += max_rows) {
        const int y1 = std::min(ny, y0 + max_rows);
        const size_t cnt = (size_t)nx * (y1 - y0);
        dispatch_step(h, h->f[h->cur], nullptr, true, stage, y0, y1);
        CUDA_TRY(h, cudaGetLastError());
        tmp.resize(cnt * 5);
        CUDA_TRY(h, cudaMemcpyAsync(tmp.data(), stage, cnt * 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        const size_t off = (size_t)y0 * nx;
        if (rho) {
            memcpy(rho + off, tmp.data(), cnt * sizeof(double));
            memcpy(rho + n + off, tmp.data() + cnt, cnt * sizeof(double));
        }
        if (u) {
            memcpy(u + off, tmp.data() + 2 * cnt, cnt * sizeof(double));
            memcpy(u + n + off, tmp.data() + 3 * cnt, cnt * sizeof(double));
        }
        if (pr) memcpy(pr + off, tmp.data() + 4 * cnt, cnt * sizeof(double));
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
    const int nx = h->p.nx, ny = h->p.ny, pitch = h->pitch;
    std::vector<char> raw(h->buf_bytes);
    CUDA_TRY(h, cudaMemcpyAsync(raw.data(), h->f[h->cur], h->buf_bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const bool shifted = h->p.precision == LBM_FP16S || h->p.precision == LBM_BF16S;
    std::vector<uint16_t> lk((size_t)ny * pitch);
    CUDA_TRY(h, cudaMemcpy(lk.data(), h->links, lk.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < 9; i++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    const size_t k = ((size_t)(a * 9 + i) * ny + y) * pitch + x;
                    const bool solid = lk[(size_t)y * pitch + x] & (1u << kSolidBit);
                    double v = to_double(raw.data(), k, h->p.precision);
                    if (shifted && !solid) v += host_weight(i) * h->hprm.rho_ref[a];
                    f[((size_t)(a * 9 + i) * ny + y) * nx + x] = solid ? 0.0 : v;
                }
    return LBM_OK;
}

int lbm_load(lbm_t* h, const double* f) {
    if (!h || !f) return fail(h, LBM_EINVAL, "NULL argument");
    const int nx = h->p.nx, ny = h->p.ny, pitch = h->pitch;
    std::vector<uint16_t> lk((size_t)ny * pitch);
    CUDA_TRY(h, cudaMemcpy(lk.data(), h->links, lk.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    std::vector<char> raw(h->buf_bytes, 0);
    const bool shifted = h->p.precision == LBM_FP16S || h->p.precision == LBM_BF16S;
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < 9; i++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    const size_t k = ((size_t)(a * 9 + i) * ny + y) * pitch + x;
                    const bool solid = lk[(size_t)y * pitch + x] & (1u << kSolidBit);
                    double v = f[((size_t)(a * 9 + i) * ny + y) * nx + x];
                    if (solid) v = 0.0;
                    else if (shifted) v -= host_weight(i) * h->hprm.rho_ref[a];
                    from_double(raw.data(), k, h->p.precision, v);
                }
    CUDA_TRY(h, cudaMemcpyAsync(h->f[h->cur], raw.data(), h->buf_bytes, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->dacc, 0, sizeof(ObsAccum), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->dobs, 0, sizeof(ObsState), h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

void lbm_destroy(lbm_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->own_arena && h->arena) cudaFree(h->arena);
    delete h;
}

const char* lbm_last_error(const lbm_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
