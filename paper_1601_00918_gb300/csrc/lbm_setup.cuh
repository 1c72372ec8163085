// Set-up kernels shared by the single-grid and the batched runtimes: link
// words from a wall mask, and the initial stored state from densities.
#pragma once

#include <climits>

#include "lbm_common.cuh"

namespace gb300lbm {

// Logical column of a storage column, or INT_MIN when it holds nothing
// (padding, or a ghost of a non-periodic grid).
__device__ __forceinline__ int logical_col(int sc, int nx, int periodic) {
    const int x = sc - kGhost;
    if (x >= 0 && x < nx) return x;
    if (!periodic || x < -kGhost || x >= nx + kGhost) return INT_MIN;
    int m = x % nx;
    return m < 0 ? m + nx : m;
}

static __global__ void links_kernel(const uint8_t* __restrict__ mask, uint16_t* __restrict__ links, int nx,
                             int ny, int pitch, int periodic) {
    const int sc = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (sc >= pitch || y >= ny) return;
    const int x = logical_col(sc, nx, periodic);
    if (x == INT_MIN) {
        links[y * pitch + sc] = uint16_t(1u << kSolidBit);
        return;
    }
    unsigned w = mask[y * nx + x] ? (1u << kSolidBit) : 0u;
    for (int i = 1; i < 9; i++) {
        int sx = x - d2q9_cx(i), sy = y - d2q9_cy(i);
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        if (mask[sy * nx + sx]) w |= 1u << i;
    }
    links[y * pitch + sc] = uint16_t(w);
}

template <typename S>
static __global__ void init_kernel(const double* __restrict__ rho, const uint16_t* __restrict__ links,
                            S* __restrict__ f, int nx, int ny, int pitch, int periodic) {
    using C = Codec<S>;
    using R = typename C::R;
    const int sc = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (sc >= pitch || y >= ny) return;
    const int plane = ny * pitch;
    const int x = logical_col(sc, nx, periodic);
    const bool solid = x == INT_MIN || (links[y * pitch + sc] & (1u << kSolidBit));
    S* node = f + y * pitch + sc;
    for (int a = 0; a < 2; a++) {
        const double r = solid ? 0.0 : rho[(size_t)a * nx * ny + (size_t)y * nx + x];
        // solid nodes, padding and unused ghosts hold the stored value 0
        R rh = R(0);
        if (C::kNodeShift) {
            const S q = C::rho_store(R(r));
            node[(18 + a) * plane] = q;
            rh = C::rho_value(q);
        }
        for (int i = 0; i < 9; i++)
            node[(a * 9 + i) * plane] = C::encode(R(weight_of<double>(i) * r), wgt<R>(i), rh);
    }
}

// One pass over the mask and the initial densities of a single grid: the
// number of fluid nodes (*nfluid), the first and last fluid row of every
// 64-column block (rows64, initialised to (ny, -1)), and *bad = 1 if a fluid
// node's densities are not finite, not >= 0, or sum to 0.  A block of
// blockDim.x (a multiple of 32) columns of one row per CTA; a warp spans 32
// columns of one 64-column block.
static __global__ void scan_kernel(const uint8_t* __restrict__ mask, const double* __restrict__ rho, int nx,
                                   int ny, int2* __restrict__ rows64, unsigned long long* __restrict__ nfluid,
                                   int* __restrict__ bad) {
    __shared__ unsigned count;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    const size_t k = (size_t)y * nx + x;
    const bool fluid = x < nx && y < ny && !mask[k];
    if (fluid) {
        const double a = rho[k], b = rho[(size_t)nx * ny + k];
        if (!(a >= 0.0) || !(b >= 0.0) || !(a + b > 0.0) || !isfinite(a + b)) atomicOr(bad, 1);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, fluid);
    if ((threadIdx.x & 31) == 0 && ballot) {
        atomicAdd(&count, (unsigned)__popc(ballot));
        int2* r = rows64 + x / 64;
        atomicMin(&r->x, y);
        atomicMax(&r->y, y);
    }
    __syncthreads();
    if (threadIdx.x == 0 && count) atomicAdd(nfluid, (unsigned long long)count);
}

}  // namespace gb300lbm
