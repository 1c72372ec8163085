// Two-component lattice-Boltzmann step on the paper's own lattice, D3Q19
// (Section 2), and its C ABI (lbm3d_* in include/lbm.h).
//
// Method: as the two-dimensional step (lbm_common.cuh), per node and
// species a, with nineteen velocities c_0 = 0, the six face neighbours
// (weight 1/18) and the twelve edge neighbours (weight 1/36), T0 = 1/3:
//   pull      f_i^a(x) = f*_i^a(x - c_i), or f*_opp(i)^a(x) at a solid source
//             (halfway bounce-back);
//   density   rho^a = sum_i f_i^a, rho_s^a at a solid node;
//   force     F^a/rho^a = G sum_i w_i c_i rho^b(x + c_i) + g (Eq. comp_interaction);
//   moments   u_mix = (j^o + j^w)/rho, nu_mix, tau_mix = nu_mix/T0 + 1/2;
//   collide   f*_i = f_i^eq(rho^a, u_mix + F^a/rho^a) + (1 - 1/tau_mix) f'_i,
//             f' = f - f^eq(rho^a, u_mix) or its regularised projection
//             (Eqs. LBM_BGK, Regualize, feq, collision_term).
//
// Design: two launches per step, both over a list of the fluid nodes only
// (x fastest, so neighbouring threads hold neighbouring x and every
// population plane is read and written coalesced; solid nodes cost
// nothing).  The density pass pulls every fluid node's 38 populations and
// writes its two densities into a density field (the solid nodes' entries
// hold the wall potentials, written once at set-up); the collide-stream
// pass pulls them again, reads the 18 neighbour densities of the force from
// that field (mostly L1/L2 hits: the field of an 8-million-node tube is
// 64 MB) and writes the 38 post-collision populations.  Storage: f[species][direction][z][y][x], dense, ping-pong;
// link words (32-bit: bit i = the pull source of direction i is solid, bit
// 31 = the node is solid).  FP64 and FP32; the FP32 rest population takes
// what the other eighteen leave of rho (mass exact to rounding).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_common.cuh"

using namespace gb300lbm;

namespace {

constexpr int kQ = 19;
constexpr int kT = 128;                 // threads per block
constexpr unsigned kSolid3 = 1u << 31;

// D3Q19 in the order: rest; +x, -x, +y, -y, +z, -z; then the edges
// (+x+y), (-x-y), (+x-y), (-x+y), (+x+z), (-x-z), (+x-z), (-x+z),
// (+y+z), (-y-z), (+y-z), (-y+z): direction 2k-1 and 2k are opposite.
__host__ __device__ __forceinline__ int cx3(int i) {
    constexpr int c[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return c[i];
}
__host__ __device__ __forceinline__ int cy3(int i) {
    constexpr int c[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return c[i];
}
__host__ __device__ __forceinline__ int cz3(int i) {
    constexpr int c[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return c[i];
}
__host__ __device__ __forceinline__ int opp3(int i) { return i == 0 ? 0 : (i & 1 ? i + 1 : i - 1); }
template <typename R>
__host__ __device__ __forceinline__ R w3(int i) {
    return i == 0 ? R(1.0 / 3.0) : (i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}

struct Params3 {
    double nu[2], G, g[3], rho_wall[2], k3, reg;
};

struct Dims {
    int nx, ny, nz;
    long long n;     // nodes
};

__device__ __forceinline__ long long wrapped(const Dims& d, int x, int y, int z) {
    x = x < 0 ? x + d.nx : (x >= d.nx ? x - d.nx : x);
    y = y < 0 ? y + d.ny : (y >= d.ny ? y - d.ny : y);
    z = z < 0 ? z + d.nz : (z >= d.nz ? z - d.nz : z);
    return ((long long)z * d.ny + y) * d.nx + x;
}

// Plane indices of the 3 x 3 x 3 neighbourhood of node (x, y, z), wrapped
// periodically: node (x + dx, y + dy, z + dz) is at yz[dz + 1][dy + 1] +
// xs[dx + 1].  A non-periodic direction has solid boundary planes (checked at
// create), so a fluid node's pulls and force stencil never cross them; the
// wrap is then never taken there.  Index type I: 32-bit unsigned when every
// offset into the population buffers (2 x 19 planes) stays below 2^32, so
// that an address is one multiply-add; 64-bit otherwise.
template <typename I>
struct Hood {
    I xs[3];
    I yz[3][3];
    __device__ __forceinline__ void init(const Dims& d, int x, int y, int z) {
        xs[0] = x == 0 ? d.nx - 1 : x - 1;
        xs[1] = x;
        xs[2] = x == d.nx - 1 ? 0 : x + 1;
        const int ys[3] = {y == 0 ? d.ny - 1 : y - 1, y, y == d.ny - 1 ? 0 : y + 1};
        const int zs[3] = {z == 0 ? d.nz - 1 : z - 1, z, z == d.nz - 1 ? 0 : z + 1};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) yz[a][b] = ((I)zs[a] * (I)d.ny + (I)ys[b]) * (I)d.nx;
    }
    __device__ __forceinline__ I at(int dx, int dy, int dz) const { return yz[dz + 1][dy + 1] + xs[dx + 1]; }
};

// The 38 pulled populations of node k with link word lk and neighbourhood h.
template <typename R, typename I>
__device__ __forceinline__ void pull3(const R* __restrict__ f, I n, I k, const Hood<I>& h, unsigned lk,
                                      R (&fl)[2][kQ]) {
    const R* __restrict__ g = f + (size_t)kQ * n;   // species w
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const bool bb = (lk >> i) & 1u;
        // a bounced population is the node's own one of the opposite direction
        const I src = bb ? k + (I)opp3(i) * n : h.at(-cx3(i), -cy3(i), -cz3(i)) + (I)i * n;
        fl[0][i] = __ldg(f + src);
        fl[1][i] = __ldg(g + src);
    }
}

// Both passes run over the fluid nodes only: thread t takes entry t of the
// fluid list (x fastest, so neighbouring threads hold neighbouring x and
// every population plane is still read and written coalesced); a node's
// coordinates are packed as x | y << 16 | z << 32 ... in 64 bits:
// x in bits 0..20, y in 21..41, z in 42..62.
template <typename I>
__device__ __forceinline__ bool node_of(const Dims& d, const unsigned long long* __restrict__ fluid,
                                        long long nfluid, int& x, int& y, int& z, I& k) {
    const long long t = (long long)blockIdx.x * kT + threadIdx.x;
    if (t >= nfluid) return false;
    const unsigned long long c = fluid[t];
    x = (int)(c & 0x1FFFFFull);
    y = (int)((c >> 21) & 0x1FFFFFull);
    z = (int)((c >> 42) & 0x1FFFFFull);
    k = ((I)z * (I)d.ny + (I)y) * (I)d.nx + (I)x;
    return true;
}

// Densities of the fluid nodes (the solid nodes' entries hold the wall
// potentials, written once at set-up).
template <typename R, typename I>
__global__ void __launch_bounds__(kT) density3_kernel(const R* __restrict__ f, const unsigned* __restrict__ links,
                                                      R* __restrict__ rho, Dims d,
                                                      const unsigned long long* __restrict__ fluid, long long nfluid) {
    int x, y, z;
    I k;
    if (!node_of(d, fluid, nfluid, x, y, z, k)) return;
    const I n = (I)d.n;
    const unsigned lk = links[k];
    Hood<I> hd;
    hd.init(d, x, y, z);
    R fl[2][kQ];
    pull3<R, I>(f, n, k, hd, lk, fl);
    R a = R(0), b = R(0);
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        a += fl[0][i];
        b += fl[1][i];
    }
    rho[k] = a;
    rho[n + k] = b;
}

// The sums of the collision written out over the nonzero terms of the
// velocity set (a product with a zero velocity component is not an exact
// no-op in IEEE arithmetic, so the compiler keeps it; these forms skip them).
// Opposite directions 2k - 1 and 2k share the even part of the equilibrium.

// Moments of one species: density and momentum, sum_i c_i f_i.
template <typename R>
__host__ __device__ __forceinline__ void moments3(const R (&f)[kQ], R& rho, R& jx, R& jy, R& jz) {
    R s = f[0];
#pragma unroll
    for (int i = 1; i < kQ; i++) s += f[i];
    rho = s;
    jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    jy = (f[3] - f[4]) + (f[7] - f[8]) + (f[10] - f[9]) + (f[15] - f[16]) + (f[17] - f[18]);
    jz = (f[5] - f[6]) + (f[11] - f[12]) + (f[14] - f[13]) + (f[15] - f[16]) + (f[18] - f[17]);
}

// sum_i w_i c_i r_i over the eighteen moving directions (r_i = rho^b at
// x + c_i, index i - 1 in nb).
template <typename R>
__host__ __device__ __forceinline__ void stencil3(const R (&nb)[kQ - 1], R& sx, R& sy, R& sz) {
    auto r = [&](int i) { return nb[i - 1]; };
    const R w1 = R(1.0 / 18.0), w2 = R(1.0 / 36.0);
    sx = w1 * (r(1) - r(2)) + w2 * ((r(7) - r(8)) + (r(9) - r(10)) + (r(11) - r(12)) + (r(13) - r(14)));
    sy = w1 * (r(3) - r(4)) + w2 * ((r(7) - r(8)) + (r(10) - r(9)) + (r(15) - r(16)) + (r(17) - r(18)));
    sz = w1 * (r(5) - r(6)) + w2 * ((r(11) - r(12)) + (r(14) - r(13)) + (r(15) - r(16)) + (r(18) - r(17)));
}

// Eq. (feq) deviation from rest, D_i = E_i + O_i with E = -1.5 u^2 +
// 4.5 (c.u)^2 and O = (c.u) (3 - k3 u^2 + k3 (c.u)^2) (T0 = 1/3), for all
// nineteen directions.
template <typename R>
__host__ __device__ __forceinline__ void dev3_all(R ux, R uy, R uz, R k3, R (&D)[kQ]) {
    const R uu = ux * ux + uy * uy + uz * uz;
    const R m = R(-1.5) * uu;
    const R B = R(3) - k3 * uu;
    D[0] = m;
    const R cu[9] = {ux, uy, uz, ux + uy, ux - uy, ux + uz, ux - uz, uy + uz, uy - uz};
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const R c = cu[k], c2 = c * c;
        const R e = R(4.5) * c2 + m;
        const R o = c * (B + k3 * c2);
        D[2 * k + 1] = e + o;
        D[2 * k + 2] = e - o;
    }
}

// Eq. (Regualize) on D3Q19: f'_i = w_i / (2 T0^2) Q_i : Pi with Q_i = c_i c_i -
// T0 I and Pi = sum_j c_j c_j f'_j, over the nonzero entries of c_j c_j.
template <typename R>
__host__ __device__ __forceinline__ void regularize3(R (&fn)[kQ]) {
    const R pxx = (fn[1] + fn[2]) + ((fn[7] + fn[8]) + (fn[9] + fn[10])) + ((fn[11] + fn[12]) + (fn[13] + fn[14]));
    const R pyy = (fn[3] + fn[4]) + ((fn[7] + fn[8]) + (fn[9] + fn[10])) + ((fn[15] + fn[16]) + (fn[17] + fn[18]));
    const R pzz = (fn[5] + fn[6]) + ((fn[11] + fn[12]) + (fn[13] + fn[14])) + ((fn[15] + fn[16]) + (fn[17] + fn[18]));
    const R pxy = (fn[7] + fn[8]) - (fn[9] + fn[10]);
    const R pxz = (fn[11] + fn[12]) - (fn[13] + fn[14]);
    const R pyz = (fn[15] + fn[16]) - (fn[17] + fn[18]);
    const R t3 = R(1.0 / 3.0) * (pxx + pyy + pzz);
    const R a1 = R(4.5) * w3<R>(1), a7 = R(4.5) * w3<R>(7);
    fn[0] = R(4.5) * w3<R>(0) * (-t3);
    fn[1] = fn[2] = a1 * (pxx - t3);
    fn[3] = fn[4] = a1 * (pyy - t3);
    fn[5] = fn[6] = a1 * (pzz - t3);
    fn[7] = fn[8] = a7 * (pxx + pyy + R(2) * pxy - t3);
    fn[9] = fn[10] = a7 * (pxx + pyy - R(2) * pxy - t3);
    fn[11] = fn[12] = a7 * (pxx + pzz + R(2) * pxz - t3);
    fn[13] = fn[14] = a7 * (pxx + pzz - R(2) * pxz - t3);
    fn[15] = fn[16] = a7 * (pyy + pzz + R(2) * pyz - t3);
    fn[17] = fn[18] = a7 * (pyy + pzz - R(2) * pyz - t3);
}

// Launch parameters in the arithmetic type (the FP64 block converted once at
// set-up, so that no thread converts them).
template <typename R>
struct Coef3 {
    R nu[2], G, g[3], k3;
    int reg;
};

template <typename R, typename I>
__global__ void __launch_bounds__(kT, sizeof(R) == 4 ? 5 : 3) collide3_kernel(const R* __restrict__ f, R* __restrict__ fo,
                                                      const unsigned* __restrict__ links, const R* __restrict__ rho,
                                                      Dims d, const Coef3<R> cf, ObsAccum* __restrict__ acc,
                                                      ObsState* __restrict__ obs, double* __restrict__ fields,
                                                      const unsigned long long* __restrict__ fluid, long long nfluid) {
    int x, y, z;
    I k;
    const bool live = node_of(d, fluid, nfluid, x, y, z, k);
    const I n = (I)d.n;
    ObsLocal<R> ob;
    if (live) {
        const unsigned lk = links[k];
        Hood<I> hd;
        hd.init(d, x, y, z);
        R fl[2][kQ];
        pull3<R, I>(f, n, k, hd, lk, fl);
        R r[2], j[2][3];
#pragma unroll
        for (int a = 0; a < 2; a++) moments3<R>(fl[a], r[a], j[a][0], j[a][1], j[a][2]);
        // F^a/rho^a = G sum_i w_i c_i rho^b(x + c_i) + g
        R sb[2][3];
        {
            R nbo[kQ - 1], nbw[kQ - 1];
#pragma unroll
            for (int i = 1; i < kQ; i++) {
                const I nb = hd.at(cx3(i), cy3(i), cz3(i));
                nbo[i - 1] = rho[nb];
                nbw[i - 1] = rho[n + nb];
            }
            stencil3<R>(nbo, sb[0][0], sb[0][1], sb[0][2]);
            stencil3<R>(nbw, sb[1][0], sb[1][1], sb[1][2]);
        }
        R acc3[2][3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            acc3[0][q] = cf.G * sb[1][q] + cf.g[q];   // species o feels rho^w
            acc3[1][q] = cf.G * sb[0][q] + cf.g[q];   // species w feels rho^o
        }
        const R rt = r[0] + r[1];
        const R inv = R(1) / rt;
        R u[3];
#pragma unroll
        for (int q = 0; q < 3; q++) u[q] = (j[0][q] + j[1][q]) * inv;
        if (fields) {
            fields[k] = double(r[0]);
            fields[n + k] = double(r[1]);
#pragma unroll
            for (int q = 0; q < 3; q++)
                fields[(2 + q) * n + k] = double(u[q] + R(0.5) * (r[0] * acc3[0][q] + r[1] * acc3[1][q]) * inv);
        } else {
            const R nu_mix = (r[0] * cf.nu[0] + r[1] * cf.nu[1]) * inv;
            const R om1 = R(1) - R(1) / (R(3) * nu_mix + R(0.5));
            R Du[kQ];
            dev3_all<R>(u[0], u[1], u[2], cf.k3, Du);
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const R rho_a = r[a];
                R fn[kQ];
#pragma unroll
                for (int i = 0; i < kQ; i++) {
                    const R wr = w3<R>(i) * rho_a;
                    fn[i] = (fl[a][i] - wr) - wr * Du[i];
                }
                if (cf.reg) regularize3<R>(fn);
                R Ds[kQ];
                dev3_all<R>(u[0] + acc3[a][0], u[1] + acc3[a][1], u[2] + acc3[a][2], cf.k3, Ds);
                R out[kQ];
                R rest = rho_a;
#pragma unroll
                for (int i = 1; i < kQ; i++) {
                    const R wr = w3<R>(i) * rho_a;
                    out[i] = wr + (wr * Ds[i] + om1 * fn[i]);
                    rest -= out[i];
                }
                out[0] = rest;   // the f*_i of a node sum to rho for both forms of f'
#pragma unroll
                for (int i = 0; i < kQ; i++) fo[(I)(a * kQ + i) * n + k] = out[i];
            }
            ob.m0 += r[0];
            ob.m1 += r[1];
            ob.px += j[0][0] + R(0.5) * r[0] * acc3[0][0];
            R v2 = R(0);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const R vq = u[q] + R(0.5) * (r[0] * acc3[0][q] + r[1] * acc3[1][q]) * inv;
                v2 += vq * vq;
            }
            ob.umax2 = fmax(ob.umax2, v2);
            ob.bad = ob.bad || !(r[0] >= R(0) && r[1] >= R(0));
        }
    }
    if (fields) return;
    reduce_observables<R, kT>(ob, acc, obs, false, gridDim.x);
}

// The wall potentials into the density field at solid nodes (set-up), and
// the fields of solid nodes (rho_s, zero velocity).
template <typename R>
__global__ void solid_density3_kernel(const unsigned* __restrict__ links, R* __restrict__ rho, Dims d,
                                      const Params3* __restrict__ p, double* __restrict__ fields) {
    const long long k = (long long)blockIdx.x * kT + threadIdx.x;
    if (k >= d.n || !(links[k] & kSolid3)) return;
    if (fields) {
        const long long n = d.n;
        fields[k] = p->rho_wall[0];
        fields[n + k] = p->rho_wall[1];
        fields[2 * n + k] = fields[3 * n + k] = fields[4 * n + k] = 0.0;
        return;
    }
    rho[k] = R(p->rho_wall[0]);
    rho[d.n + k] = R(p->rho_wall[1]);
}

__global__ void links3_kernel(const uint8_t* __restrict__ mask, unsigned* __restrict__ links, Dims d) {
    const long long k = (long long)blockIdx.x * kT + threadIdx.x;
    if (k >= d.n) return;
    const int x = (int)(k % d.nx), y = (int)((k / d.nx) % d.ny), z = (int)(k / ((long long)d.nx * d.ny));
    unsigned w = mask[k] ? kSolid3 : 0u;
    for (int i = 1; i < kQ; i++)
        if (mask[wrapped(d, x - cx3(i), y - cy3(i), z - cz3(i))]) w |= 1u << i;
    links[k] = w;
}

thread_local std::string g_err3;

int fail3(lbm3d_t* h, int code, const char* fmt, ...);

}  // namespace

struct lbm3d_t {
    lbm3d_params p{};
    Dims d{};
    size_t es = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    unsigned* links = nullptr;
    void* rho = nullptr;
    unsigned long long* fluid = nullptr;   // packed coordinates of the fluid nodes, x fastest
    long long nfluid = 0;
    Params3* dprm = nullptr;
    Params3 hp{};                          // host copy of the parameter block
    ObsAccum* dacc = nullptr;
    ObsState* dobs = nullptr;
    std::vector<uint8_t> mask;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

int fail3(lbm3d_t* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_err3 = buf;
    return code;
}

#define TRY3(h, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail3((h), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

unsigned blocks_of(long long n) { return (unsigned)((n + kT - 1) / kT); }

template <typename R>
Coef3<R> coef_of(const Params3& p) {
    Coef3<R> c;
    for (int a = 0; a < 2; a++) c.nu[a] = R(p.nu[a]);
    c.G = R(p.G);
    for (int q = 0; q < 3; q++) c.g[q] = R(p.g[q]);
    c.k3 = R(p.k3);
    c.reg = p.reg != 0.0;
    return c;
}

template <typename R, typename I>
cudaError_t step3_idx(lbm3d_t* h, double* fields) {
    const R* fin = (const R*)h->f[h->cur];
    if (fields) solid_density3_kernel<R><<<blocks_of(h->d.n), kT, 0, h->stream>>>(h->links, nullptr, h->d, h->dprm, fields);
    // one block at least: without fluid the collide pass still closes the
    // step's observables
    const unsigned grid = std::max(1u, blocks_of(h->nfluid));
    if (h->nfluid > 0)
        density3_kernel<R, I><<<grid, kT, 0, h->stream>>>(fin, h->links, (R*)h->rho, h->d, h->fluid, h->nfluid);
    collide3_kernel<R, I><<<grid, kT, 0, h->stream>>>(fin, (R*)h->f[1 - h->cur], h->links, (const R*)h->rho, h->d,
                                                      coef_of<R>(h->hp), h->dacc, h->dobs, fields, h->fluid,
                                                      h->nfluid);
    return cudaGetLastError();
}

// 32-bit offsets when all 2 x 19 population planes plus one more (the
// density field's second plane, the fields' five) stay below 2^32 elements;
// GB300LBM_INDEX64=1 takes the 64-bit kernels on any grid (the tests compare
// both).
template <typename R>
cudaError_t step3(lbm3d_t* h, double* fields) {
    const char* e = getenv("GB300LBM_INDEX64");
    const bool force64 = e && e[0] == '1';
    if (!force64 && (unsigned long long)h->d.n * (2 * kQ + 1) < (1ull << 32)) return step3_idx<R, unsigned>(h, fields);
    return step3_idx<R, unsigned long long>(h, fields);
}

cudaError_t init_solid_density(lbm3d_t* h) {
    if (h->p.precision == LBM_FP64)
        solid_density3_kernel<double><<<blocks_of(h->d.n), kT, 0, h->stream>>>(h->links, (double*)h->rho, h->d, h->dprm, nullptr);
    else
        solid_density3_kernel<float><<<blocks_of(h->d.n), kT, 0, h->stream>>>(h->links, (float*)h->rho, h->d, h->dprm, nullptr);
    return cudaGetLastError();
}

cudaError_t step_any(lbm3d_t* h, double* fields) {
    return h->p.precision == LBM_FP64 ? step3<double>(h, fields) : step3<float>(h, fields);
}

}  // namespace

extern "C" {

int lbm3d_create(const uint8_t* mask, const double* rho_init, const lbm3d_params* p, lbm3d_t** out) {
    if (!out) return fail3(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mask || !rho_init || !p) return fail3(nullptr, LBM_EINVAL, "NULL argument");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail3(nullptr, LBM_EINVAL, "nx, ny, nz must be >= 1");
    if (p->nx > (1 << 21) || p->ny > (1 << 21) || p->nz > (1 << 21))
        return fail3(nullptr, LBM_EINVAL, "nx, ny, nz must be <= 2^21");
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n * 2 * kQ >= (1LL << 40)) return fail3(nullptr, LBM_EINVAL, "grid too large");
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32)
        return fail3(nullptr, LBM_EINVAL, "precision must be LBM_FP64 or LBM_FP32");
    if (p->eq_order != 2 && p->eq_order != 3) return fail3(nullptr, LBM_EINVAL, "eq_order must be 2 or 3");
    if (p->collision != 0 && p->collision != 1) return fail3(nullptr, LBM_EINVAL, "collision must be 0 or 1");
    for (int a = 0; a < 2; a++)
        if (!(p->tau[a] > 0.5) || !std::isfinite(p->tau[a]))
            return fail3(nullptr, LBM_EINVAL, "tau[%d] must be finite and exceed 1/2", a);
    if (!std::isfinite(p->G) || !std::isfinite(p->rho_wall[0]) || !std::isfinite(p->rho_wall[1]) ||
        !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]) || !std::isfinite(p->g[2]))
        return fail3(nullptr, LBM_EINVAL, "G, g and rho_wall must be finite");
    const int dims[3] = {p->nx, p->ny, p->nz};
    for (int q = 0; q < 3; q++) {
        if (p->periodic[q]) continue;
        for (long long k = 0; k < n; k++) {
            const int c[3] = {(int)(k % p->nx), (int)((k / p->nx) % p->ny), (int)(k / ((long long)p->nx * p->ny))};
            if ((c[q] == 0 || c[q] == dims[q] - 1) && !mask[k])
                return fail3(nullptr, LBM_EINVAL, "direction %d is not periodic but its boundary plane has fluid", q);
        }
    }
    for (long long k = 0; k < n; k++) {
        if (mask[k]) continue;
        const double a = rho_init[k], b = rho_init[n + k];
        if (!std::isfinite(a) || !std::isfinite(b) || a < 0.0 || b < 0.0 || a + b <= 0.0)
            return fail3(nullptr, LBM_EINVAL, "rho_init at fluid node %lld is not finite, negative or zero", k);
    }
    lbm3d_t* h = new lbm3d_t;
    h->p = *p;
    h->d = Dims{p->nx, p->ny, p->nz, n};
    h->es = p->precision == LBM_FP64 ? 8 : 4;
    h->stream = (cudaStream_t)p->cuda_stream;
    h->mask.assign(mask, mask + n);
    auto bail = [&](int rc) {
        lbm3d_destroy(h);
        return rc;
    };
    const size_t fbytes = (size_t)n * 2 * kQ * h->es;
    for (int b = 0; b < 2; b++)
        if (cudaMalloc(&h->f[b], fbytes) != cudaSuccess) return bail(fail3(nullptr, LBM_ENOMEM, "populations"));
    if (cudaMalloc((void**)&h->links, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&h->rho, (size_t)n * 2 * h->es) != cudaSuccess ||
        cudaMalloc((void**)&h->dprm, sizeof(Params3)) != cudaSuccess ||
        cudaMalloc((void**)&h->dacc, sizeof(ObsAccum)) != cudaSuccess ||
        cudaMalloc((void**)&h->dobs, sizeof(ObsState)) != cudaSuccess)
        return bail(fail3(nullptr, LBM_ENOMEM, "device memory"));
    Params3 hp{};
    for (int a = 0; a < 2; a++) {
        hp.nu[a] = (p->tau[a] - 0.5) / 3.0;
        hp.rho_wall[a] = p->rho_wall[a];
    }
    for (int q = 0; q < 3; q++) hp.g[q] = p->g[q];
    hp.G = p->G;
    hp.k3 = p->eq_order >= 3 ? 4.5 : 0.0;
    hp.reg = p->collision == 1 ? 1.0 : 0.0;
    uint8_t* dmask = nullptr;
    if (cudaMalloc((void**)&dmask, (size_t)n) != cudaSuccess) return bail(fail3(nullptr, LBM_ENOMEM, "mask"));
    cudaError_t e = cudaMemcpyAsync(dmask, mask, (size_t)n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        links3_kernel<<<blocks_of(n), kT, 0, h->stream>>>(dmask, h->links, h->d);
        e = cudaGetLastError();
    }
    h->hp = hp;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dprm, &hp, sizeof hp, cudaMemcpyHostToDevice, h->stream);
    // the fluid list (x fastest) and the wall potentials of the solid nodes
    std::vector<unsigned long long> fl;
    for (long long k = 0; k < n; k++)
        if (!mask[k]) {
            const unsigned long long x = (unsigned long long)(k % p->nx), y = (unsigned long long)((k / p->nx) % p->ny),
                                     z = (unsigned long long)(k / ((long long)p->nx * p->ny));
            fl.push_back(x | (y << 21) | (z << 42));
        }
    h->nfluid = (long long)fl.size();
    if (e == cudaSuccess && h->nfluid > 0) {
        e = cudaMalloc((void**)&h->fluid, fl.size() * sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->fluid, fl.data(), fl.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                h->stream);
    }
    if (e == cudaSuccess) e = init_solid_density(h);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dacc, 0, sizeof(ObsAccum), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dobs, 0, sizeof(ObsState), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dmask);
    if (e != cudaSuccess) return bail(fail3(nullptr, LBM_ECUDA, "set-up: %s", cudaGetErrorString(e)));
    // initial state f*_i = w_i rho_init at fluid nodes
    std::vector<double> f((size_t)n * 2 * kQ);
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < kQ; i++)
            for (long long k = 0; k < n; k++)
                f[(size_t)(a * kQ + i) * n + k] = mask[k] ? 0.0 : w3<double>(i) * rho_init[(size_t)a * n + k];
    const int rc = lbm3d_load(h, f.data());
    if (rc) {
        g_err3 = h->err;
        return bail(rc);
    }
    *out = h;
    return LBM_OK;
}

int lbm3d_step(lbm3d_t* h, int64_t nsteps) {
    if (!h || nsteps < 0) return fail3(h, LBM_EINVAL, "bad argument");
    for (int64_t s = 0; s < nsteps; s++) {
        TRY3(h, step_any(h, nullptr));
        h->cur = 1 - h->cur;
    }
    return LBM_OK;
}

int lbm3d_observables(lbm3d_t* h, lbm_obs* out) {
    if (!h || !out) return fail3(h, LBM_EINVAL, "NULL argument");
    ObsState s{};
    TRY3(h, cudaMemcpyAsync(&s, h->dobs, sizeof s, cudaMemcpyDeviceToHost, h->stream));
    TRY3(h, cudaStreamSynchronize(h->stream));
    out->mass[0] = s.mass[0];
    out->mass[1] = s.mass[1];
    out->oil_mom_x = s.px;
    out->oil_disp_x = s.disp;
    out->max_u = s.umax;
    out->step = s.step;
    out->nan_flag = s.nan_flag;
    out->timeout_flag = s.timeout_flag;
    if (s.nan_flag) return fail3(h, LBM_EUNSTABLE, "a fluid node reached a NaN or negative density");
    return LBM_OK;
}

int lbm3d_save(lbm3d_t* h, double* f) {
    if (!h || !f) return fail3(h, LBM_EINVAL, "NULL argument");
    const size_t len = (size_t)h->d.n * 2 * kQ;
    std::vector<char> raw(len * h->es);
    TRY3(h, cudaMemcpyAsync(raw.data(), h->f[h->cur], raw.size(), cudaMemcpyDeviceToHost, h->stream));
    TRY3(h, cudaStreamSynchronize(h->stream));
    for (size_t q = 0; q < len; q++)
        f[q] = h->es == 8 ? ((const double*)raw.data())[q] : (double)((const float*)raw.data())[q];
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < kQ; i++)
            for (long long k = 0; k < h->d.n; k++)
                if (h->mask[k]) f[(size_t)(a * kQ + i) * h->d.n + k] = 0.0;
    return LBM_OK;
}

int lbm3d_load(lbm3d_t* h, const double* f) {
    if (!h || !f) return fail3(h, LBM_EINVAL, "NULL argument");
    const size_t len = (size_t)h->d.n * 2 * kQ;
    std::vector<char> raw(len * h->es);
    for (size_t q = 0; q < len; q++) {
        const long long k = (long long)(q % (size_t)h->d.n);
        const double v = h->mask[k] ? 0.0 : f[q];
        if (h->es == 8) ((double*)raw.data())[q] = v;
        else ((float*)raw.data())[q] = (float)v;
    }
    TRY3(h, cudaMemcpyAsync(h->f[h->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice, h->stream));
    TRY3(h, cudaMemsetAsync(h->dacc, 0, sizeof(ObsAccum), h->stream));
    TRY3(h, cudaMemsetAsync(h->dobs, 0, sizeof(ObsState), h->stream));
    TRY3(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm3d_get_fields(lbm3d_t* h, double* rho, double* u) {
    if (!h) return fail3(h, LBM_EINVAL, "NULL handle");
    const long long n = h->d.n;
    double* dfields = nullptr;
    TRY3(h, cudaMalloc((void**)&dfields, sizeof(double) * 5 * (size_t)n));
    cudaError_t e = step_any(h, dfields);
    std::vector<double> hf((size_t)5 * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), dfields, hf.size() * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dfields);
    if (e != cudaSuccess) return fail3(h, LBM_ECUDA, "fields: %s", cudaGetErrorString(e));
    if (rho) std::memcpy(rho, hf.data(), sizeof(double) * 2 * n);
    if (u) std::memcpy(u, hf.data() + 2 * n, sizeof(double) * 3 * n);
    return LBM_OK;
}

void lbm3d_destroy(lbm3d_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->f[0]);
    cudaFree(h->f[1]);
    cudaFree(h->links);
    cudaFree(h->rho);
    cudaFree(h->fluid);
    cudaFree(h->dprm);
    cudaFree(h->dacc);
    cudaFree(h->dobs);
    delete h;
}

const char* lbm3d_last_error(const lbm3d_t* h) { return h ? h->err.c_str() : g_err3.c_str(); }

}  // extern "C"
