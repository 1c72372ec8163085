// Device code shared by the step kernels: storage codecs, the D2Q9 lattice,
// the equilibrium of Eq. (feq), the per-node force + collision, and the
// per-step observables reduction.
//
// Storage layout (every population plane and the link-word plane):
//   element (x, y) of a plane lives at  y * pitch + kGhost + x,
// for logical columns x in [-kGhost, nx + kGhost).  Columns -2, -1, nx, nx + 1
// are "ghost" copies of nx - 2, nx - 1, 0, 1 when x is periodic (written by
// the step that writes the original column), so a row window
// [x0 - kGhost, x0 + BX + kGhost) never needs a wrap-around patch; this is
// what lets a single TMA box stage a row.  pitch >= nx + 2 kGhost, rounded up
// to 32 elements, so every row starts 128-byte aligned.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gb300lbm {

constexpr int kGhost = 8;       // ghost columns on each side (16-byte aligned for 2-byte types)
constexpr int kSolidBit = 15;   // link word: bit i (1..8) = pull source x - c_i is solid

// Device-resident parameters (read each launch, so captured graphs follow
// lbm_set_body_force).
struct StepParams {
    double nu[2];        // nu^a = T0 (tau^a - 1/2)
    double G;
    double g[2];
    double rho_wall[2];
    double k3;           // 4.5 with the cubic terms of Eq. (feq), 0 without
    double reg;          // 1: regularised non-equilibrium part (Eq. Regualize), 0: plain BGK
};

// Per-step reduction targets; reset by the last CTA of each step.
struct ObsAccum {
    double mass[2];
    double px;
    unsigned long long umax2_bits;
    unsigned int bad;
    unsigned int blocks_done;
};

// Observables as of the latest step (host-visible copy in lbm_obs).
struct ObsState {
    double mass[2];
    double px;
    double disp;
    double umax;
    long long step;
    int nan_flag;
    int timeout_flag;    // a bounded device wait gave up (data of that step invalid)
};

struct Grid {
    int nx, ny, pitch;
    int periodic_x;
    int rows_per_block;   // simple kernel: rows per CTA strip
    int row_begin;        // first row handled by blockIdx.y == 0 (fields windows)
    int row_end;          // one past the last row handled by this launch
    int strips;           // staged kernel: strips per column block (gridDim.y)
    int strip_rows;       // staged kernel: > 0: strip s holds the block's fluid rows among the
                          // absolute rows [s strip_rows, (s + 1) strip_rows); 0: the block's
                          // fluid rows split into `strips` equal parts
};

// FP32 storage stepped with the compensated FP32 arithmetic (Codec<f32c>):
// the same four bytes as a float, a distinct type so that every kernel
// template can be instantiated for it.
struct f32c {
    float v;
    f32c() = default;
    __host__ __device__ constexpr f32c(float x) : v(x) {}
    __host__ __device__ constexpr operator float() const { return v; }
};
static_assert(sizeof(f32c) == 4 && alignof(f32c) == 4, "f32c must be laid out as a float");

using ::__ldg;
using ::__ldcg;
__device__ __forceinline__ f32c __ldg(const f32c* p) { return f32c(::__ldg(reinterpret_cast<const float*>(p))); }
__device__ __forceinline__ f32c __ldcg(const f32c* p) { return f32c(::__ldcg(reinterpret_cast<const float*>(p))); }

// Population load of a march: through the read-only cache (kCoherent =
// false: the buffer is not written during the launch), or cached in L2 only
// (kCoherent = true: a persistent launch writes in one step the buffer it
// reads in the next, and L1 is not kept coherent with other SMs' writes).
template <bool kCoherent, typename S>
__device__ __forceinline__ S load_pop(const S* p) {
    if constexpr (kCoherent) return __ldcg(p);
    else return __ldg(p);
}

// ---------------------------------------------------------------------------
// storage codecs
//
// FP64 / FP32 store f_i as is (18 planes).  The 16-bit formats store
//   s_i(x) = f*_i(x) - w_i rhohat^a(x)
// where rhohat^a(x) is the writer node's own density rounded to the 16-bit
// format and kept in two extra planes (18: species o, 19: species w).  The
// reader of a population pulled from node x - c_i adds back w_i rhohat^a of
// that source node, which it reads from the same planes, so the shift is
// exact and only the small non-equilibrium part s_i is rounded to 16 bits.
// ---------------------------------------------------------------------------
template <typename S>
struct Codec;

template <>
struct Codec<double> {
    using R = double;
    static constexpr bool kNodeShift = false;
    static constexpr bool kCompensated = false;
    static constexpr int kPlanes = 18;
    static __device__ __forceinline__ double decode(double v, double, double) { return v; }
    static __device__ __forceinline__ double encode(double v, double, double) { return v; }
    static __device__ __forceinline__ double pack(double v) { return v; }
    static __device__ __forceinline__ double rho_store(double r) { return r; }
    static __device__ __forceinline__ double rho_value(double s) { return s; }
};

template <>
struct Codec<float> {
    using R = float;
    static constexpr bool kNodeShift = false;
    static constexpr bool kCompensated = false;
    static constexpr int kPlanes = 18;
    static __device__ __forceinline__ float decode(float v, float, float) { return v; }
    static __device__ __forceinline__ float encode(float v, float, float) { return v; }
    static __device__ __forceinline__ float pack(float v) { return v; }
    static __device__ __forceinline__ float rho_store(float r) { return r; }
    static __device__ __forceinline__ float rho_value(float s) { return s; }
};

template <>
struct Codec<__half> {
    using R = float;
    static constexpr bool kNodeShift = true;
    static constexpr bool kCompensated = false;
    static constexpr int kPlanes = 20;
    // f = s + w rhohat and s = f - w rhohat, each one fused multiply-add
    static __device__ __forceinline__ float decode(__half v, float w, float rh) {
        return __fmaf_rn(w, rh, __half2float(v));
    }
    static __device__ __forceinline__ __half encode(float v, float w, float rh) {
        return __float2half_rn(__fmaf_rn(-w, rh, v));
    }
    static __device__ __forceinline__ __half pack(float s) { return __float2half_rn(s); }
    static __device__ __forceinline__ __half rho_store(float r) { return __float2half_rn(r); }
    static __device__ __forceinline__ float rho_value(__half s) { return __half2float(s); }
};

template <>
struct Codec<__nv_bfloat16> {
    using R = float;
    static constexpr bool kNodeShift = true;
    static constexpr bool kCompensated = false;
    static constexpr int kPlanes = 20;
    static __device__ __forceinline__ float decode(__nv_bfloat16 v, float w, float rh) {
        return __fmaf_rn(w, rh, __bfloat162float(v));
    }
    static __device__ __forceinline__ __nv_bfloat16 encode(float v, float w, float rh) {
        return __float2bfloat16_rn(__fmaf_rn(-w, rh, v));
    }
    static __device__ __forceinline__ __nv_bfloat16 pack(float s) { return __float2bfloat16_rn(s); }
    static __device__ __forceinline__ __nv_bfloat16 rho_store(float r) { return __float2bfloat16_rn(r); }
    static __device__ __forceinline__ float rho_value(__nv_bfloat16 s) { return __bfloat162float(s); }
};

// FP32 storage, compensated FP32 arithmetic.  Plain FP32 arithmetic leaves a
// velocity error several times the one that FP32 storage alone causes
// (rounding of the stored populations with exact arithmetic): the two stages
// that set it are the density sums (several roundings of a sum of nine
// values) and the composition f*_i = w_i rho + t_i (the rounding of w_i rho,
// of the FP32 weights themselves, and of the closure of the rest
// population).  This codec makes those two stages accurate with
// error-free transformations in FP32 (Dekker's Fast2Sum and the FMA form of
// TwoProduct): rho is carried as an unevaluated sum hi + lo, w_i rho as
// wh + wl with the weights' own FP32 rounding folded into wl, and each
// stored population is rounded once from wh + (t_i + wl (1 + D_i)).  The
// rest of the step (force, moments, equilibria) stays plain FP32.
template <>
struct Codec<f32c> {
    using R = float;
    static constexpr bool kNodeShift = false;
    static constexpr bool kCompensated = true;
    static constexpr int kPlanes = 18;
    static __device__ __forceinline__ float decode(f32c v, float, float) { return v.v; }
    static __device__ __forceinline__ f32c encode(float v, float, float) { return f32c(v); }
    static __device__ __forceinline__ f32c pack(float v) { return f32c(v); }
    static __device__ __forceinline__ f32c rho_store(float r) { return f32c(r); }
    static __device__ __forceinline__ float rho_value(f32c s) { return s.v; }
};

// D2Q9, textbook order: c_0 = (0,0); c_1..c_4 = (1,0),(0,1),(-1,0),(0,-1);
// c_5..c_8 = (1,1),(-1,1),(-1,-1),(1,-1).  opp = {0,3,4,1,2,7,8,5,6}.
__host__ __device__ __forceinline__ int d2q9_cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ int d2q9_cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ __forceinline__ int d2q9_opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}

template <typename R>
__host__ __device__ __forceinline__ R weight_of(int i) {
    return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

// Lattice weights in the arithmetic type.  In FP32 the correctly rounded
// values of 4/9, 1/9 and 1/36 sum to 1 + 7.45e-9, which would create mass at
// every node and step (a drift of ~7e-6 relative after 1000 steps); taking
// 1/36 one ulp below its rounded value makes the nine FP32 weights sum to
// exactly 1, so the equilibrium conserves mass in FP32.  FP64 keeps the
// rounded values (their sum is off by < 1e-16).
template <typename R>
struct Weights {
    static __device__ __forceinline__ R w0() { return R(4.0 / 9.0); }
    static __device__ __forceinline__ R w1() { return R(1.0 / 9.0); }
    static __device__ __forceinline__ R w5() { return R(1.0 / 36.0); }
};
template <>
struct Weights<float> {
    static __device__ __forceinline__ float w0() { return __int_as_float(0x3EE38E39); }  // 4/9
    static __device__ __forceinline__ float w1() { return __int_as_float(0x3DE38E39); }  // 1/9
    static __device__ __forceinline__ float w5() { return __int_as_float(0x3CE38E38); }  // 1/36 - 1 ulp
};

// Explicitly rounded FP32 arithmetic: the compiler neither fuses nor
// reorders these operations, so every kernel that runs the collision below
// performs the same operations in the same order and produces the same
// bits.  FP64 leaves the compiler free to fuse (its rounding is far below
// any tolerance, and the FP64 pipe is the bottleneck there).
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return a + b; }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return a - b; }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return a * b; }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return fma(a, b, c); }

// Eq. (feq) with T0 = 1/3 as a deviation from rest,
//   f_i^eq(rho, u) = w_i rho (1 + D_i),  D_i = E_i + O_i,
//   E_i = -1.5 u^2 + 4.5 (c_i.u)^2,  O_i = (c_i.u) (3 - k3 u^2 + k3 (c_i.u)^2),
// k3 = 4.5 for the cubic equilibrium; opposite directions share E and flip
// O.  Keeping the 1 out of D keeps the small part at full relative
// precision in FP32 (the collision adds w_i rho last).
template <typename R>
__device__ __forceinline__ void eq_deviation(R ux, R uy, R k3, R (&D)[9]) {
    const R uu = xfma(ux, ux, xmul(uy, uy));
    const R m = xmul(R(-1.5), uu);
    const R B = xfma(-k3, uu, R(3));
    D[0] = m;
    const R cs[4] = {ux, uy, xadd(ux, uy), xsub(uy, ux)};
    const int ip[4] = {1, 2, 5, 6}, im[4] = {3, 4, 7, 8};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const R c = cs[k], c2 = xmul(c, c);
        const R e = xfma(R(4.5), c2, m);
        const R o = xmul(c, xfma(k3, c2, B));
        D[ip[k]] = xadd(e, o);
        D[im[k]] = xsub(e, o);
    }
}

// The density ring holds (rho^o, rho^w) pairs so one 8- or 16-byte access
// moves both species.
template <typename R>
struct Pair;
template <>
struct Pair<float> {
    using T = float2;
};
template <>
struct Pair<double> {
    using T = double2;
};
template <typename R>
using pair_t = typename Pair<R>::T;

template <typename R>
__device__ __forceinline__ pair_t<R> make_pair_of(R a, R b) {
    pair_t<R> v;
    v.x = a;
    v.y = b;
    return v;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Parameters of one launch in the arithmetic type, loaded once per thread.
template <typename R>
struct NodeParams {
    R G, gx, gy, rw0, rw1, nu0, nu1, k3;
    bool reg;
    __device__ __forceinline__ void load(const StepParams* __restrict__ p) {
        reg = p->reg != 0.0;
        G = R(p->G);
        gx = R(p->g[0]);
        gy = R(p->g[1]);
        rw0 = R(p->rho_wall[0]);
        rw1 = R(p->rho_wall[1]);
        nu0 = R(p->nu[0]);
        nu1 = R(p->nu[1]);
        k3 = R(p->k3);
    }
};

// Weight of direction i in the arithmetic type (the mass-exact set).
template <typename R>
__device__ __forceinline__ R wgt(int i) {
    return i == 0 ? Weights<R>::w0() : (i <= 4 ? Weights<R>::w1() : Weights<R>::w5());
}

__host__ __device__ __forceinline__ int weight_class(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }

// 1/x in the arithmetic type: FP64 divides; FP32 uses the hardware
// approximate reciprocal (__fdividef, a few ulp, no special-case branch),
// since densities and relaxation times are O(1).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }

// rho = sum_i f_i of one species' pulled populations, summed in the order
// i = 0..8.  Plain codecs: one running FP32 (FP64) sum, lo = 0.
// Compensated codec: Dekker's Fast2Sum at every addition (the rest
// population comes first and every population is smaller than the running
// sum, the condition under which each error term is exact), the errors
// accumulated and folded in at the end: hi + lo equals the exact sum to
// about 2^-48 relative, and hi is the sum rounded once.
template <typename C, typename R>
__device__ __forceinline__ void density_of(const R (&f)[9], R& hi, R& lo) {
    if constexpr (C::kCompensated) {
        R s = f[0], e = R(0);
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const R t = xadd(s, f[i]);
            e = xadd(e, xsub(f[i], xsub(t, s)));
            s = t;
        }
        hi = xadd(s, e);
        lo = xsub(e, xsub(hi, s));
    } else {
        R a = R(0);
#pragma unroll
        for (int i = 0; i < 9; i++) a += f[i];
        hi = a;
        lo = R(0);
    }
}

// Sum of v over the 16 lanes of each half-warp (butterfly), the halo
// density of one species.  The compensated codec carries each level's error
// (Knuth's TwoSum, no ordering needed) and returns the sum rounded once, so
// a halo column's density agrees with the one its owner computes.
template <typename C, typename R>
__device__ __forceinline__ R halfwarp_density(R v) {
    if constexpr (C::kCompensated) {
        R s = v, e = R(0);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            const R b = __shfl_xor_sync(0xffffffffu, s, o);
            const R eb = __shfl_xor_sync(0xffffffffu, e, o);
            const R t = xadd(s, b);
            const R bb = xsub(t, s);
            const R err = xadd(xsub(s, xsub(t, bb)), xsub(b, bb));
            e = xadd(xadd(e, eb), err);
            s = t;
        }
        return xadd(s, e);
    } else {
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        return v;
    }
}

// Per-thread observables of one step.
template <typename R>
struct ObsLocal {
    R m0 = R(0), m1 = R(0), px = R(0), umax2 = R(0);
    bool bad = false;
};

// Force, moments and BGK collision at one fluid node, then the store of the
// 18 post-collision populations (and of their periodic ghost images).
//   f[a][i]   pulled populations, rho0/rho1 their sums (density_of), rl0/rl1
//             the low parts of those sums (zero for the plain codecs)
//   nb[b][k]  rho^b at the 8 neighbours x + c_k (k = 1..8 in index k-1)
//   dst       pointer to element (x, y) of plane (species 0, direction 0)
//   x, nx     the node's column and the grid width (ghost images when periodic)
//   kReg      the collision: -1 as P.reg says (read at run time), 0 plain
//             BGK, 1 regularised (fixed at compile time: the other branch is
//             left out of the kernel)
template <typename S, typename R, int kReg = -1>
__device__ __forceinline__ void collide_store(const R (&f)[2][9], R rho0, R rho1, R rl0, R rl1, const R (&nb)[2][8],
                                              const NodeParams<R>& P, S* __restrict__ dst, int plane,
                                              int x, int nx, int periodic, ObsLocal<R>& ob) {
    using C = Codec<S>;
    // sum_i w_i c_i rho^b(x + c_i), neighbours in direction order 1..8
    R sx[2], sy[2];
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const R e = nb[b][0], n = nb[b][1], wv = nb[b][2], so = nb[b][3];
        const R ne = nb[b][4], nw = nb[b][5], sw = nb[b][6], se = nb[b][7];
        sx[b] = xfma(xsub(e, wv), R(1.0 / 9.0), xmul(xadd(xsub(xsub(ne, nw), sw), se), R(1.0 / 36.0)));
        sy[b] = xfma(xsub(n, so), R(1.0 / 9.0), xmul(xsub(xsub(xadd(ne, nw), sw), se), R(1.0 / 36.0)));
    }
    const R ax0 = xfma(P.G, sx[1], P.gx), ay0 = xfma(P.G, sy[1], P.gy);   // species o feels rho^w
    const R ax1 = xfma(P.G, sx[0], P.gx), ay1 = xfma(P.G, sy[0], P.gy);   // species w feels rho^o

    R jx[2], jy[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        jx[a] = xadd(xadd(xsub(f[a][1], f[a][3]), xsub(f[a][5], f[a][7])), xsub(f[a][8], f[a][6]));
        jy[a] = xadd(xadd(xsub(f[a][2], f[a][4]), xsub(f[a][5], f[a][7])), xsub(f[a][6], f[a][8]));
    }
    const R rt = xadd(rho0, rho1);
    const R inv_rt = recip(rt);
    const R ux = xmul(xadd(jx[0], jx[1]), inv_rt);
    const R uy = xmul(xadd(jy[0], jy[1]), inv_rt);
    const R nu_mix = xmul(xfma(rho0, P.nu0, xmul(rho1, P.nu1)), inv_rt);
    const R om1 = xsub(R(1), recip(xfma(R(3), nu_mix, R(0.5))));   // 1 - 1/tau_mix
    R out[2][9];
    // deviation of f^eq(rho^a, u_mix) from rest: the same for both species
    R Du[9];
    eq_deviation<R>(ux, uy, P.k3, Du);
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const R rho = a ? rho1 : rho0;
        const R ax = a ? ax1 : ax0, ay = a ? ay1 : ay0;
        // Eq. (collision_term): equilibrium at the force-shifted velocity
        R Ds[9];
        eq_deviation<R>(xadd(ux, ax), xadd(uy, ay), P.k3, Ds);
        const R wr[3] = {xmul(Weights<R>::w0(), rho), xmul(Weights<R>::w1(), rho), xmul(Weights<R>::w5(), rho)};
        // compensated codec: w_k rho = wr[k] + wl[k] to about 2^-48, the FMA
        // TwoProduct of the FP32 weight and rho_hi, plus the FP32 weight's
        // distance to 4/9, 1/9, 1/36 and rho's low part
        R wl[3] = {R(0), R(0), R(0)};
        if constexpr (C::kCompensated) {
            const R rl = a ? rl1 : rl0;
            const R wf[3] = {Weights<R>::w0(), Weights<R>::w1(), Weights<R>::w5()};
            const R wlo[3] = {R(-0x1.c71c72p-29), R(-0x1.c71c72p-31), R(0x1.c71c72p-30)};
#pragma unroll
            for (int k = 0; k < 3; k++) wl[k] = xfma(wlo[k], rho, xfma(wf[k], rl, xfma(wf[k], rho, -wr[k])));
        }
        S* d = dst + a * 9 * plane;
        R delta = R(0);                                 // 16-bit formats: rho - rhohat
        if (C::kNodeShift) {
            const S q = C::rho_store(rho);
            dst[(18 + a) * plane] = q;
            delta = xsub(rho, C::rho_value(q));
        }
        // non-equilibrium part f' = f - f^eq(rho^a, u_mix) = (f - w rho) - w rho D(u_mix)
        R fn[9];
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const R w = wr[weight_class(i)];
            if constexpr (C::kCompensated)
                fn[i] = xfma(-w, Du[i], xsub(xsub(f[a][i], w), wl[weight_class(i)]));
            else
                fn[i] = xfma(-w, Du[i], xsub(f[a][i], w));
        }
        if (kReg < 0 ? P.reg : kReg == 1) {
            // Eq. (Regualize): f'_i = w_i / (2 T0^2) Q_i : Pi with Q_i = c_i c_i - T0 I
            // and Pi = sum_j c_j c_j f'_j; on D2Q9 with T0 = 1/3 the
            // coefficients reduce to the combinations below (f'_0 is not
            // needed: the rest population is set by mass below)
            const R diag = xadd(xadd(fn[5], fn[6]), xadd(fn[7], fn[8]));
            const R pxx = xadd(xadd(fn[1], fn[3]), diag);
            const R pyy = xadd(xadd(fn[2], fn[4]), diag);
            const R pxy = xsub(xadd(fn[5], fn[7]), xadd(fn[6], fn[8]));
            const R s = xadd(pxx, pyy);
            const R e1 = xfma(R(1.0 / 3.0), pxx, xmul(R(-1.0 / 6.0), pyy));
            const R e2 = xfma(R(1.0 / 3.0), pyy, xmul(R(-1.0 / 6.0), pxx));
            const R dp = xfma(R(1.0 / 12.0), s, xmul(R(0.25), pxy));
            const R dm = xfma(R(1.0 / 12.0), s, xmul(R(-0.25), pxy));
            fn[1] = e1;
            fn[3] = e1;
            fn[2] = e2;
            fn[4] = e2;
            fn[5] = dp;
            fn[7] = dp;
            fn[6] = dm;
            fn[8] = dm;
        }
        // f*_i = f_i^eq(rho, u_mix + F/rho) + (1 - 1/tau_mix) f'_i, Eq. (LBM_BGK),
        // = w rho + t_i with t_i = w rho D_s + om1 f'; the rest population
        // takes what the others leave of rho (the f*_i of a node sum to rho
        // exactly for both forms of f', so this is the same value, rounded
        // once).  FP32 / FP64 store f*_i = w rho + t_i (out); the 16-bit
        // formats store s_i = f*_i - w_i rhohat = w_i (rho - rhohat) + t_i and
        // s_0 = w_0 (rho - rhohat) - sum_{i>0} t_i (out holds s), one rounding
        // to FP32 before the one to 16 bits
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const R w = wr[weight_class(i)];
            const R ti = xfma(w, Ds[i], xmul(om1, fn[i]));
            if constexpr (C::kCompensated) {
                // (wr + wl)(1 + D_s) + om1 f' rounded once: the low part of
                // w rho rides with t_i, scaled like the rest of f^eq
                const R lo = wl[weight_class(i)];
                out[a][i] = xadd(w, xadd(ti, xfma(lo, Ds[i], lo)));
                fn[i] = ti;
            } else {
                out[a][i] = C::kNodeShift ? xfma(wgt<R>(i), delta, ti) : xadd(w, ti);
                if (C::kNodeShift) fn[i] = ti;
            }
        }
        if constexpr (C::kCompensated) {
            // the f*_i of a node sum to rho, and the w_i D_s,i and f'_i of
            // a node sum to zero, so f*_0 = w_0 rho - sum_{i>0} t_i
            const R ts = xadd(xadd(xadd(fn[1], fn[3]), xadd(fn[2], fn[4])), xadd(xadd(fn[5], fn[7]), xadd(fn[6], fn[8])));
            out[a][0] = xadd(wr[0], xsub(wl[0], ts));
        } else if (C::kNodeShift) {
            const R ts = xadd(xadd(xadd(fn[1], fn[3]), xadd(fn[2], fn[4])), xadd(xadd(fn[5], fn[7]), xadd(fn[6], fn[8])));
            out[a][0] = xfma(wgt<R>(0), delta, -ts);
        } else {
            out[a][0] = xsub(rho, xadd(xadd(xadd(out[a][1], out[a][3]), xadd(out[a][2], out[a][4])),
                                       xadd(xadd(out[a][5], out[a][7]), xadd(out[a][6], out[a][8]))));
        }
#pragma unroll
        for (int i = 0; i < 9; i++) d[i * plane] = C::pack(out[a][i]);
    }
    // periodic ghost images of columns 0, 1, nx - 2, nx - 1 (ghost columns
    // -2, -1, nx, nx + 1 hold columns (nx - 2, nx - 1, 0, 1) mod nx)
    if (periodic && (x < 2 || x >= nx - 2)) {
        const int gcols[4] = {-2, -1, nx, nx + 1};
        // not unrolled: only four columns of the grid run this, and one copy
        // of the 18 stores keeps the step kernels' code small
#pragma unroll 1
        for (int k = 0; k < 4; k++) {
            int m = gcols[k] % nx;
            if (m < 0) m += nx;
            if (m != x) continue;
            const int off = gcols[k] - x;
#pragma unroll
            for (int a = 0; a < 2; a++) {
                if (C::kNodeShift) dst[(18 + a) * plane + off] = C::rho_store(a ? rho1 : rho0);
#pragma unroll
                for (int i = 0; i < 9; i++) dst[a * 9 * plane + i * plane + off] = C::pack(out[a][i]);
            }
        }
    }
    ob.m0 += rho0;
    ob.m1 += rho1;
    ob.px += jx[0] + R(0.5) * rho0 * ax0;
    const R vx = ux + R(0.5) * (rho0 * ax0 + rho1 * ax1) * inv_rt;
    const R vy = uy + R(0.5) * (rho0 * ay0 + rho1 * ay1) * inv_rt;
    ob.umax2 = fmax(ob.umax2, vx * vx + vy * vy);
    ob.bad = ob.bad || !(rho0 >= R(0) && rho1 >= R(0));
}

// Macroscopic fields at one node (fields mode).
template <typename R>
__device__ __forceinline__ void node_fields(const R (&f)[2][9], R rho0, R rho1, const R (&nb)[2][8],
                                            const NodeParams<R>& P, double* __restrict__ out,
                                            size_t fplane) {
    R sx[2], sy[2];
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const R e = nb[b][0], n = nb[b][1], wv = nb[b][2], so = nb[b][3];
        const R ne = nb[b][4], nw = nb[b][5], sw = nb[b][6], se = nb[b][7];
        sx[b] = (e - wv) * R(1.0 / 9.0) + (ne - nw - sw + se) * R(1.0 / 36.0);
        sy[b] = (n - so) * R(1.0 / 9.0) + (ne + nw - sw - se) * R(1.0 / 36.0);
    }
    const R ax0 = P.G * sx[1] + P.gx, ay0 = P.G * sy[1] + P.gy;
    const R ax1 = P.G * sx[0] + P.gx, ay1 = P.G * sy[0] + P.gy;
    R jx = R(0), jy = R(0);
#pragma unroll
    for (int a = 0; a < 2; a++) {
        jx += (f[a][1] - f[a][3]) + (f[a][5] - f[a][7]) + (f[a][8] - f[a][6]);
        jy += (f[a][2] - f[a][4]) + (f[a][5] - f[a][7]) + (f[a][6] - f[a][8]);
    }
    const R rt = rho0 + rho1;
    const R inv_rt = R(1) / rt;
    out[0] = double(rho0);
    out[fplane] = double(rho1);
    out[2 * fplane] = double((jx + R(0.5) * (rho0 * ax0 + rho1 * ax1)) * inv_rt);
    out[3 * fplane] = double((jy + R(0.5) * (rho0 * ay0 + rho1 * ay1)) * inv_rt);
    out[4 * fplane] = double(R(1.0 / 3.0) * rt - P.G * R(1.0 / 3.0) * rho0 * rho1);
}

// Block reduction of the per-thread observables, FP64 atomics into `acc`, and
// finalisation of the step by the last of the `nblocks` CTAs that reduce into
// the same accumulators (all CTAs of the grid by default).
template <typename R, int NT>
__device__ __forceinline__ void reduce_observables(ObsLocal<R> ob, ObsAccum* __restrict__ acc,
                                                   ObsState* __restrict__ obs, bool timed_out,
                                                   unsigned nblocks = 0u) {
    __shared__ R red[NT / 32][4];
    __shared__ unsigned red_bad;
    __shared__ bool is_last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) red_bad = timed_out ? 2u : 0u;
    R m0 = warp_sum(ob.m0), m1 = warp_sum(ob.m1), px = warp_sum(ob.px), u2 = warp_max(ob.umax2);
    const unsigned any_bad = __any_sync(0xffffffffu, ob.bad);
    __syncthreads();
    if (lane == 0) {
        red[warp][0] = m0;
        red[warp][1] = m1;
        red[warp][2] = px;
        red[warp][3] = u2;
        if (any_bad) atomicOr(&red_bad, 1u);
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; w++) {
            a += double(red[w][0]);
            b += double(red[w][1]);
            c += double(red[w][2]);
            d = fmax(d, double(red[w][3]));
        }
        atomicAdd(&acc->mass[0], a);
        atomicAdd(&acc->mass[1], b);
        atomicAdd(&acc->px, c);
        atomicMax(&acc->umax2_bits, (unsigned long long)__double_as_longlong(d));
        if (red_bad) atomicOr(&acc->bad, red_bad);
        __threadfence();
        const unsigned ticket = atomicAdd(&acc->blocks_done, 1u);
        is_last = ticket == (nblocks ? nblocks : gridDim.x * gridDim.y) - 1;
    }
    __syncthreads();
    if (is_last && t == 0) {
        __threadfence();
        const double ma = __ldcg(&acc->mass[0]);
        const double mb = __ldcg(&acc->mass[1]);
        const double p = __ldcg(&acc->px);
        const double u2s = __longlong_as_double((long long)__ldcg(&acc->umax2_bits));
        const unsigned nb = __ldcg(&acc->bad);
        obs->mass[0] = ma;
        obs->mass[1] = mb;
        obs->px = p;
        obs->umax = sqrt(u2s);
        if (ma > 0.0) obs->disp += p / ma;
        obs->step += 1;
        if (nb & 1u) obs->nan_flag = 1;
        if (nb & 2u) obs->timeout_flag = 1;
        acc->mass[0] = 0.0;
        acc->mass[1] = 0.0;
        acc->px = 0.0;
        acc->umax2_bits = 0ull;
        acc->bad = 0u;
        __threadfence();
        acc->blocks_done = 0u;
    }
}

}  // namespace gb300lbm
