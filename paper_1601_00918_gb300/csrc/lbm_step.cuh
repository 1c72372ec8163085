// Two-component D2Q9 time step for sm_103a: one fused kernel per step.
//
// Method (Otomo et al., Section 2): per node and species a in {o, w}
//   pull      f_i^a(x) = f*_i^a(x - c_i), or f*_opp(i)^a(x) when x - c_i is
//             solid (halfway bounce-back);
//   density   rho^a = sum_i f_i^a; a solid node carries rho_s^a;
//   force     F^a/rho^a = G sum_i w_i c_i rho^b(x + c_i) + g
//             (Eq. comp_interaction, wall potentials, Section 3.4 body force);
//   moments   j^a = sum_i c_i f_i^a, u_mix = (j^o + j^w)/rho,
//             nu_mix = (rho^o nu^o + rho^w nu^w)/rho, tau_mix = nu_mix/T0 + 1/2;
//   collide   f*_i^a = f_i^eq(rho^a, u_mix + F^a/rho^a)
//                    + (1 - 1/tau_mix) (f_i^a - f_i^eq(rho^a, u_mix))
//             (Eqs. LBM_BGK, feq, collision_term).
//
// Design.  The force at x needs rho^b at the eight neighbours, i.e. the
// pulled populations of neighbouring nodes, so a plain one-node-per-thread
// kernel needs either a separate density pass (an extra read of every
// population) or a halo recompute.  Here a CTA owns BX consecutive columns
// and marches down a strip of rows.  For each new row it pulls that row's 18
// populations into registers and writes the row's densities into a 4-row
// ring in shared memory; the row above, whose three density rows are then
// complete, is collided from the registers kept from the previous iteration.
// Every population is read from global memory once per step (plus one halo
// row per strip and a halo column on each side computed by one warp each),
// every post-collision population is written once.  The per-step
// observables are reduced in the same kernel (warp shuffles, FP64 atomics,
// the last CTA finalising), so one step is one launch.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gb300lbm {

constexpr int kSolidBit = 15;   // link word: bit i (1..8) = pull source x - c_i is solid

// Device-resident parameters (read each launch, so captured graphs follow
// lbm_set_body_force).
struct StepParams {
    double nu[2];        // nu^a = T0 (tau^a - 1/2)
    double G;
    double g[2];
    double rho_wall[2];
    double k3;           // 4.5 with the cubic terms of Eq. (feq), 0 without
    double rho_ref[2];   // shift of the 16-bit storage: stored = f - w_i rho_ref^a
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
    int pad;
};

// ---------------------------------------------------------------------------
// storage codecs: plain FP64 / FP32, or 16-bit shifted by w_i rho_ref^a
// ---------------------------------------------------------------------------
template <typename S>
struct Codec;

template <>
struct Codec<double> {
    using R = double;
    static __device__ __forceinline__ double load(const double* p, double) { return __ldg(p); }
    static __device__ __forceinline__ void store(double* p, double v, double) { *p = v; }
};

template <>
struct Codec<float> {
    using R = float;
    static __device__ __forceinline__ float load(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v, float) { *p = v; }
};

template <>
struct Codec<__half> {
    using R = float;
    static __device__ __forceinline__ float load(const __half* p, float shift) {
        return __half2float(__ldg(p)) + shift;
    }
    static __device__ __forceinline__ void store(__half* p, float v, float shift) {
        *p = __float2half_rn(v - shift);
    }
};

template <>
struct Codec<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, float shift) {
        return __bfloat162float(__ldg(p)) + shift;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, float shift) {
        *p = __float2bfloat16_rn(v - shift);
    }
};

// D2Q9, textbook order: c_0 = (0,0); c_1..c_4 = (1,0),(0,1),(-1,0),(0,-1);
// c_5..c_8 = (1,1),(-1,1),(-1,-1),(1,-1).  opp = {0,3,4,1,2,7,8,5,6}.
__device__ __forceinline__ int d2q9_cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ int d2q9_cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ int d2q9_opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }

template <typename R>
__device__ __forceinline__ R weight_of(int i) {
    return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

// Eq. (feq) with T0 = 1/3, written by parity of c_i.u:
//   f_i^eq = w_i rho [E + O],  E = 1 - 1.5 u^2 + 4.5 (c.u)^2,
//                              O = (c.u) (3 - k3 u^2 + k3 (c.u)^2),
// k3 = 4.5 for the cubic equilibrium; opposite directions share E and flip O.
template <typename R>
__device__ __forceinline__ void equilibrium(R rho, R ux, R uy, R k3, R (&out)[9]) {
    const R uu = ux * ux + uy * uy;
    const R A = R(1) - R(1.5) * uu;
    const R B = R(3) - k3 * uu;
    const R w0 = rho * R(4.0 / 9.0), w1 = rho * R(1.0 / 9.0), w5 = rho * R(1.0 / 36.0);
    out[0] = w0 * A;
    {
        const R c = ux, c2 = c * c, e = A + R(4.5) * c2, o = c * (B + k3 * c2);
        out[1] = w1 * (e + o);
        out[3] = w1 * (e - o);
    }
    {
        const R c = uy, c2 = c * c, e = A + R(4.5) * c2, o = c * (B + k3 * c2);
        out[2] = w1 * (e + o);
        out[4] = w1 * (e - o);
    }
    {
        const R c = ux + uy, c2 = c * c, e = A + R(4.5) * c2, o = c * (B + k3 * c2);
        out[5] = w5 * (e + o);
        out[7] = w5 * (e - o);
    }
    {
        const R c = uy - ux, c2 = c * c, e = A + R(4.5) * c2, o = c * (B + k3 * c2);
        out[6] = w5 * (e + o);
        out[8] = w5 * (e - o);
    }
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

struct Grid {
    int nx, ny, pitch;
    int rows_per_block;
    int row_begin;        // first row handled by blockIdx.y == 0 (fields windows)
    int row_end;          // one past the last row handled by this launch
};

// FIELDS = false: one time step fin -> fout with observables.
// FIELDS = true : macroscopic fields of fin into `fields` (no fout write):
//   fields[0..1][y][x] = rho^o, rho^w; [2..3] = u_x, u_y; [4] = pressure,
//   rows [row_begin, row_end), planes of nx * (row_end - row_begin) doubles.
template <typename S, int BX, bool FIELDS>
__global__ void __launch_bounds__(BX) step_kernel(const S* __restrict__ fin, S* __restrict__ fout,
                                                  const uint16_t* __restrict__ links,
                                                  const StepParams* __restrict__ prm,
                                                  ObsAccum* __restrict__ acc, ObsState* __restrict__ obs,
                                                  double* __restrict__ fields, Grid grid) {
    using C = Codec<S>;
    using R = typename C::R;
    constexpr unsigned kSolid = 1u << kSolidBit;

    const int nx = grid.nx, ny = grid.ny, pitch = grid.pitch;
    const int plane = ny * pitch;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int x0 = blockIdx.x * BX;
    const int y0 = grid.row_begin + blockIdx.y * grid.rows_per_block;
    const int y1 = min(y0 + grid.rows_per_block, grid.row_end);

    __shared__ R s_rho[4][2][BX + 2];

    const R G = R(prm->G), gxa = R(prm->g[0]), gya = R(prm->g[1]);
    const R rw0 = R(prm->rho_wall[0]), rw1 = R(prm->rho_wall[1]);
    const R nu0 = R(prm->nu[0]), nu1 = R(prm->nu[1]), k3 = R(prm->k3);
    const R ref0 = R(prm->rho_ref[0]), ref1 = R(prm->rho_ref[1]);
    const R sh0[3] = {ref0 * R(4.0 / 9.0), ref0 * R(1.0 / 9.0), ref0 * R(1.0 / 36.0)};
    const R sh1[3] = {ref1 * R(4.0 / 9.0), ref1 * R(1.0 / 9.0), ref1 * R(1.0 / 36.0)};

    // column owned by this thread; the first thread past the right edge of
    // the grid pulls the periodic image column 0 (its density only).
    const int gxc = x0 + t;
    const bool active = gxc < nx;
    const bool rho_col = gxc <= nx;
    const int cx = active ? gxc : 0;
    const int xm = cx == 0 ? nx - 1 : cx - 1;
    const int xp = cx == nx - 1 ? 0 : cx + 1;

    auto slot = [&](int r) { return (r - y0 + 1) & 3; };
    auto wrap_y = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };

    // Pull the 18 populations of row y at column cx.  Returns true at a
    // solid node (then f is untouched and r0, r1 = wall potentials).
    auto pull = [&](int y, R(&f)[2][9], R& r0, R& r1) -> bool {
        const unsigned lk = links[y * pitch + cx];
        if (lk & kSolid) {
            r0 = rw0;
            r1 = rw1;
            return true;
        }
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int oy = y * pitch, oym = ym * pitch, oyp = yp * pitch;
        int src[9];
        src[0] = oy + cx;
        src[1] = (lk & (1u << 1)) ? 3 * plane + oy + cx : 1 * plane + oy + xm;
        src[2] = (lk & (1u << 2)) ? 4 * plane + oy + cx : 2 * plane + oym + cx;
        src[3] = (lk & (1u << 3)) ? 1 * plane + oy + cx : 3 * plane + oy + xp;
        src[4] = (lk & (1u << 4)) ? 2 * plane + oy + cx : 4 * plane + oyp + cx;
        src[5] = (lk & (1u << 5)) ? 7 * plane + oy + cx : 5 * plane + oym + xm;
        src[6] = (lk & (1u << 6)) ? 8 * plane + oy + cx : 6 * plane + oym + xp;
        src[7] = (lk & (1u << 7)) ? 5 * plane + oy + cx : 7 * plane + oyp + xp;
        src[8] = (lk & (1u << 8)) ? 6 * plane + oy + cx : 8 * plane + oyp + xm;
        const S* f1 = fin + 9 * plane;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            // bounced populations come from the opposite direction, whose
            // weight (and so whose storage shift) is the same
            const int wi = i == 0 ? 0 : (i <= 4 ? 1 : 2);
            f[0][i] = C::load(fin + src[i], sh0[wi]);
            f[1][i] = C::load(f1 + src[i], sh1[wi]);
        }
        R a = R(0), b = R(0);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            a += f[0][i];
            b += f[1][i];
        }
        r0 = a;
        r1 = b;
        return false;
    };

    // Densities of the two halo columns x0 - 1 (warp 0) and x0 + BX (warp 1)
    // at row y: lanes 0..8 pull species o, lanes 16..24 species w.
    auto halo = [&](int y, int sl) {
        if (warp >= 2) return;
        const bool right = warp == 1;
        if (right && x0 + BX > nx) return;  // image column pulled by a thread instead
        int hx = right ? x0 + BX : x0 - 1;
        hx = hx < 0 ? hx + nx : (hx >= nx ? hx - nx : hx);
        const unsigned lk = links[y * pitch + hx];
        const int sp = lane >> 4, i = lane & 15;
        R v = R(0);
        if (!(lk & kSolid) && i < 9) {
            int sxp = hx - d2q9_cx(i);
            sxp = sxp < 0 ? sxp + nx : (sxp >= nx ? sxp - nx : sxp);
            const int syp = wrap_y(y - d2q9_cy(i));
            const int idx = (lk & (1u << i)) ? d2q9_opp(i) * plane + y * pitch + hx
                                             : i * plane + syp * pitch + sxp;
            v = C::load(fin + sp * 9 * plane + idx, weight_of<R>(i) * (sp ? ref1 : ref0));
        }
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if ((lane & 15) == 0) {
            const R val = (lk & kSolid) ? (sp ? rw1 : rw0) : v;
            s_rho[sl][sp][right ? BX + 1 : 0] = val;
        }
    };

    R cur[2][9], nxt[2][9];
    R rc0 = R(0), rc1 = R(0), rn0 = R(0), rn1 = R(0);
    bool solid_cur = true, solid_nxt = true;

    // observables (per thread)
    R m0 = R(0), m1 = R(0), pxs = R(0), umax2 = R(0);
    bool bad = false;

    // prologue: densities of rows y0 - 1 and y0
    {
        const int y = wrap_y(y0 - 1);
        if (rho_col) {
            R tmp[2][9], a, b;
            pull(y, tmp, a, b);
            s_rho[slot(y0 - 1)][0][t + 1] = a;
            s_rho[slot(y0 - 1)][1][t + 1] = b;
        }
        halo(y, slot(y0 - 1));
    }
    if (rho_col) {
        solid_cur = pull(y0, cur, rc0, rc1);
        s_rho[slot(y0)][0][t + 1] = rc0;
        s_rho[slot(y0)][1][t + 1] = rc1;
    }
    halo(y0, slot(y0));

    for (int r = y0; r < y1; ++r) {
        const int yn = r + 1 == ny ? 0 : r + 1;
        const int sn = slot(r + 1);
        if (rho_col) {
            solid_nxt = pull(yn, nxt, rn0, rn1);
            s_rho[sn][0][t + 1] = rn0;
            s_rho[sn][1][t + 1] = rn1;
        }
        halo(yn, sn);
        __syncthreads();

        if (active) {
            const int s0 = slot(r), sm = slot(r - 1), sp = sn;
            if (solid_cur) {
                if (FIELDS) {
                    const int o = (r - grid.row_begin) * nx + cx;
                    const size_t fp = (size_t)nx * (grid.row_end - grid.row_begin);
                    fields[o] = double(rw0);
                    fields[fp + o] = double(rw1);
                    fields[2 * fp + o] = 0.0;
                    fields[3 * fp + o] = 0.0;
                    fields[4 * fp + o] = 0.0;
                }
            } else {
                // sum_i w_i c_i rho^b(x + c_i) for b = w (acting on o) and b = o
                R sx[2], sy[2];
#pragma unroll
                for (int b = 0; b < 2; b++) {
                    const R e = s_rho[s0][b][t + 2], wv = s_rho[s0][b][t];
                    const R n = s_rho[sp][b][t + 1], so = s_rho[sm][b][t + 1];
                    const R ne = s_rho[sp][b][t + 2], nw = s_rho[sp][b][t];
                    const R sw = s_rho[sm][b][t], se = s_rho[sm][b][t + 2];
                    sx[b] = (e - wv) * R(1.0 / 9.0) + (ne - nw - sw + se) * R(1.0 / 36.0);
                    sy[b] = (n - so) * R(1.0 / 9.0) + (ne + nw - sw - se) * R(1.0 / 36.0);
                }
                const R ax0 = G * sx[1] + gxa, ay0 = G * sy[1] + gya;   // species o
                const R ax1 = G * sx[0] + gxa, ay1 = G * sy[0] + gya;   // species w

                R jx[2], jy[2];
#pragma unroll
                for (int a = 0; a < 2; a++) {
                    const R(&f)[9] = cur[a];
                    jx[a] = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
                    jy[a] = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
                }
                const R rt = rc0 + rc1;
                const R inv_rt = R(1) / rt;
                const R ux = (jx[0] + jx[1]) * inv_rt;
                const R uy = (jy[0] + jy[1]) * inv_rt;

                if (FIELDS) {
                    const int o = (r - grid.row_begin) * nx + cx;
                    const size_t fp = (size_t)nx * (grid.row_end - grid.row_begin);
                    fields[o] = double(rc0);
                    fields[fp + o] = double(rc1);
                    fields[2 * fp + o] = double(ux + R(0.5) * (rc0 * ax0 + rc1 * ax1) * inv_rt);
                    fields[3 * fp + o] = double(uy + R(0.5) * (rc0 * ay0 + rc1 * ay1) * inv_rt);
                    fields[4 * fp + o] =
                        double(R(1.0 / 3.0) * rt - G * R(1.0 / 3.0) * rc0 * rc1);
                } else {
                    const R nu_mix = (rc0 * nu0 + rc1 * nu1) * inv_rt;
                    const R om1 = R(1) - R(1) / (R(3) * nu_mix + R(0.5));   // 1 - 1/tau_mix
                    const int o = r * pitch + cx;
#pragma unroll
                    for (int a = 0; a < 2; a++) {
                        const R rho = a ? rc1 : rc0;
                        const R ax = a ? ax1 : ax0, ay = a ? ay1 : ay0;
                        R fu[9], fs[9];
                        equilibrium<R>(rho, ux, uy, k3, fu);
                        equilibrium<R>(rho, ux + ax, uy + ay, k3, fs);
                        S* dst = fout + a * 9 * plane + o;
#pragma unroll
                        for (int i = 0; i < 9; i++) {
                            const int wi = i == 0 ? 0 : (i <= 4 ? 1 : 2);
                            const R v = fs[i] + om1 * (cur[a][i] - fu[i]);
                            C::store(dst + i * plane, v, a ? sh1[wi] : sh0[wi]);
                        }
                    }
                    m0 += rc0;
                    m1 += rc1;
                    pxs += jx[0] + R(0.5) * rc0 * ax0;
                    const R vx = ux + R(0.5) * (rc0 * ax0 + rc1 * ax1) * inv_rt;
                    const R vy = uy + R(0.5) * (rc0 * ay0 + rc1 * ay1) * inv_rt;
                    umax2 = fmax(umax2, vx * vx + vy * vy);
                    bad = bad || !(rc0 >= R(0) && rc1 >= R(0));
                }
            }
        }
        // rotate the register rows (the ring slot of row r - 1 is reused two
        // iterations later, after the next barrier)
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int i = 0; i < 9; i++) cur[a][i] = nxt[a][i];
        rc0 = rn0;
        rc1 = rn1;
        solid_cur = solid_nxt;
    }

    if (FIELDS) return;

    // ---- observables: block reduction, FP64 atomics, last block finalises ----
    __shared__ R red[BX / 32][4];
    __shared__ unsigned red_bad;
    __shared__ bool is_last;
    if (t == 0) red_bad = 0u;
    m0 = warp_sum(m0);
    m1 = warp_sum(m1);
    pxs = warp_sum(pxs);
    umax2 = warp_max(umax2);
    const unsigned any_bad = __any_sync(0xffffffffu, bad);
    __syncthreads();
    if (lane == 0) {
        red[warp][0] = m0;
        red[warp][1] = m1;
        red[warp][2] = pxs;
        red[warp][3] = umax2;
        if (any_bad) atomicOr(&red_bad, 1u);
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
#pragma unroll
        for (int w = 0; w < BX / 32; w++) {
            a += double(red[w][0]);
            b += double(red[w][1]);
            c += double(red[w][2]);
            d = fmax(d, double(red[w][3]));
        }
        atomicAdd(&acc->mass[0], a);
        atomicAdd(&acc->mass[1], b);
        atomicAdd(&acc->px, c);
        atomicMax(&acc->umax2_bits, (unsigned long long)__double_as_longlong(d));
        if (red_bad) atomicOr(&acc->bad, 1u);
        __threadfence();
        const unsigned ticket = atomicAdd(&acc->blocks_done, 1u);
        is_last = ticket == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (is_last && t == 0) {
        __threadfence();
        const double ma = __ldcg(&acc->mass[0]);
        const double mb = __ldcg(&acc->mass[1]);
        const double p = __ldcg(&acc->px);
        const double u2 = __longlong_as_double((long long)__ldcg(&acc->umax2_bits));
        const unsigned nb = __ldcg(&acc->bad);
        obs->mass[0] = ma;
        obs->mass[1] = mb;
        obs->px = p;
        obs->umax = sqrt(u2);
        if (ma > 0.0) obs->disp += p / ma;
        obs->step += 1;
        if (nb) obs->nan_flag = 1;
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
