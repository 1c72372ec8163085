// Two-component D2Q9 time step, "simple" variant: global loads straight into
// registers.
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
// pulled populations of neighbouring nodes, so a one-node-per-thread kernel
// needs either a separate density pass (an extra read of every population)
// or a halo recompute.  Here a CTA owns BX consecutive columns and marches
// down a strip of rows.  For each new row it pulls that row's 18 populations
// into registers and writes the row's densities into a 4-row ring in shared
// memory; the row above, whose three density rows are then complete, is
// collided from the registers kept from the previous iteration.  Every
// population is read from global memory once per step (plus one halo row per
// strip and a halo column on each side, computed by one warp each) and every
// post-collision population is written once.  Solid nodes issue no loads.
// This variant also computes the macroscopic fields (FIELDS = true).
#pragma once

#include <cooperative_groups.h>

#include "lbm_common.cuh"

namespace gb300lbm {

// The march of one CTA over rows [y0, y1) of columns [x0, x0 + BX).
// FIELDS = false: one time step fin -> fout, observables into `ob`.
// FIELDS = true : macroscopic fields of fin into `fields` (no fout write):
//   fields[0..1][y][x] = rho^o, rho^w; [2..3] = u_x, u_y; [4] = pressure,
//   for rows [fr0, fr0 + frows), planes of nx * frows doubles.
// fin, fout and links point at logical column 0 of row 0.  periodic_x only
// controls the ghost images written for the staged kernel's row windows
// (pass 0 for a layout without ghost columns); pulls wrap in x and y.
// kCoherent: populations are loaded through L2 only (load_pop), for a
// persistent launch that reads what it wrote in the previous step.
template <typename S, int BX, bool FIELDS, bool kCoherent = false>
__device__ __forceinline__ void march_simple(const S* __restrict__ fin, S* __restrict__ fout,
                                             const uint16_t* __restrict__ links,
                                             const NodeParams<typename Codec<S>::R>& P,
                                             double* __restrict__ fields, int nx, int ny, int pitch,
                                             int periodic_x, int x0, int y0, int y1, int fr0, int frows,
                                             ObsLocal<typename Codec<S>::R>& ob,
                                             pair_t<typename Codec<S>::R> (*s_rho)[BX + 2]) {
    using C = Codec<S>;
    using R = typename C::R;
    constexpr unsigned kSolid = 1u << kSolidBit;
    const int plane = ny * pitch;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;

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
    // solid node (then f is untouched and r0, r1 = wall potentials); l0, l1
    // receive the low parts of the density sums (density_of).
    auto pull = [&](int y, R(&f)[2][9], R& r0, R& r1, R& l0, R& l1) -> bool {
        const unsigned lk = links[y * pitch + cx];
        if (lk & kSolid) {
            r0 = P.rw0;
            r1 = P.rw1;
            l0 = l1 = R(0);
            return true;
        }
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int oy = y * pitch, oym = ym * pitch, oyp = yp * pitch;
        // node (offset within a plane) and plane of each pulled population;
        // a bounced population is the node's own one of the opposite direction
        const int own = oy + cx;
        int nd[9], pl[9];
        nd[0] = own;
        pl[0] = 0;
        const bool b1 = lk & (1u << 1), b2 = lk & (1u << 2), b3 = lk & (1u << 3), b4 = lk & (1u << 4);
        const bool b5 = lk & (1u << 5), b6 = lk & (1u << 6), b7 = lk & (1u << 7), b8 = lk & (1u << 8);
        nd[1] = b1 ? own : oy + xm;   pl[1] = b1 ? 3 : 1;
        nd[2] = b2 ? own : oym + cx;  pl[2] = b2 ? 4 : 2;
        nd[3] = b3 ? own : oy + xp;   pl[3] = b3 ? 1 : 3;
        nd[4] = b4 ? own : oyp + cx;  pl[4] = b4 ? 2 : 4;
        nd[5] = b5 ? own : oym + xm;  pl[5] = b5 ? 7 : 5;
        nd[6] = b6 ? own : oym + xp;  pl[6] = b6 ? 8 : 6;
        nd[7] = b7 ? own : oyp + xp;  pl[7] = b7 ? 5 : 7;
        nd[8] = b8 ? own : oyp + xm;  pl[8] = b8 ? 6 : 8;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            // 16-bit formats: shift by the source node's density (the same
            // weight for i and opp(i))
            R r0s = R(0), r1s = R(0);
            if (C::kNodeShift) {
                r0s = C::rho_value(load_pop<kCoherent>(fin + 18 * plane + nd[i]));
                r1s = C::rho_value(load_pop<kCoherent>(fin + 19 * plane + nd[i]));
            }
            f[0][i] = C::decode(load_pop<kCoherent>(fin + pl[i] * plane + nd[i]), wgt<R>(i), r0s);
            f[1][i] = C::decode(load_pop<kCoherent>(fin + (9 + pl[i]) * plane + nd[i]), wgt<R>(i), r1s);
        }
        density_of<C>(f[0], r0, l0);
        density_of<C>(f[1], r1, l1);
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
            const bool bb = lk & (1u << i);
            const int node = bb ? y * pitch + hx : syp * pitch + sxp;
            const int pln = bb ? d2q9_opp(i) : i;
            R rs = R(0);
            if (C::kNodeShift) rs = C::rho_value(load_pop<kCoherent>(fin + (18 + sp) * plane + node));
            v = C::decode(load_pop<kCoherent>(fin + (sp * 9 + pln) * plane + node), wgt<R>(i), rs);
        }
        v = halfwarp_density<C>(v);
        if ((lane & 15) == 0) {
            const R val = (lk & kSolid) ? (sp ? P.rw1 : P.rw0) : v;
            reinterpret_cast<R*>(&s_rho[sl][right ? BX + 1 : 0])[sp] = val;
        }
    };

    R cur[2][9], nxt[2][9];
    R rc0 = R(0), rc1 = R(0), rn0 = R(0), rn1 = R(0);
    R lc0 = R(0), lc1 = R(0), ln0 = R(0), ln1 = R(0);
    bool solid_cur = true, solid_nxt = true;

    // prologue: densities of rows y0 - 1 and y0
    {
        const int y = wrap_y(y0 - 1);
        if (rho_col) {
            R tmp[2][9], a, b, la, lb;
            pull(y, tmp, a, b, la, lb);
            s_rho[slot(y0 - 1)][t + 1] = make_pair_of<R>(a, b);
        }
        halo(y, slot(y0 - 1));
    }
    if (rho_col) {
        solid_cur = pull(y0, cur, rc0, rc1, lc0, lc1);
        s_rho[slot(y0)][t + 1] = make_pair_of<R>(rc0, rc1);
    }
    halo(y0, slot(y0));

    for (int r = y0; r < y1; ++r) {
        const int yn = r + 1 == ny ? 0 : r + 1;
        const int sn = slot(r + 1);
        if (rho_col) {
            solid_nxt = pull(yn, nxt, rn0, rn1, ln0, ln1);
            s_rho[sn][t + 1] = make_pair_of<R>(rn0, rn1);
        }
        halo(yn, sn);
        __syncthreads();

        if (active) {
            const int s0 = slot(r), sm = slot(r - 1), sp = sn;
            if (solid_cur) {
                if (FIELDS) {
                    const size_t fp = (size_t)nx * frows;
                    double* o = fields + (size_t)(r - fr0) * nx + cx;
                    o[0] = double(P.rw0);
                    o[fp] = double(P.rw1);
                    o[2 * fp] = 0.0;
                    o[3 * fp] = 0.0;
                    o[4 * fp] = 0.0;
                }
            } else {
                R nb[2][8];
                {
                    const pair_t<R> e = s_rho[s0][t + 2], n = s_rho[sp][t + 1], wv = s_rho[s0][t];
                    const pair_t<R> so = s_rho[sm][t + 1], ne = s_rho[sp][t + 2], nw = s_rho[sp][t];
                    const pair_t<R> sw = s_rho[sm][t], se = s_rho[sm][t + 2];
                    // neighbours x + c_k in direction order k = 1..8
                    nb[0][0] = e.x;  nb[1][0] = e.y;
                    nb[0][1] = n.x;  nb[1][1] = n.y;
                    nb[0][2] = wv.x; nb[1][2] = wv.y;
                    nb[0][3] = so.x; nb[1][3] = so.y;
                    nb[0][4] = ne.x; nb[1][4] = ne.y;
                    nb[0][5] = nw.x; nb[1][5] = nw.y;
                    nb[0][6] = sw.x; nb[1][6] = sw.y;
                    nb[0][7] = se.x; nb[1][7] = se.y;
                }
                if (FIELDS) {
                    node_fields<R>(cur, rc0, rc1, nb, P, fields + (size_t)(r - fr0) * nx + cx,
                                   (size_t)nx * frows);
                } else {
                    collide_store<S, R>(cur, rc0, rc1, lc0, lc1, nb, P, fout + r * pitch + cx, plane, cx, nx,
                                        periodic_x, ob);
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
        lc0 = ln0;
        lc1 = ln1;
        solid_cur = solid_nxt;
    }
}

// One time step (or the fields) of a single grid: CTA (bx, by) marches rows
// [row_begin + by * rows_per_block, ...) of columns [bx * BX, bx * BX + BX).
template <typename S, int BX, bool FIELDS>
__global__ void __launch_bounds__(BX) step_simple_kernel(const S* __restrict__ fin, S* __restrict__ fout,
                                                         const uint16_t* __restrict__ links,
                                                         const StepParams* __restrict__ prm,
                                                         ObsAccum* __restrict__ acc,
                                                         ObsState* __restrict__ obs,
                                                         double* __restrict__ fields, Grid grid) {
    using R = typename Codec<S>::R;
    __shared__ pair_t<R> s_rho[4][BX + 2];
    NodeParams<R> P;
    P.load(prm);
    const int x0 = blockIdx.x * BX;
    const int y0 = grid.row_begin + blockIdx.y * grid.rows_per_block;
    const int y1 = min(y0 + grid.rows_per_block, grid.row_end);
    ObsLocal<R> ob;
    march_simple<S, BX, FIELDS>(fin, fout, links, P, fields, grid.nx, grid.ny, grid.pitch, grid.periodic_x,
                                x0, y0, y1, grid.row_begin, grid.row_end - grid.row_begin, ob, s_rho);
    if (FIELDS) return;
    reduce_observables<R, BX>(ob, acc, obs, false);
}

// Many steps of one small grid in one launch: a cooperative grid of
// resident CTAs, each marching its share of the (128-column block, row
// strip) tiles of a step, then a grid-wide barrier before the next step
// (steps alternate between f0 and f1 starting from `parity`).  Populations
// are loaded through L2 (the buffer read in step s + 1 is written in step
// s); every CTA reduces its observables once per step.  For grids whose
// steps are a few microseconds of work, this replaces one launch (or graph
// node) per step.
template <typename S, int BX>
__global__ void __launch_bounds__(BX) step_persist_kernel(S* f0, S* f1, const uint16_t* __restrict__ links,
                                                          const StepParams* __restrict__ prm, ObsAccum* __restrict__ acc,
                                                          ObsState* __restrict__ obs, Grid grid, int nsteps, int parity) {
    using R = typename Codec<S>::R;
    __shared__ pair_t<R> s_rho[4][BX + 2];
    NodeParams<R> P;
    P.load(prm);
    const int ncb = (grid.nx + BX - 1) / BX;
    const int nstrip = (grid.ny + grid.rows_per_block - 1) / grid.rows_per_block;
    const int ntiles = ncb * nstrip;
    cooperative_groups::grid_group gg = cooperative_groups::this_grid();
    for (int s = 0; s < nsteps; s++) {
        const bool odd = ((parity + s) & 1) != 0;
        const S* fin = odd ? f1 : f0;
        S* fout = odd ? f0 : f1;
        ObsLocal<R> ob;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int x0 = (tile % ncb) * BX;
            const int y0 = (tile / ncb) * grid.rows_per_block;
            const int y1 = min(y0 + grid.rows_per_block, grid.ny);
            march_simple<S, BX, false, true>(fin, fout, links, P, nullptr, grid.nx, grid.ny, grid.pitch,
                                             grid.periodic_x, x0, y0, y1, 0, 0, ob, s_rho);
            __syncthreads();   // the next tile's prologue reuses the density ring
        }
        reduce_observables<R, BX>(ob, acc, obs, false, gridDim.x);
        gg.sync();
    }
}

}  // namespace gb300lbm
