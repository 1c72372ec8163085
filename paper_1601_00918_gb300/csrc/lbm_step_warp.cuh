// Two-component D2Q9 time step, "warp-pipelined" variant.
//
// Same method, same TMA row staging as the staged variant (lbm_step_tma.cuh):
// one elected thread streams rows of all population planes into a ring of
// D + 3 shared-memory stages with cp.async.bulk.tensor, D rows ahead.  What
// differs is the synchronisation.  Each warp owns 32 of the CTA's columns
// and marches down the strip on its own:
//   - it computes the densities of its own two halo columns (one
//     cooperative pull per side: lanes 0..8 species o, 16..24 species w),
//     so no warp needs another warp's densities;
//   - it keeps its densities in a private 4-row ring of shared memory,
//     ordered by __syncwarp only;
//   - when it has pulled its last row out of a stage it arrives on that
//     stage's "empty" mbarrier (one arrival per warp); the producer waits on
//     it before it reuses the slot.
// So the loop has no CTA-wide barrier: a warp waits only for its data (the
// stage's "full" mbarrier) and the producer only for the slowest warp to
// release a slot it wants to refill.  All waits are bounded; a wait that
// gives up marks the step (timeout_flag) and the remaining waits are skipped.
#pragma once

#include "lbm_step_tma.cuh"

namespace gb300lbm {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <typename S, int BX, int D>
struct WarpPlan {
    static constexpr int kW = BX + 2 * kGhost;
    static constexpr int kWarps = BX / 32;
    static constexpr int kStages = D + 3;
    static constexpr int kPlanes = Codec<S>::kPlanes;
    static constexpr int kPopBytes = kPlanes * kW * (int)sizeof(S);
    static constexpr int kPopSlot = (kPopBytes + 127) / 128 * 128;
    static constexpr int kLinkSlot = (kW * 2 + 127) / 128 * 128;
    static constexpr int kSlot = kPopSlot + kLinkSlot;
    static constexpr int kBarOffset = kStages * kSlot;                       // full[NS], empty[NS]
    static constexpr int kRhoOffset = kBarOffset + ((2 * kStages * 8 + 127) / 128) * 128;
    static constexpr int kRhoBytes = kWarps * 4 * 34 * 2 * (int)sizeof(typename Codec<S>::R);
    static constexpr int kBytes = kRhoOffset + kRhoBytes + 128;
    static constexpr uint32_t kTxBytes = (uint32_t)(kPopBytes + kW * 2);
};

template <typename S, int BX, int D>
__global__ void __launch_bounds__(BX, sizeof(S) == 8 ? 2 : (BX == 64 ? 8 : 4))
    step_warp_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap lmap,
                     S* __restrict__ fout, const int2* __restrict__ rows64, const StepParams* __restrict__ prm,
                     ObsAccum* __restrict__ acc, ObsState* __restrict__ obs, Grid grid) {
    using C = Codec<S>;
    using R = typename C::R;
    using Plan = WarpPlan<S, BX, D>;
    constexpr int W = Plan::kW;
    constexpr int NS = Plan::kStages;
    constexpr int NW = Plan::kWarps;
    constexpr unsigned kSolid = 1u << kSolidBit;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned start, found in the shared window itself: pointer
    // arithmetic on the __shared__ array keeps every access a shared one
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* full = (uint64_t*)(smem + Plan::kBarOffset);
    uint64_t* empty = full + NS;
    auto pops = [&](int stage) { return (const S*)(smem + (stage % NS) * Plan::kSlot); };
    auto lnks = [&](int stage) {
        return (const uint16_t*)(smem + (stage % NS) * Plan::kSlot + Plan::kPopSlot);
    };

    const int nx = grid.nx, ny = grid.ny, pitch = grid.pitch;
    const int plane = ny * pitch;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int x0 = blockIdx.x * BX;
    // this warp's private density ring: [4 rows][34 columns] of (rho^o, rho^w)
    pair_t<R>(*wr)[34] = (pair_t<R>(*)[34])(smem + Plan::kRhoOffset) + warp * 4;

    int2 rr = make_int2(ny, -1);
    {
        const int k0 = x0 / 64, k1 = min((x0 + BX + 63) / 64, (nx + 63) / 64);
        for (int k = k0; k < k1; k++) {
            const int2 q = rows64[k];
            rr.x = min(rr.x, q.x);
            rr.y = max(rr.y, q.y);
        }
    }
    const int nrows = rr.y - rr.x + 1;
    const int rpb = nrows > 0 ? (nrows + grid.strips - 1) / grid.strips : 0;
    const int y0 = rr.x + blockIdx.y * rpb;
    const int y1 = min(y0 + rpb, rr.y + 1);
    const bool empty_cta = nrows <= 0 || y0 >= y1;
    const int n_stage = empty_cta ? 0 : (y1 - y0) + 4;

    NodeParams<R> P;
    P.load(prm);

    const int gxc = x0 + t;
    const bool active = gxc < nx;
    const bool rho_col = gxc <= nx;
    const int wi = t + kGhost;
    // the warp's halo columns (window indices); the right one only when it is
    // a column some lane of this warp needs (<= nx)
    const int wl_left = warp * 32 + kGhost - 1;
    const int wl_right = warp * 32 + 32 + kGhost;
    const bool need_right = x0 + warp * 32 + 32 <= nx;
    const bool warp_live = x0 + warp * 32 <= nx;      // some lane of this warp owns a column <= nx

    auto slot = [&](int r) { return (r - y0 + 1) & 3; };

    bool timed_out = false;
    int next_issue = 0;
    auto issue = [&](int j) {
        uint64_t* bar = &full[j % NS];
        int row = (y0 - 2 + j) % ny;
        row = row < 0 ? row + ny : row;
        mbar_expect_tx(bar, Plan::kTxBytes);
        tma_load_3d((void*)pops(j), &fmap, x0, row, 0, bar);
        tma_load_2d((void*)lnks(j), &lmap, x0, row, bar);
    };
    // producer: issue every stage up to `upto` whose slot the warps released
    auto produce = [&](int upto) {
        while (next_issue <= upto && next_issue < n_stage) {
            if (next_issue >= NS && !timed_out &&
                !mbar_wait(&empty[next_issue % NS], (uint32_t)(((next_issue / NS) - 1) & 1)))
                timed_out = true;
            issue(next_issue++);
        }
    };
    auto wait_full = [&](int j) {
        if (!timed_out && !mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1))) timed_out = true;
    };
    // a warp is done with stage j: one arrival per warp
    auto release = [&](int j) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[j % NS]);
    };

    auto pull = [&](int jm, int jc, int jp, int w, R(&f)[2][9], R& r0, R& r1, R& l0, R& l1) -> bool {
        const unsigned lk = lnks(jc)[w];
        if (lk & kSolid) {
            r0 = P.rw0;
            r1 = P.rw1;
            l0 = l1 = R(0);
            return true;
        }
        const S* pm = pops(jm);
        const S* pc = pops(jc);
        const S* pp = pops(jp);
        if (lk == 0) {
            const S* q[9] = {pc + w, pc + w - 1, pm + w, pc + w + 1, pp + w, pm + w - 1, pm + w + 1, pp + w + 1,
                             pp + w - 1};
#pragma unroll
            for (int i = 0; i < 9; i++) {
                R r0s = R(0), r1s = R(0);
                if (C::kNodeShift) {
                    r0s = C::rho_value(q[i][18 * W]);
                    r1s = C::rho_value(q[i][19 * W]);
                }
                f[0][i] = C::decode(q[i][i * W], wgt<R>(i), r0s);
                f[1][i] = C::decode(q[i][(9 + i) * W], wgt<R>(i), r1s);
            }
        } else {
            const bool b1 = lk & (1u << 1), b2 = lk & (1u << 2), b3 = lk & (1u << 3), b4 = lk & (1u << 4);
            const bool b5 = lk & (1u << 5), b6 = lk & (1u << 6), b7 = lk & (1u << 7), b8 = lk & (1u << 8);
            const S* q[9];
            int pl[9];
            q[0] = pc + w;                        pl[0] = 0;
            q[1] = b1 ? pc + w : pc + w - 1;      pl[1] = b1 ? 3 : 1;
            q[2] = b2 ? pc + w : pm + w;          pl[2] = b2 ? 4 : 2;
            q[3] = b3 ? pc + w : pc + w + 1;      pl[3] = b3 ? 1 : 3;
            q[4] = b4 ? pc + w : pp + w;          pl[4] = b4 ? 2 : 4;
            q[5] = b5 ? pc + w : pm + w - 1;      pl[5] = b5 ? 7 : 5;
            q[6] = b6 ? pc + w : pm + w + 1;      pl[6] = b6 ? 8 : 6;
            q[7] = b7 ? pc + w : pp + w + 1;      pl[7] = b7 ? 5 : 7;
            q[8] = b8 ? pc + w : pp + w - 1;      pl[8] = b8 ? 6 : 8;
#pragma unroll
            for (int i = 0; i < 9; i++) {
                R r0s = R(0), r1s = R(0);
                if (C::kNodeShift) {
                    r0s = C::rho_value(q[i][18 * W]);
                    r1s = C::rho_value(q[i][19 * W]);
                }
                f[0][i] = C::decode(q[i][pl[i] * W], wgt<R>(i), r0s);
                f[1][i] = C::decode(q[i][(9 + pl[i]) * W], wgt<R>(i), r1s);
            }
        }
        density_of<C>(f[0], r0, l0);
        density_of<C>(f[1], r1, l1);
        return false;
    };

    // density of one halo column of this warp (window column w) into the
    // warp ring entry col (0 = left, 33 = right): lanes 0..8 species o,
    // lanes 16..24 species w
    auto halo_one = [&](int jm, int jc, int jp, int w, int sl, int col) {
        const unsigned lk = lnks(jc)[w];
        const int sp = lane >> 4, i = lane & 15;
        R v = R(0);
        if (!(lk & kSolid) && i < 9) {
            const S* q;
            int pln;
            if (lk & (1u << i)) {
                q = pops(jc) + w;
                pln = d2q9_opp(i);
            } else {
                const int cy = d2q9_cy(i);
                q = (cy > 0 ? pops(jm) : (cy < 0 ? pops(jp) : pops(jc))) + w - d2q9_cx(i);
                pln = i;
            }
            R rs = R(0);
            if (C::kNodeShift) rs = C::rho_value(q[(18 + sp) * W]);
            v = C::decode(q[(sp * 9 + pln) * W], wgt<R>(i), rs);
        }
        v = halfwarp_density<C>(v);
        if ((lane & 15) == 0) reinterpret_cast<R*>(&wr[sl][col])[sp] = (lk & kSolid) ? (sp ? P.rw1 : P.rw0) : v;
    };
    auto halos = [&](int jm, int jc, int jp, int sl) {
        if (!warp_live) return;
        halo_one(jm, jc, jp, wl_left, sl, 0);
        if (need_right) halo_one(jm, jc, jp, wl_right, sl, 33);
    };

    if (t == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    ObsLocal<R> ob;
    if (!empty_cta) {
        if (t == 0) produce(NS - 1);
        R cur[2][9], nxt[2][9];
        R rc0 = R(0), rc1 = R(0), rn0 = R(0), rn1 = R(0);
        R lc0 = R(0), lc1 = R(0), ln0 = R(0), ln1 = R(0);
        bool solid_cur = true, solid_nxt = true;
        const int c = lane + 1;                         // this lane's column in the warp ring

        // prologue: rows y0 - 1 (stages 0,1,2) and y0 (stages 1,2,3)
        wait_full(0);
        wait_full(1);
        wait_full(2);
        if (rho_col) {
            R tmp[2][9], a, b, la, lb;
            pull(0, 1, 2, wi, tmp, a, b, la, lb);
            wr[slot(y0 - 1)][c] = make_pair_of<R>(a, b);
        }
        halos(0, 1, 2, slot(y0 - 1));
        release(0);
        wait_full(3);
        if (rho_col) {
            solid_cur = pull(1, 2, 3, wi, cur, rc0, rc1, lc0, lc1);
            wr[slot(y0)][c] = make_pair_of<R>(rc0, rc1);
        }
        halos(1, 2, 3, slot(y0));
        release(1);

        for (int r = y0; r < y1; ++r) {
            const int j = r - y0 + 2;                   // stages j, j+1, j+2 hold rows r, r+1, r+2
            if (t == 0) produce(j - 1 + NS);
            const int sn = slot(r + 1);
            wait_full(j + 2);
            if (rho_col) {
                solid_nxt = pull(j, j + 1, j + 2, wi, nxt, rn0, rn1, ln0, ln1);
                wr[sn][c] = make_pair_of<R>(rn0, rn1);
            }
            halos(j, j + 1, j + 2, sn);
            release(j);                                  // includes the __syncwarp for the ring
            if (active && !solid_cur) {
                const int s0 = slot(r), sm = slot(r - 1), sp = sn;
                R nb[2][8];
                {
                    const pair_t<R> e = wr[s0][c + 1], n = wr[sp][c], wv = wr[s0][c - 1];
                    const pair_t<R> so = wr[sm][c], ne = wr[sp][c + 1], nw = wr[sp][c - 1];
                    const pair_t<R> sw = wr[sm][c - 1], se = wr[sm][c + 1];
                    nb[0][0] = e.x;  nb[1][0] = e.y;
                    nb[0][1] = n.x;  nb[1][1] = n.y;
                    nb[0][2] = wv.x; nb[1][2] = wv.y;
                    nb[0][3] = so.x; nb[1][3] = so.y;
                    nb[0][4] = ne.x; nb[1][4] = ne.y;
                    nb[0][5] = nw.x; nb[1][5] = nw.y;
                    nb[0][6] = sw.x; nb[1][6] = sw.y;
                    nb[0][7] = se.x; nb[1][7] = se.y;
                }
                collide_store<S, R>(cur, rc0, rc1, lc0, lc1, nb, P, fout + r * pitch + gxc, plane, gxc, nx,
                                    grid.periodic_x, ob);
            }
            // the ring slot of row r - 1 is rewritten two iterations later,
            // after this warp's next __syncwarp
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
    const bool any_timeout = __syncthreads_or(timed_out) != 0;
    if (any_timeout && t == 0) {
        for (int j = max(0, next_issue - NS); j < next_issue; j++) mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1));
    }
    reduce_observables<R, BX>(ob, acc, obs, any_timeout);
}

}  // namespace gb300lbm
