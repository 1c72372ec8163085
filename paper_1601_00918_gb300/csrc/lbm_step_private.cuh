// Two-component D2Q9 time step, "private" variant: every warp stages, pulls,
// collides and stores its own 32 columns with no other warp involved.
//
// Same method as the staged variant (lbm_step_tma.cuh).  The staged variant
// shares one row ring per CTA and needs a CTA barrier per row (the
// densities of a row are read by the neighbouring threads, and the ring
// slot can be refilled only when every warp is done with it).  Here each
// warp owns:
//   - a ring of D + 3 row stages holding only the columns its pulls reach
//     (x0w - 2 .. x0w + 33, widened to the 16-byte TMA alignment), filled by
//     its lane 0 with one cp.async.bulk.tensor box of all planes plus one
//     box of link words per row;
//   - its halo densities: lanes 0 and 31 also pull the columns x0w - 1 and
//     x0w + 32 (density only);
//   - its density exchange: the densities of columns x +- 1 come from the
//     neighbouring lanes by shuffles, those of the warp's edges from the halo
//     lanes, the rows above and below stay in registers.
// So the only synchronisation in the row loop is the wait on the stage's
// mbarrier and a __syncwarp before lane 0 refills the slot it just freed.
// The loop is unrolled by two rows so that the populations pulled for the
// next row and those of the row being collided swap roles without copies.
//
// Every wait is bounded; a warp whose wait gives up marks the step
// (ObsState.timeout_flag), issues no further copies and, before the CTA
// exits, waits (bounded) for the copies it still has in flight.
#pragma once

#include "lbm_step_tma.cuh"

namespace gb300lbm {

// Shared-memory plan of the private kernel (host and device agree on it).
// A warp owns columns [x0w, x0w + 32) with x0w a multiple of 32; logical
// column c sits at element c + kGhost of a row.  The population window
// starts kLead columns before x0w so that its first element is 16-byte
// aligned; the link window (2-byte words) starts 8 columns before x0w.
template <typename S, int NWARP, int D>
struct PrivatePlan {
    static constexpr int kLead = sizeof(S) == 8 ? 2 : (sizeof(S) == 4 ? 4 : 8);
    static constexpr int kAlign = 16 / (int)sizeof(S);
    static constexpr int kW = (kLead + 34 + kAlign - 1) / kAlign * kAlign;   // 36 / 40 / 48 columns
    static constexpr int kLinkLead = 8;
    static constexpr int kLW = 48;                                          // x0w - 8 .. x0w + 39
    static constexpr int kStages = D + 3;
    static constexpr int kPlanes = Codec<S>::kPlanes;
    static constexpr int kPopBytes = kPlanes * kW * (int)sizeof(S);
    static constexpr int kPopSlot = (kPopBytes + 127) / 128 * 128;
    static constexpr int kLinkSlot = (kLW * 2 + 127) / 128 * 128;
    static constexpr int kSlot = kPopSlot + kLinkSlot;
    static constexpr int kWarpBytes = kStages * kSlot;
    static constexpr int kBarOffset = NWARP * kWarpBytes;
    static constexpr int kBytes = kBarOffset + ((NWARP * kStages * 8 + 127) / 128) * 128 + 128;
    static constexpr uint32_t kTxBytes = (uint32_t)(kPopBytes + kLW * 2);
};

// One time step fin -> fout.  fmap views fin as [planes][ny][pitch] with a
// box of {kW, 1, planes}; lmap views the link words as [ny][pitch] with a
// box of {kLW, 1}.  fout points at logical column 0 of row 0.  rows64[k] =
// (first, last) row with fluid in columns [64 k, 64 k + 64).
template <typename S, int BX, int D>
__global__ void __launch_bounds__(BX, sizeof(S) == 8 ? 2 : (BX == 64 ? 8 : 4))
    step_private_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap lmap,
                        S* __restrict__ fout, const int2* __restrict__ rows64,
                        const StepParams* __restrict__ prm, ObsAccum* __restrict__ acc,
                        ObsState* __restrict__ obs, Grid grid) {
    using C = Codec<S>;
    using R = typename C::R;
    constexpr int NW = BX / 32;
    using Plan = PrivatePlan<S, NW, D>;
    constexpr int W = Plan::kW;
    constexpr int NS = Plan::kStages;
    constexpr int L = Plan::kLead;
    constexpr int LL = Plan::kLinkLead;
    constexpr unsigned kSolid = 1u << kSolidBit;
    constexpr unsigned kAll = 0xffffffffu;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned start, found in the shared window itself: pointer
    // arithmetic on the __shared__ array keeps every access a shared one
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    unsigned char* wbase = smem + warp * Plan::kWarpBytes;
    uint64_t* full = (uint64_t*)(smem + Plan::kBarOffset) + warp * NS;
    auto pops = [&](int stage) { return (const S*)(wbase + (stage % NS) * Plan::kSlot); };
    auto lnks = [&](int stage) { return (const uint16_t*)(wbase + (stage % NS) * Plan::kSlot + Plan::kPopSlot); };

    const int nx = grid.nx, ny = grid.ny, pitch = grid.pitch;
    const int plane = ny * pitch;
    const int x0w = blockIdx.x * BX + warp * 32;
    const int gxc = x0w + lane;
    const bool active = gxc < nx;
    const bool warp_live = x0w < nx;
    const bool need_right = x0w + 32 <= nx;         // lane 31 collides: column x0w + 32 is needed

    // this warp's strip of the fluid rows of its columns (all in one 64-column entry)
    const int2 rr = warp_live ? rows64[x0w / 64] : make_int2(ny, -1);
    const int nrows = rr.y - rr.x + 1;
    const int rps = nrows > 0 ? (nrows + grid.strips - 1) / grid.strips : 0;
    const int y0 = rr.x + blockIdx.y * rps;
    const int y1 = min(y0 + rps, rr.y + 1);
    const bool idle = !warp_live || nrows <= 0 || y0 >= y1;
    const int n_stage = idle ? 0 : (y1 - y0) + 4;   // rows y0 - 2 .. y1 + 1

    NodeParams<R> P;
    P.load(prm);

    const int wi = lane + L;                        // own column in the population window
    const int li = lane + LL;                       // own column in the link window
    const bool halo_lane = lane == 0 || (lane == 31 && need_right);
    const int hw = lane == 0 ? L - 1 : L + 32;      // halo column (lanes 0 and 31)
    const int hl = lane == 0 ? LL - 1 : LL + 32;

    bool timed_out = false;                         // warp-uniform
    int next_issue = 0;                             // lane 0 only: next stage to issue
    int next_row = (y0 - 2) % ny;                   // lane 0 only: its row (stage j holds row y0 - 2 + j mod ny)
    next_row = next_row < 0 ? next_row + ny : next_row;
    auto issue = [&]() {
        const int j = next_issue++;
        uint64_t* bar = &full[j % NS];
        mbar_expect_tx(bar, Plan::kTxBytes);
        tma_load_3d((void*)pops(j), &fmap, x0w - L + kGhost, next_row, 0, bar);
        tma_load_2d((void*)lnks(j), &lmap, x0w - LL + kGhost, next_row, bar);
        next_row = next_row + 1 == ny ? 0 : next_row + 1;
    };
    auto wait_full = [&](int j) {
        if (!timed_out) timed_out = __any_sync(kAll, !mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1))) != 0;
    };

    // Pull the populations of the row held by stage jc (rows above/below in
    // jm/jp) at population column w / link column lw.  True at a solid node,
    // whose "density" is the wall potential; l0, l1 receive the low parts of
    // the density sums (density_of).
    auto pull = [&](int jm, int jc, int jp, int w, int lw, R(&f)[2][9], R& r0, R& r1, R& l0, R& l1) -> bool {
        const unsigned lk = lnks(jc)[lw];
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
            // interior node: every population comes from its upwind neighbour
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
            // bounced populations come from the node itself, direction opp(i)
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

    // density only, for the halo columns: the same sources and the same sum
    // (density_of) as pull()
    auto pull_rho = [&](int jm, int jc, int jp, int w, int lw, R& r0, R& r1) {
        const unsigned lk = lnks(jc)[lw];
        if (lk & kSolid) {
            r0 = P.rw0;
            r1 = P.rw1;
            return;
        }
        const S* rows[3] = {pops(jm), pops(jc), pops(jp)};
        R g[2][9];
        if (lk == 0) {
            // interior node
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const S* q = rows[1 - d2q9_cy(i)] + w - d2q9_cx(i);
                R r0s = R(0), r1s = R(0);
                if (C::kNodeShift) {
                    r0s = C::rho_value(q[18 * W]);
                    r1s = C::rho_value(q[19 * W]);
                }
                g[0][i] = C::decode(q[i * W], wgt<R>(i), r0s);
                g[1][i] = C::decode(q[(9 + i) * W], wgt<R>(i), r1s);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const bool bb = (lk >> i) & 1u;             // bit 0 is never set: the rest population stays
                const S* q = bb ? rows[1] + w : rows[1 - d2q9_cy(i)] + w - d2q9_cx(i);
                const int pl = bb ? d2q9_opp(i) : i;
                R r0s = R(0), r1s = R(0);
                if (C::kNodeShift) {
                    r0s = C::rho_value(q[18 * W]);
                    r1s = C::rho_value(q[19 * W]);
                }
                g[0][i] = C::decode(q[pl * W], wgt<R>(i), r0s);
                g[1][i] = C::decode(q[(9 + pl) * W], wgt<R>(i), r1s);
            }
        }
        R l0, l1;
        density_of<C>(g[0], r0, l0);
        density_of<C>(g[1], r1, l1);
    };

    if (lane == 0) {
        for (int s = 0; s < NS; s++) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    ObsLocal<R> ob;
    if (!idle) {
        if (lane == 0)
            while (next_issue < NS && next_issue < n_stage) issue();
        R fa[2][9], fb[2][9];
        // densities of this lane's column (and of the halo column on lanes
        // 0 and 31) in rows r - 1, r, r + 1 of the row being collided
        R rm0 = R(0), rm1 = R(0), rc0 = R(0), rc1 = R(0), rn0 = R(0), rn1 = R(0);
        R hm0 = R(0), hm1 = R(0), hc0 = R(0), hc1 = R(0), hn0 = R(0), hn1 = R(0);
        R lc0 = R(0), lc1 = R(0), ln0 = R(0), ln1 = R(0);
        bool sa = true, sb = true;

        // prologue: densities of rows y0 - 1 (stages 0, 1, 2) and y0 (1, 2, 3)
        wait_full(0);
        wait_full(1);
        wait_full(2);
        pull_rho(0, 1, 2, wi, li, rm0, rm1);
        if (halo_lane) pull_rho(0, 1, 2, hw, hl, hm0, hm1);
        wait_full(3);
        sa = pull(1, 2, 3, wi, li, fa, rc0, rc1, lc0, lc1);
        if (halo_lane) pull_rho(1, 2, 3, hw, hl, hc0, hc1);
        // stages 0 and 1 are done: refill their slots
        __syncwarp();
        if (lane == 0 && !timed_out)
            while (next_issue <= NS + 1 && next_issue < n_stage) issue();

        auto from_right = [&](R own, R halo) {
            const R v = __shfl_down_sync(kAll, own, 1);
            return lane == 31 ? halo : v;
        };
        auto from_left = [&](R own, R halo) {
            const R v = __shfl_up_sync(kAll, own, 1);
            return lane == 0 ? halo : v;
        };

        // row r: pull row r + 1 into nxt, then collide row r from cur
        auto row_step = [&](int r, R(&cur)[2][9], R(&nxt)[2][9], bool s_cur, bool& s_nxt) {
            const int j = r - y0 + 2;                   // stages j, j+1, j+2 hold rows r, r+1, r+2
            wait_full(j + 2);
            rn0 = rn1 = R(0);
            hn0 = hn1 = R(0);
            s_nxt = true;
            s_nxt = pull(j, j + 1, j + 2, wi, li, nxt, rn0, rn1, ln0, ln1);
            if (halo_lane) pull_rho(j, j + 1, j + 2, hw, hl, hn0, hn1);
            // stage j (row r) is no longer read: lane 0 refills its slot
            __syncwarp();
            if (lane == 0 && !timed_out && next_issue <= j + NS && next_issue < n_stage) issue();
            R nb[2][8];
            nb[0][0] = from_right(rc0, hc0);  nb[1][0] = from_right(rc1, hc1);   // (x + 1, r)
            nb[0][1] = rn0;                   nb[1][1] = rn1;                    // (x, r + 1)
            nb[0][2] = from_left(rc0, hc0);   nb[1][2] = from_left(rc1, hc1);    // (x - 1, r)
            nb[0][3] = rm0;                   nb[1][3] = rm1;                    // (x, r - 1)
            nb[0][4] = from_right(rn0, hn0);  nb[1][4] = from_right(rn1, hn1);   // (x + 1, r + 1)
            nb[0][5] = from_left(rn0, hn0);   nb[1][5] = from_left(rn1, hn1);    // (x - 1, r + 1)
            nb[0][6] = from_left(rm0, hm0);   nb[1][6] = from_left(rm1, hm1);    // (x - 1, r - 1)
            nb[0][7] = from_right(rm0, hm0);  nb[1][7] = from_right(rm1, hm1);   // (x + 1, r - 1)
            if (active && !s_cur)
                collide_store<S, R>(cur, rc0, rc1, lc0, lc1, nb, P, fout + r * pitch + gxc, plane, gxc, nx, grid.periodic_x,
                                    ob);
            rm0 = rc0;
            rm1 = rc1;
            rc0 = rn0;
            rc1 = rn1;
            lc0 = ln0;
            lc1 = ln1;
            hm0 = hc0;
            hm1 = hc1;
            hc0 = hn0;
            hc1 = hn1;
        };

        int r = y0;
        for (; r + 1 < y1; r += 2) {
            row_step(r, fa, fb, sa, sb);
            row_step(r + 1, fb, fa, sb, sa);
        }
        if (r < y1) row_step(r, fa, fb, sa, sb);
    }
    const bool any_timeout = __syncthreads_or(timed_out) != 0;
    if (any_timeout && lane == 0 && !idle) {
        // a wait gave up somewhere: let this warp's copies still in flight land before exit
        for (int j = max(0, next_issue - NS); j < next_issue; j++) mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1));
    }
    reduce_observables<R, BX>(ob, acc, obs, any_timeout);
}

}  // namespace gb300lbm
