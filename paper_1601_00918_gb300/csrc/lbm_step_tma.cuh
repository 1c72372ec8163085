// Two-component D2Q9 time step, "staged" variant: rows of all 18 population
// planes are moved from HBM to shared memory by the Tensor Memory Accelerator.
//
// Same method and same marching structure as the simple variant (see
// lbm_step.cuh): a CTA owns BX columns and marches down a strip of rows,
// pulling row r + 1 while colliding row r.  The difference is where the
// pulled values come from.  One elected thread keeps D + 3 row stages in a
// shared-memory ring: each stage is ONE cp.async.bulk.tensor.3d copy of a
// box {BX + 16 columns, 1 row, all planes} plus one 2-D copy of the row's
// link words, both completing on the stage's mbarrier (the 16-bit formats
// stage 20 planes: their two density planes ride in the same box).  Stages are issued up
// to D rows ahead, so the loads of the next rows are in flight while the
// CTA computes; the pull itself (with bounce-back) reads shared memory.  The
// 8-column ghost margins of the layout make every box a plain rectangle:
// periodic wrap in x needs no patch, and rows wrap in y by coordinate.
//
// Each column block only stages and marches over the rows that contain
// fluid in its columns (a per-block row range computed at set-up), so the
// solid bands of a channel are neither read nor written.
//
// Every wait on an mbarrier is bounded; a wait that gives up marks the step
// (ObsState.timeout_flag) and the CTA carries on to its end without hanging
// the barriers of the other threads, then waits (bounded) for its own copies
// in flight before it exits.
#pragma once

#include <cuda.h>

#include "lbm_common.cuh"

namespace gb300lbm {

// A waiting thread is suspended for up to kSuspendNs per poll (it resumes as
// soon as the phase completes, and the hardware may resume it earlier), so
// waits do not burn issue slots; after kWaitLimit polls the wait gives up
// (about 0.5 s on GB300, measured by lbm_wait_selftest; a row copy takes
// microseconds).
constexpr unsigned kSuspendNs = 20000;
constexpr unsigned kWaitLimit = 1u << 17;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the phase did not complete within kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

// Shared-memory plan of the staged kernel (host and device agree on it).
// Pulls and halo densities reach two columns beyond each side of the block.
// The population window starts kLead columns before it, so that its first
// element is 16-byte aligned (4 columns for 4- and 8-byte types, 8 for the
// 2-byte ones); the link window (2-byte words) starts 8 columns before.
template <typename S, int BX, int D>
struct StagedPlan {
    static constexpr int kLead = sizeof(S) == 2 ? 8 : 4;
    static constexpr int kW = BX + 2 * kLead;             // staged population columns per row
    static constexpr int kLinkLead = 8;
    static constexpr int kLW = BX + 2 * kLinkLead;        // staged link-word columns per row
    static constexpr int kStages = D + 3;                 // ring: rows r..r+2 in use + D ahead
    static constexpr int kPlanes = Codec<S>::kPlanes;        // 18, or 20 with the density planes
    static constexpr int kPopBytes = kPlanes * kW * (int)sizeof(S);
    static constexpr int kPopSlot = (kPopBytes + 127) / 128 * 128;
    static constexpr int kLinkSlot = (kLW * 2 + 127) / 128 * 128;
    static constexpr int kSlot = kPopSlot + kLinkSlot;
    static constexpr int kRhoBytes = 4 * 2 * (BX + 2) * (int)sizeof(typename Codec<S>::R);
    static constexpr int kBarOffset = kStages * kSlot;
    static constexpr int kRhoOffset = kBarOffset + ((kStages * 8 + 127) / 128) * 128;
    static constexpr int kBytes = kRhoOffset + kRhoBytes + 128;   // + alignment slack
    static constexpr uint32_t kTxBytes = (uint32_t)(kPopBytes + kLW * 2);
};

// One CTA's march over the rows [y0, y1) of the BX columns starting at x0,
// in direction dir (+1: increasing y), for one time step fin -> fout.  fmap
// views fin as [planes][ny][pitch] (box {kW, 1, planes}), lmap views the link
// words as [ny][pitch] (box {kLW, 1}); either may live in kernel parameter
// space or in global memory (written before the launch).  fout
// points at logical column 0 of row 0.  y0 >= y1: nothing to do.  Returns
// (uniformly over the CTA) whether a bounded wait gave up; the caller
// reduces the observables gathered in ob.  kReg picks the collision as in
// collide_store (-1: at run time from prm).
template <typename S, int BX, int D, int kReg = -1>
__device__ __forceinline__ bool staged_march(const CUtensorMap* fmap, const CUtensorMap* lmap,
                                             S* __restrict__ fout, const StepParams* __restrict__ prm, int nx,
                                             int ny, int pitch, int periodic_x, int x0, int y0, int y1, int dir,
                                             ObsLocal<typename Codec<S>::R>& ob) {
    using C = Codec<S>;
    using R = typename C::R;
    using Plan = StagedPlan<S, BX, D>;
    constexpr int W = Plan::kW;
    constexpr int NS = Plan::kStages;
    constexpr unsigned kSolid = 1u << kSolidBit;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned start, found in the shared window itself: pointer
    // arithmetic on the __shared__ array keeps every access a shared one
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* bars = (uint64_t*)(smem + Plan::kBarOffset);
    pair_t<R>(*s_rho)[BX + 2] = (pair_t<R>(*)[BX + 2])(smem + Plan::kRhoOffset);
    // stage indices are never negative: unsigned arithmetic keeps the ring
    // index a plain mask (or a multiply-shift for rings of 3 or 5 slots)
    auto pops = [&](int stage) { return (const S*)(smem + ((unsigned)stage % NS) * Plan::kSlot); };
    auto lnks = [&](int stage) {
        return (const uint16_t*)(smem + ((unsigned)stage % NS) * Plan::kSlot + Plan::kPopSlot);
    };

    const int plane = ny * pitch;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const bool empty = y0 >= y1;
    const int n_stage = empty ? 0 : (y1 - y0) + 4;   // rows y0 - 2 .. y1 + 1

    NodeParams<R> P;
    P.load(prm);

    const int gxc = x0 + t;
    const bool active = gxc < nx;
    const int wi = t + Plan::kLead;                 // this thread's column in the population window
    const int li = t + Plan::kLinkLead;             // ... and in the link window

    // Stage j holds the row first + dir (j - 2); the density ring is indexed
    // by the (unwrapped) row.
    const int first = dir > 0 ? y0 : y1 - 1;
    auto slot = [&](int r) { return r & 3; };
    // stages of the rows below (y - 1) and above (y + 1) the row of stage j + 1
    auto below = [&](int j) { return dir > 0 ? j : j + 2; };
    auto above = [&](int j) { return dir > 0 ? j + 2 : j; };

    bool timed_out = false;
    int next_issue = 0;                             // thread 0 only: next stage to issue
    int next_row = (first - 2 * dir) % ny;          // thread 0 only: the row of stage next_issue
    next_row = next_row < 0 ? next_row + ny : next_row;
    auto issue = [&]() {
        const int j = next_issue++;
        uint64_t* bar = &bars[(unsigned)j % NS];
        mbar_expect_tx(bar, Plan::kTxBytes);
        tma_load_3d((void*)pops(j), fmap, x0 + kGhost - Plan::kLead, next_row, 0, bar);
        tma_load_2d((void*)lnks(j), lmap, x0 + kGhost - Plan::kLinkLead, next_row, bar);
        next_row += dir;
        next_row = next_row == ny ? 0 : (next_row < 0 ? ny - 1 : next_row);
    };
    // after one wait gave up the data is invalid anyway: skip the others
    auto wait_stage = [&](int j) {
        if (!timed_out && !mbar_wait(&bars[(unsigned)j % NS], ((unsigned)j / NS) & 1u)) timed_out = true;
    };

    // Pull the populations of the row held by stage jc (rows above/below in
    // jm/jp) at population window column w / link window column lw.  Returns
    // true at a solid node; r0, r1 (l0, l1) receive the densities (their low
    // parts, density_of).
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
        // (plane, stage, column) of each pulled population; bounced: own opp(i)
        const bool b1 = lk & (1u << 1), b2 = lk & (1u << 2), b3 = lk & (1u << 3), b4 = lk & (1u << 4);
        const bool b5 = lk & (1u << 5), b6 = lk & (1u << 6), b7 = lk & (1u << 7), b8 = lk & (1u << 8);
        const S* rowp[9];
        int col[9], pl[9];
        rowp[0] = pc; col[0] = w;                     pl[0] = 0;
        rowp[1] = pc; col[1] = b1 ? w : w - 1;        pl[1] = b1 ? 3 : 1;
        rowp[2] = b2 ? pc : pm; col[2] = w;           pl[2] = b2 ? 4 : 2;
        rowp[3] = pc; col[3] = b3 ? w : w + 1;        pl[3] = b3 ? 1 : 3;
        rowp[4] = b4 ? pc : pp; col[4] = w;           pl[4] = b4 ? 2 : 4;
        rowp[5] = b5 ? pc : pm; col[5] = b5 ? w : w - 1; pl[5] = b5 ? 7 : 5;
        rowp[6] = b6 ? pc : pm; col[6] = b6 ? w : w + 1; pl[6] = b6 ? 8 : 6;
        rowp[7] = b7 ? pc : pp; col[7] = b7 ? w : w + 1; pl[7] = b7 ? 5 : 7;
        rowp[8] = b8 ? pc : pp; col[8] = b8 ? w : w - 1; pl[8] = b8 ? 6 : 8;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const S* q = rowp[i] + col[i];
            R r0s = R(0), r1s = R(0);
            if (C::kNodeShift) {
                r0s = C::rho_value(q[18 * W]);
                r1s = C::rho_value(q[19 * W]);
            }
            f[0][i] = C::decode(q[pl[i] * W], wgt<R>(i), r0s);
            f[1][i] = C::decode(q[(9 + pl[i]) * W], wgt<R>(i), r1s);
        }
        }
        density_of<C>(f[0], r0, l0);
        density_of<C>(f[1], r1, l1);
        return false;
    };

    // Densities of the halo columns x0 - 1 (warp 0) and x0 + BX (warp 1),
    // lanes 0..8 species o, lanes 16..24 species w, from the staged window.
    auto halo = [&](int jm, int jc, int jp, int sl) {
        // the last two warps: warp 0 also issues the row copies, so the
        // extra work of a row is spread over three warps
        if (warp < BX / 32 - 2) return;
        const bool right = warp == BX / 32 - 1;
        if (right && x0 + BX > nx) return;          // image column pulled by a thread instead
        const int w = right ? BX + Plan::kLead : Plan::kLead - 1;
        const unsigned lk = lnks(jc)[right ? BX + Plan::kLinkLead : Plan::kLinkLead - 1];
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
        if ((lane & 15) == 0)
            reinterpret_cast<R*>(&s_rho[sl][right ? BX + 1 : 0])[sp] = (lk & kSolid) ? (sp ? P.rw1 : P.rw0) : v;
    };

    if (t == 0) {
        for (int s = 0; s < NS; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    if (!empty) {
        if (t == 0) {
            while (next_issue < NS && next_issue < n_stage) issue();
        }
        R fa[2][9], fb[2][9];
        R rc0 = R(0), rc1 = R(0), rn0 = R(0), rn1 = R(0);
        R lc0 = R(0), lc1 = R(0), ln0 = R(0), ln1 = R(0);
        bool sa = true, sb = true;

        // prologue: densities of the rows first - dir (stage 1) and first (stage 2)
        wait_stage(0);
        wait_stage(1);
        wait_stage(2);
        // every thread pulls (its window column always exists); densities of
        // columns beyond nx are read only by threads that do not collide
        {
            R a, b, la, lb;
            pull(below(0), 1, above(0), wi, li, fb, a, b, la, lb);
            s_rho[slot(first - dir)][t + 1] = make_pair_of<R>(a, b);
        }
        halo(below(0), 1, above(0), slot(first - dir));
        if constexpr (D == 0) {
            // a ring of three slots: stage 3 goes into the slot of stage 0,
            // which the pull above has just read
            __syncthreads();
            if (t == 0 && !timed_out && next_issue < n_stage) issue();
        }
        wait_stage(3);
        sa = pull(below(1), 2, above(1), wi, li, fa, rc0, rc1, lc0, lc1);
        s_rho[slot(first)][t + 1] = make_pair_of<R>(rc0, rc1);
        halo(below(1), 2, above(1), slot(first));
        // stages 0 and 1 are no longer needed: refill their slots now, so
        // that stage 4 (the first one the loop waits for) is on its way even
        // with a ring of only D + 3 = 4 slots
        __syncthreads();
        if (t == 0 && !timed_out) {
            while (next_issue <= 1 + NS && next_issue < n_stage) issue();
        }

        // k-th row of the march, r = first + dir k: pull row r + dir into nxt,
        // then collide row r from cur.  The loop below is not unrolled: the
        // copy of nxt into cur costs less than the instruction-cache misses
        // of a loop body twice the size, with five CTAs per SM.
        auto row_step = [&](int k, R(&cur)[2][9], R(&nxt)[2][9], bool s_cur, bool& s_nxt) {
            const int r = first + dir * k;
            const int j = k + 2;                      // stages j, j+1, j+2 hold rows r, r+dir, r+2dir
            const int sn = slot(r + dir);
            wait_stage(j + 2);
            s_nxt = pull(below(j), j + 1, above(j), wi, li, nxt, rn0, rn1, ln0, ln1);
            s_rho[sn][t + 1] = make_pair_of<R>(rn0, rn1);
            halo(below(j), j + 1, above(j), sn);
            __syncthreads();
            // every stage <= j is now free: refill the ring
            if (t == 0 && !timed_out) {
                while (next_issue <= j + NS && next_issue < n_stage) issue();
            }
            if (active && !s_cur) {
                const int s0 = slot(r), sm = slot(r - 1), sp = slot(r + 1);
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
                collide_store<S, R, kReg>(cur, rc0, rc1, lc0, lc1, nb, P, fout + r * pitch + gxc, plane, gxc, nx,
                                    periodic_x, ob);
            }
            rc0 = rn0;
            rc1 = rn1;
            lc0 = ln0;
            lc1 = ln1;
        };

        const int nk = y1 - y0;
        int k = 0;
#pragma unroll 1
        for (; k < nk; ++k) {
            row_step(k, fa, fb, sa, sb);
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int i = 0; i < 9; i++) fa[a][i] = fb[a][i];
            sa = sb;
        }
    }
    const bool any_timeout = __syncthreads_or(timed_out) != 0;
    if (any_timeout && t == 0) {
        // a wait gave up: let the copies still in flight land before exit
        for (int j = max(0, next_issue - NS); j < next_issue; j++) mbar_wait(&bars[j % NS], (uint32_t)((j / NS) & 1));
    }
    return any_timeout;
}

// One time step fin -> fout of one grid: CTA (bx, by) marches over strip by
// of column block bx.  fmap / lmap as in staged_march; rows64[k] = (first,
// last) row with fluid in columns [64 k, 64 k + 64); a CTA of BX columns
// merges BX / 64 of them.
// Resident CTAs per SM the register budget is sized for: FP32 at 128 columns
// fits five CTAs one row ahead (96 registers without spills, 45.4 KB of
// shared memory each) and six with no row ahead (80 registers, 34.7 KB); the
// 16-bit formats five (96 registers; at six they spill and run slower), FP32
// two rows ahead four, FP64 two.
template <typename S, int BX, int D>
constexpr int staged_min_ctas() {
    return sizeof(S) == 8 ? 2 : (BX == 64 ? 8 : (sizeof(S) == 4 ? (D == 0 ? 6 : (D == 1 ? 5 : 4)) : 5));
}

// kReg: the collision, fixed at compile time (0 plain BGK, 1 regularised).
template <typename S, int BX, int D, int kReg>
__global__ void __launch_bounds__(BX, staged_min_ctas<S, BX, D>())
    step_staged_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap lmap,
                       S* __restrict__ fout, const int2* __restrict__ rows64, const StepParams* __restrict__ prm,
                       ObsAccum* __restrict__ acc, ObsState* __restrict__ obs, Grid grid) {
    using R = typename Codec<S>::R;
    const int nx = grid.nx, ny = grid.ny;
    const int x0 = blockIdx.x * BX;

    // this CTA's strip of the block's fluid rows
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
    int y0, y1;
    if (grid.strip_rows > 0) {
        // strips at the same absolute rows in every column block: neighbouring
        // blocks (adjacent in launch order) march over the same rows at the
        // same time, so the window columns they share come from L2
        y0 = max(rr.x, (int)blockIdx.y * grid.strip_rows);
        y1 = min(rr.y + 1, ((int)blockIdx.y + 1) * grid.strip_rows);
    } else {
        const int rpb = nrows > 0 ? (nrows + grid.strips - 1) / grid.strips : 0;
        y0 = rr.x + blockIdx.y * rpb;
        y1 = min(y0 + rpb, rr.y + 1);
    }
    // Odd strips march upwards: a boundary between two strips is then
    // reached by both of them at the same time (both start there or both
    // end there), so its rows are read from DRAM once and from L2 the
    // second time.
    const int dir = (blockIdx.y & 1) ? -1 : 1;
    ObsLocal<R> ob;
    const bool any_timeout = staged_march<S, BX, D, kReg>(&fmap, &lmap, fout, prm, nx, ny, grid.pitch,
                                                          grid.periodic_x, x0, y0, y1, dir, ob);
    reduce_observables<R, BX>(ob, acc, obs, any_timeout);
}

}  // namespace gb300lbm
