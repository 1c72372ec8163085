/*
 * Oracle for the two-component D2Q9 lattice-Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement
 * of what one time step computes.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product library never
 * links, loads or calls it, and it shares no code, table or header with the
 * CUDA path.
 *
 * What it follows (Otomo et al., "Simulation of residual oil displacement in
 * a sinusoidal channel with the lattice Boltzmann method", Section 2):
 *   - Eq. (basic_LBM_eq) and the rearranged BGK update Eq. (LBM_BGK):
 *         f_i(x + c_i, t + 1) = f_i^eq(rho, u) + (1 - 1/tau_mix) f'_i
 *     read with the force carried by the equilibrium velocity shift
 *     Eq. (collision_term), so the separate F_i term is zero and the
 *     non-equilibrium part is f'_i = f_i - f_i^eq(rho, u_mix) (plain BGK,
 *     collision = 0) or its regularised projection Eq. (Regualize) onto the
 *     second-order Hermite polynomials (collision = 1);
 *   - the mixture relaxation time tau_mix = nu_mix/T0 + 1/2 with
 *     nu_mix = (rho^o nu^o + rho^w nu^w)/(rho^o + rho^w) and T0 = 1/3;
 *   - the third-order equilibrium Eq. (feq) (second order as an option);
 *   - the inter-component force Eq. (comp_interaction),
 *         F^{a,b}(x) = G rho^a(x) sum_i w_i c_i rho^b(x + c_i),
 *     with the wall potentials rho_s^o, rho_s^w standing in for the density
 *     of a solid neighbour (end of Section 2);
 *   - the mixture velocity u_mix = (j^o + j^w)/(rho^o + rho^w);
 *   - the homogeneous body force of Section 3.4 (acceleration g on every
 *     species, force rho^a g);
 *   - walls: halfway bounce-back on a node mask (a population that would be
 *     pulled from a solid node is replaced by the node's own post-collision
 *     population in the opposite direction).
 *
 * Storage convention: f holds the post-collision populations f*_i^a(x, t),
 * index ((a*9 + i)*ny + y)*nx + x.  One step pulls them (streaming with
 * bounce-back), takes densities, forces and moments of the pulled state, and
 * collides, producing f*(t + 1).  Solid nodes hold zeros and are never read.
 *
 * Lattice: c_0 = (0,0); c_1..c_4 = (1,0),(0,1),(-1,0),(0,-1);
 * c_5..c_8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36.
 * A direction that is not periodic must have solid nodes on both of its
 * boundary lines; indices always wrap, so that rule keeps every pull and
 * every force neighbour of a fluid node inside the grid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    double tau[2];      /* tau^o, tau^w */
    double G;           /* interaction strength; repulsive when G < 0 */
    double rho_wall[2]; /* rho_s^o, rho_s^w */
    double g[2];        /* body-force acceleration (x, y) */
    int32_t eq_order;   /* 3: Eq. (feq) as printed; 2: drop the cubic terms */
    int32_t collision;  /* 0: f' = f - f^eq (BGK); 1: f' regularised, Eq. (Regualize) */
} oracle_params;

static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double T0 = 1.0 / 3.0;

static int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

static size_t fidx(const oracle_params *p, int a, int i, int x, int y) {
    return (((size_t)a * 9 + (size_t)i) * (size_t)p->ny + (size_t)y) * (size_t)p->nx + (size_t)x;
}

static int is_solid(const oracle_params *p, const uint8_t *solid, int x, int y) {
    return solid[(size_t)wrap(y, p->ny) * p->nx + wrap(x, p->nx)] != 0;
}

/* 0 when the mask obeys the boundary rule above, -1 otherwise. */
int oracle_check(const oracle_params *p, const uint8_t *solid) {
    if (p->nx < 1 || p->ny < 1) return -1;
    if (p->collision != 0 && p->collision != 1) return -1;
    if (!p->periodic_x)
        for (int y = 0; y < p->ny; y++)
            if (!solid[(size_t)y * p->nx] || !solid[(size_t)y * p->nx + p->nx - 1]) return -1;
    if (!p->periodic_y)
        for (int x = 0; x < p->nx; x++)
            if (!solid[x] || !solid[(size_t)(p->ny - 1) * p->nx + x]) return -1;
    return 0;
}

/* Eq. (feq): rho w_i [1 + c.u/T0 + (c.u)^2/(2T0^2) - u^2/(2T0)
 *                     + (c.u)^3/(6T0^3) - (c.u) u^2/(2T0^2)]. */
void oracle_feq(int order, double rho, double ux, double uy, double *out) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        double b = 1.0 + cu / T0 + cu * cu / (2.0 * T0 * T0) - uu / (2.0 * T0);
        if (order >= 3) b += cu * cu * cu / (6.0 * T0 * T0 * T0) - cu * uu / (2.0 * T0 * T0);
        out[i] = W[i] * rho * b;
    }
}

/* Initial stored state: f*_i = f_i^eq(rho_init, 0) = w_i rho_init at fluid
 * nodes, zero at solid nodes.  rho_init is [2][ny][nx]. */
void oracle_init(const oracle_params *p, const uint8_t *solid, const double *rho_init, double *f) {
    size_t n = (size_t)p->nx * p->ny;
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < 9; i++)
            for (int y = 0; y < p->ny; y++)
                for (int x = 0; x < p->nx; x++) {
                    size_t k = (size_t)y * p->nx + x;
                    f[fidx(p, a, i, x, y)] = solid[k] ? 0.0 : W[i] * rho_init[a * n + k];
                }
}

/* Streaming with halfway bounce-back: the population of direction i arriving
 * at (x, y) left (x - c_i, y - c_i) one step earlier; if that node is solid,
 * the population that left (x, y) towards it in direction opp(i) comes back. */
static double pulled(const oracle_params *p, const uint8_t *solid, const double *fs, int a, int i,
                     int x, int y) {
    int sx = x - CX[i], sy = y - CY[i];
    if (is_solid(p, solid, sx, sy)) return fs[fidx(p, a, OPP[i], x, y)];
    return fs[fidx(p, a, i, wrap(sx, p->nx), wrap(sy, p->ny))];
}

/* Density of species a at (x, y) after streaming; a solid node carries the
 * wall potential rho_s^a (end of Section 2). */
static double density_at(const oracle_params *p, const uint8_t *solid, const double *fs, int a,
                         int x, int y) {
    x = wrap(x, p->nx);
    y = wrap(y, p->ny);
    if (is_solid(p, solid, x, y)) return p->rho_wall[a];
    double r = 0.0;
    for (int i = 0; i < 9; i++) r += pulled(p, solid, fs, a, i, x, y);
    return r;
}

/* Eq. (comp_interaction) divided by rho^a, plus the body-force acceleration:
 *   F^a/rho^a = G sum_i w_i c_i rho^b(x + c_i) + g.
 * rho_b is the other species' density field (ny*nx, solid nodes already
 * holding rho_s^b). */
static void accel_at(const oracle_params *p, const double *rho_b, int x, int y, double *ax,
                     double *ay) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < 9; i++) {
        double rb = rho_b[(size_t)wrap(y + CY[i], p->ny) * p->nx + wrap(x + CX[i], p->nx)];
        sx += W[i] * CX[i] * rb;
        sy += W[i] * CY[i] * rb;
    }
    *ax = p->G * sx + p->g[0];
    *ay = p->G * sy + p->g[1];
}

/* Collision at one fluid node given the pulled populations fl[a][i] and the
 * accelerations acc[a][2].  Writes the post-collision populations out[a][i]
 * and, if mac is non-NULL, mac = {rho^o, rho^w, j^o_x, j^o_y, j^w_x, j^w_y}. */
static void collide_node(const oracle_params *p, const double fl[2][9], const double acc[2][2],
                         double out[2][9], double *mac) {
    double rho[2], jx[2], jy[2];
    for (int a = 0; a < 2; a++) {
        rho[a] = jx[a] = jy[a] = 0.0;
        for (int i = 0; i < 9; i++) {
            rho[a] += fl[a][i];
            jx[a] += CX[i] * fl[a][i];
            jy[a] += CY[i] * fl[a][i];
        }
    }
    double rt = rho[0] + rho[1];
    /* mixture velocity and mixture relaxation time (Section 2) */
    double ux = (jx[0] + jx[1]) / rt;
    double uy = (jy[0] + jy[1]) / rt;
    double nu0 = T0 * (p->tau[0] - 0.5), nu1 = T0 * (p->tau[1] - 0.5);
    double nu_mix = (rho[0] * nu0 + rho[1] * nu1) / rt;
    double tau_mix = nu_mix / T0 + 0.5;
    for (int a = 0; a < 2; a++) {
        double feq_u[9], feq_s[9], fneq[9];
        /* f' = f - f^eq(rho^a, u_mix): the non-equilibrium part */
        oracle_feq(p->eq_order, rho[a], ux, uy, feq_u);
        for (int i = 0; i < 9; i++) fneq[i] = fl[a][i] - feq_u[i];
        if (p->collision == 1) {
            /* Eq. (Regualize): keep only the part of f' that carries the
             * non-equilibrium momentum flux Pi = sum_j c_j c_j f'_j, through
             * the second-order Hermite polynomial Q_i = c_i c_i - T0 I:
             * f'_i = w_i / (2 T0^2) Q_i : Pi */
            double pxx = 0.0, pyy = 0.0, pxy = 0.0;
            for (int j = 0; j < 9; j++) {
                pxx += CX[j] * CX[j] * fneq[j];
                pyy += CY[j] * CY[j] * fneq[j];
                pxy += CX[j] * CY[j] * fneq[j];
            }
            for (int i = 0; i < 9; i++) {
                double qxx = CX[i] * CX[i] - T0, qyy = CY[i] * CY[i] - T0, qxy = CX[i] * CY[i];
                fneq[i] = W[i] / (2.0 * T0 * T0) * (qxx * pxx + qyy * pyy + 2.0 * qxy * pxy);
            }
        }
        /* Eq. (collision_term): equilibrium at the force-shifted velocity */
        oracle_feq(p->eq_order, rho[a], ux + acc[a][0], uy + acc[a][1], feq_s);
        for (int i = 0; i < 9; i++)
            out[a][i] = feq_s[i] + (1.0 - 1.0 / tau_mix) * fneq[i];
    }
    if (mac) {
        mac[0] = rho[0];
        mac[1] = rho[1];
        mac[2] = jx[0];
        mac[3] = jy[0];
        mac[4] = jx[1];
        mac[5] = jy[1];
    }
}

/* Density field of the pulled state, [2][ny][nx], rho_s at solid nodes. */
void oracle_density(const oracle_params *p, const uint8_t *solid, const double *fs, double *rho) {
    size_t n = (size_t)p->nx * p->ny;
    for (int a = 0; a < 2; a++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++)
                rho[a * n + (size_t)y * p->nx + x] = density_at(p, solid, fs, a, x, y);
}

/* Acceleration field F^a/rho^a + g, [2 species][2 components][ny][nx], from a
 * density field [2][ny][nx] (solid nodes holding rho_s).  Zero at solid nodes. */
void oracle_accel(const oracle_params *p, const uint8_t *solid, const double *rho, double *acc) {
    size_t n = (size_t)p->nx * p->ny;
    for (int a = 0; a < 2; a++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                size_t k = (size_t)y * p->nx + x;
                double ax = 0.0, ay = 0.0;
                if (!solid[k]) accel_at(p, rho + (size_t)(1 - a) * n, x, y, &ax, &ay);
                acc[(a * 2 + 0) * n + k] = ax;
                acc[(a * 2 + 1) * n + k] = ay;
            }
}

/*
 * One full time step f*(t) -> f*(t+1) over the grid.
 * obs (may be NULL) receives, for the pulled state of this step:
 *   obs[0], obs[1] = sum over fluid nodes of rho^o, rho^w
 *   obs[2] = sum over fluid nodes of j^o_x + F^o_x / 2   (oil momentum)
 *   obs[3] = max over fluid nodes of |u|, u = (j^o + j^w + (F^o + F^w)/2)/rho
 *   obs[4] = 1 if any fluid node has a NaN or negative density, else 0
 * Returns 0, or -1 when the mask breaks the boundary rule.
 */
int oracle_step(const oracle_params *p, const uint8_t *solid, const double *fin, double *fout,
                double *obs) {
    if (oracle_check(p, solid)) return -1;
    size_t n = (size_t)p->nx * p->ny;
    double *rho = (double *)malloc(sizeof(double) * 2 * n);
    if (!rho) return -2;
    oracle_density(p, solid, fin, rho);
    double mo = 0.0, mw = 0.0, px = 0.0, umax2 = 0.0, bad = 0.0;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            size_t k = (size_t)y * p->nx + x;
            if (solid[k]) {
                for (int a = 0; a < 2; a++)
                    for (int i = 0; i < 9; i++) fout[fidx(p, a, i, x, y)] = 0.0;
                continue;
            }
            double fl[2][9], acc[2][2], out[2][9], mac[6];
            for (int a = 0; a < 2; a++)
                for (int i = 0; i < 9; i++) fl[a][i] = pulled(p, solid, fin, a, i, x, y);
            for (int a = 0; a < 2; a++)
                accel_at(p, rho + (size_t)(1 - a) * n, x, y, &acc[a][0], &acc[a][1]);
            collide_node(p, fl, acc, out, mac);
            for (int a = 0; a < 2; a++)
                for (int i = 0; i < 9; i++) fout[fidx(p, a, i, x, y)] = out[a][i];
            double r0 = mac[0], r1 = mac[1], rt = r0 + r1;
            mo += r0;
            mw += r1;
            px += mac[2] + 0.5 * r0 * acc[0][0];
            double ux = (mac[2] + mac[4] + 0.5 * (r0 * acc[0][0] + r1 * acc[1][0])) / rt;
            double uy = (mac[3] + mac[5] + 0.5 * (r0 * acc[0][1] + r1 * acc[1][1])) / rt;
            double u2 = ux * ux + uy * uy;
            if (u2 > umax2) umax2 = u2;
            if (!(r0 >= 0.0) || !(r1 >= 0.0)) bad = 1.0;
        }
    free(rho);
    if (obs) {
        obs[0] = mo;
        obs[1] = mw;
        obs[2] = px;
        obs[3] = sqrt(umax2);
        obs[4] = bad;
    }
    return 0;
}

/* n steps, ping-ponging between f (input and final output) and a scratch
 * buffer.  obs_hist (may be NULL) receives 5 values per step. */
int oracle_run(const oracle_params *p, const uint8_t *solid, double *f, int64_t nsteps,
               double *obs_hist) {
    size_t len = (size_t)2 * 9 * p->nx * p->ny;
    double *tmp = (double *)malloc(sizeof(double) * len);
    if (!tmp) return -2;
    double *a = f, *b = tmp;
    for (int64_t s = 0; s < nsteps; s++) {
        int rc = oracle_step(p, solid, a, b, obs_hist ? obs_hist + 5 * s : NULL);
        if (rc) {
            free(tmp);
            return rc;
        }
        double *t = a;
        a = b;
        b = t;
    }
    if (a != f) memcpy(f, a, sizeof(double) * len);
    free(tmp);
    return 0;
}

/*
 * Macroscopic fields of the state one pull ahead of the stored f*:
 *   rho[2][ny][nx] (rho_s at solid nodes),
 *   u[2][ny][nx] = mixture velocity components (u_x plane, then u_y plane),
 *                  u = (j^o + j^w + (F^o + F^w)/2)/(rho^o + rho^w), 0 at solid,
 *   pr[ny][nx]   = T0 (rho^o + rho^w) - G T0 rho^o rho^w (the non-ideal
 *                  mixture equation of state implied by Eq. (comp_interaction)
 *                  in the continuum limit), 0 at solid.
 * Any output pointer may be NULL.
 */
void oracle_fields(const oracle_params *p, const uint8_t *solid, const double *fs, double *rho_out,
                   double *u_out, double *p_out) {
    size_t n = (size_t)p->nx * p->ny;
    double *rho = (double *)malloc(sizeof(double) * 2 * n);
    if (!rho) return;
    oracle_density(p, solid, fs, rho);
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            size_t k = (size_t)y * p->nx + x;
            double r0 = rho[k], r1 = rho[n + k];
            double ux = 0.0, uy = 0.0, pr = 0.0;
            if (!solid[k]) {
                double jx = 0.0, jy = 0.0, acc[2][2];
                for (int a = 0; a < 2; a++) {
                    accel_at(p, rho + (size_t)(1 - a) * n, x, y, &acc[a][0], &acc[a][1]);
                    for (int i = 0; i < 9; i++) {
                        double v = pulled(p, solid, fs, a, i, x, y);
                        jx += CX[i] * v;
                        jy += CY[i] * v;
                    }
                }
                double rt = r0 + r1;
                ux = (jx + 0.5 * (r0 * acc[0][0] + r1 * acc[1][0])) / rt;
                uy = (jy + 0.5 * (r0 * acc[0][1] + r1 * acc[1][1])) / rt;
                pr = T0 * rt - p->G * T0 * r0 * r1;
            }
            if (rho_out) {
                rho_out[k] = r0;
                rho_out[n + k] = r1;
            }
            if (u_out) {
                u_out[k] = ux;
                u_out[n + k] = uy;
            }
            if (p_out) p_out[k] = pr;
        }
    free(rho);
}

/*
 * The step at a few nodes only, for spot checks on grids too large for the
 * full oracle: for each (xs[k], ys[k]) writes the 18 post-collision
 * populations out[k][a][i] that oracle_step would write there (zeros at a
 * solid node).  Neighbour densities are recomputed from fin locally.
 */
void oracle_step_nodes(const oracle_params *p, const uint8_t *solid, const double *fin, int64_t count,
                       const int32_t *xs, const int32_t *ys, double *out) {
    for (int64_t k = 0; k < count; k++) {
        int x = xs[k], y = ys[k];
        double *o = out + 18 * k;
        if (is_solid(p, solid, x, y)) {
            for (int j = 0; j < 18; j++) o[j] = 0.0;
            continue;
        }
        double fl[2][9], acc[2][2], res[2][9];
        for (int a = 0; a < 2; a++)
            for (int i = 0; i < 9; i++) fl[a][i] = pulled(p, solid, fin, a, i, x, y);
        for (int a = 0; a < 2; a++) {
            int b = 1 - a;
            double sx = 0.0, sy = 0.0;
            for (int i = 0; i < 9; i++) {
                double rb = density_at(p, solid, fin, b, x + CX[i], y + CY[i]);
                sx += W[i] * CX[i] * rb;
                sy += W[i] * CY[i] * rb;
            }
            acc[a][0] = p->G * sx + p->g[0];
            acc[a][1] = p->G * sy + p->g[1];
        }
        collide_node(p, fl, acc, res, NULL);
        for (int a = 0; a < 2; a++)
            for (int i = 0; i < 9; i++) o[a * 9 + i] = res[a][i];
    }
}
