/*
 * Oracle for the two-component D3Q19 lattice-Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 CPU statement of the time step
 * on the paper's own lattice (Section 2: "D3Q19", T0 = 1/3).  Only the test
 * suite may load it; the product library never links or calls it and shares
 * no code with it.
 *
 * Same method as lbm_oracle.c, on the three-dimensional velocity set:
 *   - Eq. (basic_LBM_eq) with the collision of Eq. (LBM_BGK): the force
 *     carried by the equilibrium velocity shift of Eq. (collision_term),
 *     f*_i = f_i^eq(rho^a, u_mix + F^a/rho^a) + (1 - 1/tau_mix) f'_i, with
 *     f' = f - f^eq(rho^a, u_mix) (collision = 0) or its regularised
 *     projection of Eq. (Regualize), w_i Q_i : Pi / (2 T0^2),
 *     Q_i = c_i c_i - T0 I, Pi = sum_j c_j c_j f'_j (collision = 1);
 *   - tau_mix = nu_mix/T0 + 1/2, nu_mix = (rho^o nu^o + rho^w nu^w)/rho;
 *   - Eq. (feq), third order as printed (second order as an option);
 *   - Eq. (comp_interaction), F^a = G rho^a sum_i w_i c_i rho^b(x + c_i),
 *     with the wall potentials standing in for solid neighbours;
 *   - the homogeneous body force of Section 3.4;
 *   - halfway bounce-back on a node mask.
 *
 * Lattice: c_0 = 0; c_1..c_6 the six face neighbours (+-1,0,0), (0,+-1,0),
 * (0,0,+-1), weight 1/18; c_7..c_18 the twelve edge neighbours
 * (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1), weight 1/36; rest 1/3.
 * Storage: f[(a*19 + i)][z][y][x], x fastest.  Indices wrap in every
 * direction; a direction that is not periodic needs solid boundary planes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
    double tau[2];
    double G;
    double rho_wall[2];
    double g[3];
    int32_t eq_order;
    int32_t collision;
} oracle3_params;

static const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double T0 = 1.0 / 3.0;

static double weight(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

/* the direction opposite to i */
static int opposite(int i) {
    for (int j = 0; j < 19; j++)
        if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
    return -1;
}

static int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

static size_t node(const oracle3_params *p, int x, int y, int z) {
    return ((size_t)wrap(z, p->nz) * p->ny + (size_t)wrap(y, p->ny)) * p->nx + (size_t)wrap(x, p->nx);
}

static size_t fidx(const oracle3_params *p, int a, int i, size_t k) {
    return ((size_t)a * 19 + (size_t)i) * (size_t)p->nx * p->ny * p->nz + k;
}

/* 0 when every non-periodic direction has solid boundary planes. */
int oracle3_check(const oracle3_params *p, const uint8_t *solid) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->collision != 0 && p->collision != 1) return -1;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                int edge = (!p->periodic[0] && (x == 0 || x == p->nx - 1)) ||
                           (!p->periodic[1] && (y == 0 || y == p->ny - 1)) ||
                           (!p->periodic[2] && (z == 0 || z == p->nz - 1));
                if (edge && !solid[node(p, x, y, z)]) return -1;
            }
    return 0;
}

/* Eq. (feq) on D3Q19: rho w_i [1 + c.u/T0 + (c.u)^2/(2T0^2) - u^2/(2T0)
 *                              + (c.u)^3/(6T0^3) - (c.u) u^2/(2T0^2)]. */
void oracle3_feq(int order, double rho, double ux, double uy, double uz, double *out) {
    double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; i++) {
        double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
        double b = 1.0 + cu / T0 + cu * cu / (2.0 * T0 * T0) - uu / (2.0 * T0);
        if (order >= 3) b += cu * cu * cu / (6.0 * T0 * T0 * T0) - cu * uu / (2.0 * T0 * T0);
        out[i] = weight(i) * rho * b;
    }
}

/* f*_i = w_i rho_init at fluid nodes, 0 at solid ones; rho_init [2][nz][ny][nx]. */
void oracle3_init(const oracle3_params *p, const uint8_t *solid, const double *rho_init, double *f) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    for (int a = 0; a < 2; a++)
        for (int i = 0; i < 19; i++)
            for (size_t k = 0; k < n; k++) f[fidx(p, a, i, k)] = solid[k] ? 0.0 : weight(i) * rho_init[a * n + k];
}

/* halfway bounce-back pull of direction i at (x, y, z) */
static double pulled(const oracle3_params *p, const uint8_t *solid, const double *fs, int a, int i, int x,
                     int y, int z) {
    size_t src = node(p, x - CX[i], y - CY[i], z - CZ[i]);
    if (solid[src]) return fs[fidx(p, a, opposite(i), node(p, x, y, z))];
    return fs[fidx(p, a, i, src)];
}

static double density_at(const oracle3_params *p, const uint8_t *solid, const double *fs, int a, int x, int y,
                         int z) {
    size_t k = node(p, x, y, z);
    if (solid[k]) return p->rho_wall[a];
    double r = 0.0;
    for (int i = 0; i < 19; i++) r += pulled(p, solid, fs, a, i, x, y, z);
    return r;
}

/* Density field of the pulled state, [2][nz][ny][nx], rho_s at solid nodes. */
void oracle3_density(const oracle3_params *p, const uint8_t *solid, const double *fs, double *rho) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    for (int a = 0; a < 2; a++)
        for (int z = 0; z < p->nz; z++)
            for (int y = 0; y < p->ny; y++)
                for (int x = 0; x < p->nx; x++) rho[a * n + node(p, x, y, z)] = density_at(p, solid, fs, a, x, y, z);
}

/* F^a/rho^a + g = G sum_i w_i c_i rho^b(x + c_i) + g from the field rho_b. */
static void accel_at(const oracle3_params *p, const double *rho_b, int x, int y, int z, double acc[3]) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; i++) {
        double rb = rho_b[node(p, x + CX[i], y + CY[i], z + CZ[i])];
        s[0] += weight(i) * CX[i] * rb;
        s[1] += weight(i) * CY[i] * rb;
        s[2] += weight(i) * CZ[i] * rb;
    }
    for (int d = 0; d < 3; d++) acc[d] = p->G * s[d] + p->g[d];
}

/* Collision at one node from its pulled populations fl[a][i] and the
 * accelerations acc[a][3]; mac (may be NULL) = {rho^o, rho^w, j^o (3), j^w (3)}. */
static void collide_node(const oracle3_params *p, const double fl[2][19], const double acc[2][3],
                         double out[2][19], double *mac) {
    double rho[2], j[2][3];
    for (int a = 0; a < 2; a++) {
        rho[a] = j[a][0] = j[a][1] = j[a][2] = 0.0;
        for (int i = 0; i < 19; i++) {
            rho[a] += fl[a][i];
            j[a][0] += CX[i] * fl[a][i];
            j[a][1] += CY[i] * fl[a][i];
            j[a][2] += CZ[i] * fl[a][i];
        }
    }
    double rt = rho[0] + rho[1];
    double u[3];
    for (int d = 0; d < 3; d++) u[d] = (j[0][d] + j[1][d]) / rt;
    double nu0 = T0 * (p->tau[0] - 0.5), nu1 = T0 * (p->tau[1] - 0.5);
    double nu_mix = (rho[0] * nu0 + rho[1] * nu1) / rt;
    double tau_mix = nu_mix / T0 + 0.5;
    for (int a = 0; a < 2; a++) {
        double feq_u[19], feq_s[19], fneq[19];
        oracle3_feq(p->eq_order, rho[a], u[0], u[1], u[2], feq_u);
        for (int i = 0; i < 19; i++) fneq[i] = fl[a][i] - feq_u[i];
        if (p->collision == 1) {
            /* Eq. (Regualize): f'_i = w_i / (2 T0^2) Q_i : Pi */
            double P[3][3] = {{0}};
            for (int k = 0; k < 19; k++) {
                int c[3] = {CX[k], CY[k], CZ[k]};
                for (int r = 0; r < 3; r++)
                    for (int s = 0; s < 3; s++) P[r][s] += c[r] * c[s] * fneq[k];
            }
            for (int i = 0; i < 19; i++) {
                int c[3] = {CX[i], CY[i], CZ[i]};
                double qp = 0.0;
                for (int r = 0; r < 3; r++)
                    for (int s = 0; s < 3; s++) qp += (c[r] * c[s] - (r == s ? T0 : 0.0)) * P[r][s];
                fneq[i] = weight(i) / (2.0 * T0 * T0) * qp;
            }
        }
        oracle3_feq(p->eq_order, rho[a], u[0] + acc[a][0], u[1] + acc[a][1], u[2] + acc[a][2], feq_s);
        for (int i = 0; i < 19; i++) out[a][i] = feq_s[i] + (1.0 - 1.0 / tau_mix) * fneq[i];
    }
    if (mac) {
        mac[0] = rho[0];
        mac[1] = rho[1];
        for (int d = 0; d < 3; d++) {
            mac[2 + d] = j[0][d];
            mac[5 + d] = j[1][d];
        }
    }
}

/*
 * One step f*(t) -> f*(t+1).  obs (may be NULL): [0], [1] masses of the two
 * species over fluid nodes; [2] = sum of j^o_x + F^o_x / 2 (oil momentum in
 * x); [3] = max |u|, u = (j^o + j^w + (F^o + F^w)/2)/rho; [4] = 1 if a fluid
 * node has a NaN or negative density.  Returns 0, or -1 for a mask that
 * breaks the boundary rule.
 */
int oracle3_step(const oracle3_params *p, const uint8_t *solid, const double *fin, double *fout, double *obs) {
    if (oracle3_check(p, solid)) return -1;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *rho = (double *)malloc(sizeof(double) * 2 * n);
    if (!rho) return -2;
    oracle3_density(p, solid, fin, rho);
    double mo = 0.0, mw = 0.0, px = 0.0, umax2 = 0.0, bad = 0.0;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                size_t k = node(p, x, y, z);
                if (solid[k]) {
                    for (int a = 0; a < 2; a++)
                        for (int i = 0; i < 19; i++) fout[fidx(p, a, i, k)] = 0.0;
                    continue;
                }
                double fl[2][19], acc[2][3], out[2][19], mac[8];
                for (int a = 0; a < 2; a++)
                    for (int i = 0; i < 19; i++) fl[a][i] = pulled(p, solid, fin, a, i, x, y, z);
                for (int a = 0; a < 2; a++) accel_at(p, rho + (size_t)(1 - a) * n, x, y, z, acc[a]);
                collide_node(p, fl, acc, out, mac);
                for (int a = 0; a < 2; a++)
                    for (int i = 0; i < 19; i++) fout[fidx(p, a, i, k)] = out[a][i];
                double r0 = mac[0], r1 = mac[1], rt = r0 + r1, u2 = 0.0;
                mo += r0;
                mw += r1;
                px += mac[2] + 0.5 * r0 * acc[0][0];
                for (int d = 0; d < 3; d++) {
                    double ud = (mac[2 + d] + mac[5 + d] + 0.5 * (r0 * acc[0][d] + r1 * acc[1][d])) / rt;
                    u2 += ud * ud;
                }
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

/* n steps; obs_hist (may be NULL) receives 5 values per step. */
int oracle3_run(const oracle3_params *p, const uint8_t *solid, double *f, int64_t nsteps, double *obs_hist) {
    size_t len = (size_t)2 * 19 * p->nx * p->ny * p->nz;
    double *tmp = (double *)malloc(sizeof(double) * len);
    if (!tmp) return -2;
    double *a = f, *b = tmp;
    for (int64_t s = 0; s < nsteps; s++) {
        int rc = oracle3_step(p, solid, a, b, obs_hist ? obs_hist + 5 * s : NULL);
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

/* rho [2][nz][ny][nx] and u [3][nz][ny][nx] (mixture velocity with half the
 * force) one pull ahead of f*; 0 velocity at solid nodes. */
void oracle3_fields(const oracle3_params *p, const uint8_t *solid, const double *fs, double *rho_out,
                    double *u_out) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *rho = (double *)malloc(sizeof(double) * 2 * n);
    if (!rho) return;
    oracle3_density(p, solid, fs, rho);
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                size_t k = node(p, x, y, z);
                double r0 = rho[k], r1 = rho[n + k], u[3] = {0.0, 0.0, 0.0};
                if (!solid[k]) {
                    double jx[3] = {0.0, 0.0, 0.0}, acc[2][3];
                    for (int a = 0; a < 2; a++) {
                        accel_at(p, rho + (size_t)(1 - a) * n, x, y, z, acc[a]);
                        for (int i = 0; i < 19; i++) {
                            double v = pulled(p, solid, fs, a, i, x, y, z);
                            jx[0] += CX[i] * v;
                            jx[1] += CY[i] * v;
                            jx[2] += CZ[i] * v;
                        }
                    }
                    for (int d = 0; d < 3; d++) u[d] = (jx[d] + 0.5 * (r0 * acc[0][d] + r1 * acc[1][d])) / (r0 + r1);
                }
                if (rho_out) {
                    rho_out[k] = r0;
                    rho_out[n + k] = r1;
                }
                if (u_out)
                    for (int d = 0; d < 3; d++) u_out[d * n + k] = u[d];
            }
    free(rho);
}

/* The velocity set, for tests that take moments: c[19][3], w[19]. */
void oracle3_lattice(int32_t *c, double *w) {
    for (int i = 0; i < 19; i++) {
        c[3 * i] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
        w[i] = weight(i);
    }
}
