// The paper's question posed from channel descriptions (C ABI, include/lbm.h).
//
// Section 3.4 of the paper asks for the smallest homogeneous body force at
// which an oil slug resting in a sinusoidal channel starts to move, and
// reports it as a critical Bond number.  The calls here take that question
// as the user states it -- a wavelength, an amplitude ratio, a slug length,
// a contact angle and a viscosity ratio -- and do every set-up step inside
// the library:
//   - the channel and the slug (lbm_channel_geometry: the planar 2-D
//     channel, mean half-width 0.1875 lambda, slug centred on a neck);
//   - the wall potentials of the requested contact angle, from the
//     flat-plate calibration of Section 3.3 run on the GPU
//     (lbm_wetting_calibrate: interface points where the oil fraction
//     crosses 1/2, Pratt's algebraic circle fit, Eq. contact_angle);
//   - the relaxation times of the viscosity ratio (Section 2, tau^w = 1);
//   - the starting bracket: the planar analogue of the Section 3.4 static
//     balance (lbm_planar_critical_balance), or the surrogate network's
//     +-k sigma bracket;
//   - the surface tension and bulk density that turn g into a Bond number,
//     from the Laplace law of Section 3.1 run on the GPU
//     (lbm_surface_tension);
//   - the batched bisection (lbm_critical_pressure_batch).
// Host arithmetic is FP64; the simulations run in the storage format the
// caller picks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kG = -1.79;            // interaction strength of the channel model (flat-interface coexistence 1.0 / 0.03)
constexpr double kRhoHi = 1.0;          // initial bulk densities of a phase
constexpr double kRhoLo = 0.03;
constexpr double kTauMin = 0.75;        // lowest tau^o a channel is run at (positivity of the minority density)
constexpr double kT0 = 1.0 / 3.0;
constexpr int kCalibH = 32;             // flat plates: fluid rows 1..H
constexpr int kCalibNx = 192;
constexpr int64_t kCalibSteps = 20000;
constexpr int kLaplaceN = 128;          // droplets in a periodic box
constexpr double kLaplaceR[4] = {12.0, 16.0, 20.0, 24.0};
constexpr int64_t kLaplaceSteps = 6000;
constexpr double kSurrogateFloor = 1.05;   // a surrogate bracket is at least this factor wide

thread_local std::string g_chan_err;

int cfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_chan_err = buf;
    return code;
}

// ---------------------------------------------------------------------------
// channel geometry
// ---------------------------------------------------------------------------
struct Geom {
    int nx, ny;
    int slugs;            // identical slugs, centred on necks spaced n_periods / slugs apart
    double lam, h0, amp, yc, centre, half, spacing;
};

// 0 selects the default; a negative count is out of range (geom_of rejects it)
int periods_of(const lbm_channel_spec& s) { return s.n_periods != 0 ? s.n_periods : 4; }
int slugs_of(const lbm_channel_spec& s) { return s.n_slugs != 0 ? s.n_slugs : 1; }

bool geom_of(const lbm_channel_spec& s, Geom* g) {
    const int np = periods_of(s), ns = slugs_of(s);
    if (s.lambda < 8 || s.lambda > (1 << 16) || np < 2 || np > 64) return false;
    if (ns < 1 || ns > np || np % ns != 0) return false;
    if (!(s.amp_ratio >= 0.0 && s.amp_ratio <= 0.95)) return false;
    if (!(s.slug_len_over_lambda > 0.0 && s.slug_len_over_lambda <= np / ns - (ns > 1 ? 0.25 : 1.0))) return false;
    if (!(s.theta_deg > 0.0 && s.theta_deg < 180.0) || !(s.visc_ratio > 0.0) || !std::isfinite(s.visc_ratio))
        return false;
    g->lam = (double)s.lambda;
    g->h0 = 0.1875 * g->lam;
    g->amp = s.amp_ratio * g->h0;
    g->nx = s.lambda * np;
    g->ny = 2 * (int)std::ceil(g->h0 + g->amp) + 2;
    g->yc = (g->ny - 1) / 2.0;
    g->slugs = ns;
    g->spacing = g->lam * (np / ns);
    g->centre = g->lam * (np / (2 * ns));      // the first slug; the others follow every `spacing`
    g->half = 0.5 * s.slug_len_over_lambda * g->lam;
    return true;
}

// smooth step of width 2: (1 + tanh(d / 2)) / 2
double step2(double d) { return 0.5 * (1.0 + std::tanh(d / 2.0)); }

void fill(const Geom& g, uint8_t* mask, double* rho) {
    const size_t n = (size_t)g.nx * g.ny;
    for (int y = 0; y < g.ny; y++)
        for (int x = 0; x < g.nx; x++) {
            const double h = g.h0 - g.amp * std::cos(2.0 * kPi * (double)x / g.lam);
            bool solid = std::fabs(y - g.yc) > h;
            if (y == 0 || y == g.ny - 1) solid = true;
            const size_t k = (size_t)y * g.nx + x;
            if (mask) mask[k] = solid ? 1 : 0;
            if (rho) {
                double sl = 0.0;
                for (int j = 0; j < g.slugs; j++) {
                    const double c = g.centre + j * g.spacing;
                    sl += step2(x - (c - g.half)) - step2(x - (c + g.half));
                }
                const double ro = kRhoLo + (kRhoHi - kRhoLo) * sl;
                rho[k] = ro;
                rho[n + k] = kRhoHi + kRhoLo - ro;
            }
        }
}

// ---------------------------------------------------------------------------
// Section 3.4, planar form: menisci as axis-centred arcs
// ---------------------------------------------------------------------------
struct Channel {
    double h0, amp, lam;
};

// Curvature (1 / radius, signed) of the meniscus whose contact line sits at
// x, and the signed area of its circular segment beyond the contact chord.
// The wall is inclined by phi = atan h'(x); the arc meets it at the contact
// angle theta (through water) on the front (advancing) or rear side.
void meniscus(const Channel& c, double theta, double x, bool front, double* kappa, double* seg) {
    const double k = 2.0 * kPi / c.lam;
    const double h = c.h0 - c.amp * std::cos(k * x);
    const double phi = std::atan(c.amp * k * std::sin(k * x));
    const double alpha = 0.5 * kPi + (front ? phi : -phi) - theta;
    *kappa = std::sin(alpha) / h;
    const double a = std::max(std::fabs(alpha), 1e-9);
    const double sg = alpha > 0.0 ? 1.0 : (alpha < 0.0 ? -1.0 : 0.0);
    const double r = h / std::sin(a);
    *seg = sg * r * r * (a - std::sin(a) * std::cos(a));
}

// Oil area between the rear contact line xr and the front one xf: the
// channel between the two contact chords plus the two segments (front
// meniscus at angle theta_f, rear at theta_r).
double oil_area(const Channel& c, double theta_f, double theta_r, double xr, double xf) {
    const double k = 2.0 * kPi / c.lam;
    const double inner = 2.0 * c.h0 * (xf - xr) - 2.0 * c.amp / k * (std::sin(k * xf) - std::sin(k * xr));
    double kf, sf, kr, sr;
    meniscus(c, theta_f, xf, true, &kf, &sf);
    meniscus(c, theta_r, xr, false, &kr, &sr);
    return inner + sf + sr;
}

// rho g L / sigma at which a slug of oil area `area` starts to move, loaded
// quasi-statically from the rest position nearest x_rest (rear contact
// line): the balance kappa_front - kappa_rear is sampled over the rear
// position (front from the area by bisection), the slug climbs each rising
// branch and jumps ahead past each local maximum, and it counts as moving
// at the first jump longer than lambda / 2 (or out of the period).
// theta_front_deg / theta_rear_deg: the contact angles through water at
// the front (advancing oil, receding water) and rear menisci; equal for the
// static balance, apart when the contact angle shows hysteresis.
int planar_balance2(double theta_front_deg, double theta_rear_deg, double area, double h0, double amp, double lam,
                    double x_rest, double* out) {
    const Channel c{h0, amp, lam};
    const double thf = theta_front_deg * kPi / 180.0, thr = theta_rear_deg * kPi / 180.0;
    constexpr int n = 2001;
    std::vector<double> s(n), bal(n);
    const double s0 = x_rest - 0.5 * lam, ds = 2.0 * lam / (n - 1);
    double bmax = 0.0;
    for (int i = 0; i < n; i++) {
        s[i] = s0 + ds * i;
        double lo = s[i] + 1e-6, hi = s[i] + area / (2.0 * std::max(h0 - amp, 1e-9)) + 2.0 * lam;
        for (int it = 0; it < 80; it++) {
            const double mid = 0.5 * (lo + hi);
            if (oil_area(c, thf, thr, s[i], mid) > area) hi = mid;
            else lo = mid;
        }
        const double xf = 0.5 * (lo + hi);
        double kf, sf, kr, sr;
        meniscus(c, thf, xf, true, &kf, &sf);
        meniscus(c, thr, s[i], false, &kr, &sr);
        bal[i] = kf - kr;
        bmax = std::max(bmax, std::fabs(bal[i]));
    }
    if (bmax < 1e-12) {      // no capillary resistance (straight channel, neutral wetting)
        *out = 0.0;
        return LBM_OK;
    }
    int best = -1;
    for (int i = 0; i + 1 < n; i++)
        if (bal[i] <= 0.0 && 0.0 < bal[i + 1] && s[i] <= x_rest + 0.5 * lam)
            if (best < 0 || std::fabs(s[i] - x_rest) < std::fabs(s[best] - x_rest)) best = i;
    if (best < 0) return cfail(LBM_EINVAL, "planar balance: no rest position within half a wavelength");
    const double end = s[best] + lam, jump = 0.5 * lam;
    int j = best + 1;
    while (true) {
        int p = j;
        while (p + 1 < n && !(bal[p + 1] < bal[p])) p++;   // next local maximum
        j = p;
        int k = j + 1;
        while (k < n && bal[k] < bal[j]) k++;               // next sample as high
        if (k >= n || s[k] - s[j] > jump || s[k] >= end) break;
        j = k;
    }
    *out = bal[j];
    return LBM_OK;
}

int planar_balance(double theta_deg, double area, double h0, double amp, double lam, double x_rest, double* out) {
    return planar_balance2(theta_deg, theta_deg, area, h0, amp, lam, x_rest, out);
}

// ---------------------------------------------------------------------------
// Section 3.3: contact angle of a slug between flat plates
// ---------------------------------------------------------------------------
// x where an oil-fraction row crosses 1/2 at the left or right end of the
// oil (linear interpolation between the two nodes around the crossing).
bool half_crossing(const double* frac, int n, bool right, double* x) {
    int lo = -1, hi = -1;
    for (int i = 0; i < n; i++)
        if (frac[i] > 0.5) {
            if (lo < 0) lo = i;
            hi = i;
        }
    if (lo < 0) return false;
    int count = 0;
    for (int i = 0; i < n; i++) count += frac[i] > 0.5;
    if (count == n) return false;
    if (right) {
        const double a = frac[hi], b = frac[(hi + 1) % n];
        *x = hi + (a - 0.5) / (a - b);
    } else {
        const double a = frac[(lo - 1 + n) % n], b = frac[lo];
        *x = (lo - 1) + (0.5 - a) / (b - a);
    }
    return true;
}

double det3(const double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

// cofactor (i, j) of a 4 x 4 matrix
double cofactor4(const double a[4][4], int i, int j) {
    double m[3][3];
    for (int r = 0, rr = 0; r < 4; r++) {
        if (r == i) continue;
        for (int c = 0, cc = 0; c < 4; c++)
            if (c != j) m[rr][cc++] = a[r][c];
        rr++;
    }
    return ((i + j) & 1 ? -1.0 : 1.0) * det3(m);
}

double det4(const double a[4][4]) {
    double d = 0.0;
    for (int c = 0; c < 4; c++) d += a[0][c] * cofactor4(a, 0, c);
    return d;
}

// Pratt's algebraic circle fit (Pratt, Computer Graphics 21, 1987): the
// circle or line A (x^2 + y^2) + B x + C y + D = 0 minimising the sum of
// squared algebraic residuals subject to B^2 + C^2 - 4 A D = 1, i.e. the
// generalised eigenvector of the moment matrix M with the smallest
// non-negative eigenvalue eta, M v = eta N v.  eta is the first root of
// det(M - eta N) above 0, reached by Newton's method from 0 (the
// determinant decreases from det M >= 0 to that root); v spans the null
// space of M - eta N (the largest column of its adjugate).  Data are
// centred for conditioning and the shift undone at the end.  Stays well
// posed as the points straighten into a line (A -> 0).
bool pratt_fit(const std::vector<double>& xs, const std::vector<double>& ys, double* A, double* B, double* C,
               double* D) {
    const int n = (int)xs.size();
    if (n < 3) return false;
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < n; i++) {
        mx += xs[i];
        my += ys[i];
    }
    mx /= n;
    my /= n;
    double M[4][4] = {};
    for (int i = 0; i < n; i++) {
        const double u = xs[i] - mx, v = ys[i] - my;
        const double z[4] = {u * u + v * v, u, v, 1.0};
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) M[r][c] += z[r] * z[c] / n;
    }
    const double N[4][4] = {{0, 0, 0, -2}, {0, 1, 0, 0}, {0, 0, 1, 0}, {-2, 0, 0, 0}};
    double a[4][4];
    auto set = [&](double eta) {
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) a[r][c] = M[r][c] - eta * N[r][c];
    };
    // Newton on P(eta) = det(M - eta N); P' = -tr(adj(M - eta N) N), and the
    // only non-zero entries of N are (0,3), (3,0) = -2 and (1,1), (2,2) = 1
    double eta = 0.0;
    for (int it = 0; it < 100; it++) {
        set(eta);
        const double p = det4(a);
        const double dp = -(-2.0 * cofactor4(a, 0, 3) - 2.0 * cofactor4(a, 3, 0) + cofactor4(a, 1, 1) +
                            cofactor4(a, 2, 2));
        if (p == 0.0 || dp == 0.0) break;
        const double next = eta - p / dp;
        if (!std::isfinite(next) || next < 0.0) break;
        const bool done = std::fabs(next - eta) <= 1e-15 * std::max(1.0, std::fabs(next));
        eta = next;
        if (done) break;
    }
    set(eta);
    // null vector: the row of cofactors (a column of the adjugate) with the
    // largest norm
    double best[4] = {}, bestn = -1.0;
    for (int i = 0; i < 4; i++) {
        double v[4];
        for (int j = 0; j < 4; j++) v[j] = cofactor4(a, i, j);
        const double nv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
        if (nv > bestn) {
            bestn = nv;
            std::memcpy(best, v, sizeof best);
        }
    }
    double a0 = best[0], b0 = best[1], c0 = best[2], d0 = best[3];
    const double norm = std::sqrt(std::max(b0 * b0 + c0 * c0 - 4.0 * a0 * d0, 1e-300));
    a0 /= norm;
    b0 /= norm;
    c0 /= norm;
    d0 /= norm;
    *A = a0;
    *B = b0 - 2.0 * a0 * mx;
    *C = c0 - 2.0 * a0 * my;
    *D = d0 + a0 * (mx * mx + my * my) - b0 * mx - c0 * my;
    return std::isfinite(*A) && std::isfinite(*B) && std::isfinite(*C) && std::isfinite(*D);
}

// Contact angle through water (degrees) of one end of a slug between flat
// plates with fluid rows y_lo..y_hi, from the densities [2][ny][nx]; rows
// within `margin` of a wall are left out.  Eq. (contact_angle): the acute
// angle between wall and interface has cos = y0 / R (y0 the half width);
// it is the angle through water when the circle's centre is on the oil
// side, 180 degrees minus it otherwise.
bool contact_angle(const double* rho, int nx, int ny, int y_lo, int y_hi, bool right, double* theta) {
    const size_t n = (size_t)nx * ny;
    std::vector<double> frac(nx), xs, ys;
    const int margin = 3;
    for (int y = y_lo + margin; y <= y_hi - margin; y++) {
        for (int x = 0; x < nx; x++) {
            const double ro = rho[(size_t)y * nx + x], rw = rho[n + (size_t)y * nx + x];
            frac[x] = ro / (ro + rw);
        }
        double x;
        if (half_crossing(frac.data(), nx, right, &x)) {
            xs.push_back(x);
            ys.push_back((double)y);
        }
    }
    double A, B, C, D;
    if (xs.size() < 3 || !pratt_fit(xs, ys, &A, &B, &C, &D)) return false;
    if (std::fabs(A) < 1e-12) {
        *theta = 90.0;
        return true;
    }
    const double y0 = 0.5 * (y_hi - y_lo + 1);
    const double acute = std::acos(std::min(2.0 * std::fabs(A) * y0, 1.0)) * 180.0 / kPi;
    const double xc = -B / (2.0 * A);
    // interface position on the axis (linear interpolation in y)
    const double ya = 0.5 * (y_lo + y_hi);
    double x_axis = xs.back();
    for (size_t i = 0; i + 1 < ys.size(); i++)
        if (ys[i] <= ya && ya <= ys[i + 1]) {
            x_axis = xs[i] + (xs[i + 1] - xs[i]) * (ya - ys[i]) / (ys[i + 1] - ys[i]);
            break;
        }
    const bool on_oil = right ? xc < x_axis : xc > x_axis;
    *theta = on_oil ? acute : 180.0 - acute;
    return true;
}

// ---------------------------------------------------------------------------
// Section 3.4: contact angles of a slug's menisci in the sinusoidal channel
// ---------------------------------------------------------------------------
// One meniscus of a slug in the planar channel h(x) = h0 - amp cos(2 pi x /
// lam) about y_c = (ny - 1) / 2: on every fluid row at least two nodes from
// the wall, the oil-fraction crossing of 1/2 nearest to the meniscus's
// position x_end on the centre row (within lam / 3); Pratt's circle through
// those points; its intersection with the upper wall y = y_c + h(x) nearest
// the topmost point; the angle there between the wall (pointing into the
// water) and the interface (pointing into the fluid), i.e. the contact
// angle through water.
bool meniscus_angle(const std::vector<double>& frac, int nx, int ny, double h0, double amp, double lam, double x_end,
                    bool front, double* theta, double* x_contact, double* radius) {
    const double yc = (ny - 1) / 2.0, k = 2.0 * kPi / lam;
    auto h_at = [&](double x) { return h0 - amp * std::cos(k * x); };
    std::vector<double> xs, ys;
    const int lo = std::max(1, (int)std::floor(x_end - lam / 3.0)), hi = std::min(nx - 2, (int)std::ceil(x_end + lam / 3.0));
    for (int y = 1; y < ny - 1; y++) {
        double best = 0.0;
        bool found = false;
        for (int x = lo; x < hi; x++) {
            if (std::fabs(y - yc) > h_at(x) || std::fabs(y - yc) > h_at(x + 1)) continue;
            const double a = frac[(size_t)y * nx + x], b = frac[(size_t)y * nx + x + 1];
            double c;
            if (front && a > 0.5 && b <= 0.5) c = x + (a - 0.5) / (a - b);
            else if (!front && a <= 0.5 && b > 0.5) c = x + (0.5 - a) / (b - a);
            else continue;
            if (!found || std::fabs(c - x_end) < std::fabs(best - x_end)) best = c;
            found = true;
        }
        if (found && std::fabs(y - yc) <= h_at(best) - 2.0) {
            xs.push_back(best);
            ys.push_back((double)y);
        }
    }
    double A, B, C, D;
    if (xs.size() < 5 || !pratt_fit(xs, ys, &A, &B, &C, &D)) return false;
    // contact with the upper wall: F(x) = A (x^2 + y^2) + B x + C y + D on y = y_c + h(x)
    size_t top = 0;
    for (size_t q = 1; q < ys.size(); q++)
        if (ys[q] > ys[top]) top = q;
    auto F = [&](double x) {
        const double y = yc + h_at(x);
        return A * (x * x + y * y) + B * x + C * y + D;
    };
    const double x0 = xs[top];
    double xc = 0.0;
    bool hit = false;
    constexpr int kSamples = 2400;
    double prev = F(x0 - 6.0);
    for (int q = 1; q <= kSamples; q++) {
        const double xa = x0 - 6.0 + 12.0 * (q - 1) / kSamples, xb = x0 - 6.0 + 12.0 * q / kSamples;
        const double fb = F(xb);
        if ((prev < 0.0) != (fb < 0.0)) {
            const double cand = xa - prev * (xb - xa) / (fb - prev);
            if (!hit || std::fabs(cand - x0) < std::fabs(xc - x0)) xc = cand;
            hit = true;
        }
        prev = fb;
    }
    if (!hit) return false;
    const double yP = yc + h_at(xc), hp = amp * k * std::sin(k * xc);
    double ti[2] = {-(2.0 * A * yP + C), 2.0 * A * xc + B};     // tangent of the circle at the contact
    const double tn = std::hypot(ti[0], ti[1]);
    if (!(tn > 0.0)) return false;
    ti[0] /= tn;
    ti[1] /= tn;
    if (ti[1] > 0.0) {                                          // pointing into the fluid (down)
        ti[0] = -ti[0];
        ti[1] = -ti[1];
    }
    const double wn = std::hypot(1.0, hp);
    const double sgn = front ? 1.0 : -1.0;                      // the water lies ahead of the front, behind the rear
    const double dot = sgn * (ti[0] + hp * ti[1]) / wn;
    *theta = std::acos(std::max(-1.0, std::min(1.0, dot))) * 180.0 / kPi;
    *x_contact = xc;
    *radius = std::fabs(A) > 0.0 ? 1.0 / (2.0 * std::fabs(A)) : INFINITY;
    return true;
}

// ---------------------------------------------------------------------------
// GPU runs: calibration table, surface tension (cached per device)
// ---------------------------------------------------------------------------
struct Calib {
    std::vector<double> r, theta;
};
struct Laplace {
    double sigma = 0.0, rho_bulk = 0.0;
};
std::mutex g_cache_mu;
constexpr int kMaxDev = 64;
Calib g_calib[kMaxDev];
Laplace g_laplace[kMaxDev];

int batch_error(const char* what, int rc, lbm_batch_t* b) {
    return cfail(rc, "%s: %s", what, lbm_batch_last_error(b));
}

int calibrate(const double* r, int n, int64_t steps, int32_t precision, void* stream, double* theta) {
    const int H = kCalibH, nx = kCalibNx, ny = H + 2;
    const size_t nn = (size_t)nx * ny;
    std::vector<uint8_t> mask(nn, 0);
    std::vector<double> rho(2 * nn);
    for (int x = 0; x < nx; x++) {
        mask[x] = 1;
        mask[(size_t)(ny - 1) * nx + x] = 1;
    }
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            const double sl = step2(x - nx / 4.0) - step2(x - 3.0 * nx / 4.0);
            const double ro = kRhoLo + (kRhoHi - kRhoLo) * sl;
            rho[(size_t)y * nx + x] = ro;
            rho[nn + (size_t)y * nx + x] = kRhoHi + kRhoLo - ro;
        }
    std::vector<lbm_instance> inst(n);
    for (int i = 0; i < n; i++) {
        lbm_instance& I = inst[i];
        std::memset(&I, 0, sizeof I);
        I.nx = nx;
        I.ny = ny;
        I.periodic_x = 1;
        I.periodic_y = 0;
        I.tau[0] = I.tau[1] = 1.0;
        I.G = kG;
        I.rho_wall[0] = std::max(-r[i], 0.0);
        I.rho_wall[1] = std::max(r[i], 0.0);
        I.mask = mask.data();
        I.rho_init = rho.data();
        I.disp_threshold = 0.5 * nx;
        I.collision = 0;
    }
    lbm_batch_t* b = nullptr;
    int rc = lbm_batch_create(inst.data(), n, precision, 3, stream, &b);
    if (rc) return batch_error("calibration batch", rc, nullptr);
    std::vector<lbm_obs> obs(n);
    std::vector<double> f((size_t)18 * nn), dens(2 * nn);
    rc = lbm_batch_step(b, steps);
    if (!rc) rc = lbm_batch_observables(b, obs.data());
    if (rc) {
        const int e = batch_error("calibration run", rc, b);
        lbm_batch_destroy(b);
        return e;
    }
    for (int i = 0; i < n && !rc; i++) {
        rc = lbm_batch_save(b, i, f.data());
        if (rc) {
            batch_error("calibration save", rc, b);
            break;
        }
        for (int a = 0; a < 2; a++)
            for (size_t k = 0; k < nn; k++) {
                double s = 0.0;
                for (int q = 0; q < 9; q++) s += f[(size_t)(a * 9 + q) * nn + k];
                dens[a * nn + k] = s;
            }
        double tr, tl;
        if (!contact_angle(dens.data(), nx, ny, 1, H, true, &tr) ||
            !contact_angle(dens.data(), nx, ny, 1, H, false, &tl)) {
            rc = cfail(LBM_EINVAL, "calibration: no interface found for r = %g", r[i]);
            break;
        }
        theta[i] = 0.5 * (tr + tl);
    }
    lbm_batch_destroy(b);
    return rc;
}

int laplace(int64_t steps, int32_t precision, void* stream, double* sigma, double* rho_bulk) {
    // four droplets in a periodic box, and a flat interface (two bands in a
    // periodic 128 x 4 strip) for the bulk density at zero curvature
    const int N = kLaplaceN;
    const size_t nn = (size_t)N * N;
    constexpr int nd = 4;
    const int fx = N, fy = 4;
    const size_t nf = (size_t)fx * fy;
    std::vector<uint8_t> mask(nn, 0);
    std::vector<std::vector<double>> rho(nd + 1);
    std::vector<lbm_instance> inst(nd + 1);
    const double c = N / 2.0;
    for (int d = 0; d <= nd; d++) {
        const bool flat = d == nd;
        const int nx = flat ? fx : N, ny = flat ? fy : N;
        const size_t n = (size_t)nx * ny;
        rho[d].resize(2 * n);
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                double s;
                if (flat) {
                    s = step2(x - fx / 4.0) - step2(x - 3.0 * fx / 4.0);
                } else {
                    const double r = std::sqrt((x - c) * (x - c) + (y - c) * (y - c));
                    s = step2(kLaplaceR[d] - r);
                }
                const double ro = kRhoLo + (kRhoHi - kRhoLo) * s;
                rho[d][(size_t)y * nx + x] = ro;
                rho[d][n + (size_t)y * nx + x] = kRhoHi + kRhoLo - ro;
            }
        lbm_instance& I = inst[d];
        std::memset(&I, 0, sizeof I);
        I.nx = nx;
        I.ny = ny;
        I.periodic_x = I.periodic_y = 1;
        I.tau[0] = I.tau[1] = 1.0;
        I.G = kG;
        I.mask = mask.data();
        I.rho_init = rho[d].data();
        I.disp_threshold = nx;
    }
    lbm_batch_t* b = nullptr;
    int rc = lbm_batch_create(inst.data(), nd + 1, precision, 3, stream, &b);
    if (rc) return batch_error("Laplace batch", rc, nullptr);
    std::vector<lbm_obs> obs(nd + 1);
    rc = lbm_batch_step(b, steps);
    if (!rc) rc = lbm_batch_observables(b, obs.data());
    if (rc) {
        const int e = batch_error("Laplace run", rc, b);
        lbm_batch_destroy(b);
        return e;
    }
    std::vector<double> f((size_t)18 * nn), ro(nn), rw(nn);
    auto densities = [&](int d, size_t n) {
        int e = lbm_batch_save(b, d, f.data());
        if (e) return batch_error("Laplace save", e, b);
        for (size_t k = 0; k < n; k++) {
            double a = 0.0, w = 0.0;
            for (int q = 0; q < 9; q++) {
                a += f[(size_t)q * n + k];
                w += f[(size_t)(9 + q) * n + k];
            }
            ro[k] = a;
            rw[k] = w;
        }
        return (int)LBM_OK;
    };
    double inv_r[nd], dp[nd];
    for (int d = 0; d < nd && !rc; d++) {
        rc = densities(d, nn);
        if (rc) break;
        const int ic = N / 2;
        const size_t kc = (size_t)ic * N + ic;
        // radius: where rho^o crosses the mean of its inside and outside
        // values along the central row and column (the centre of the tanh
        // profile of Eq. den-fitting), half the chord, averaged
        const double mid = 0.5 * (ro[kc] + ro[0]);
        double rsum = 0.0;
        for (int dir = 0; dir < 2; dir++) {
            auto at = [&](int t) { return dir ? ro[(size_t)t * N + ic] : ro[(size_t)ic * N + t]; };
            double xl = 0.0, xr = 0.0;
            for (int t = 0; t + 1 < N; t++) {
                const double a = at(t), bb = at(t + 1);
                if (a <= mid && bb > mid) xl = t + (mid - a) / (bb - a);
                if (a > mid && bb <= mid) xr = t + (a - mid) / (a - bb);
            }
            rsum += 0.5 * (xr - xl);
        }
        const double R = 0.5 * rsum;
        // pressure jump between the centre and the far corner, from the
        // mixture equation of state p = T0 rho - G T0 rho^o rho^w
        auto pr = [&](size_t k) { return kT0 * (ro[k] + rw[k]) - kG * kT0 * ro[k] * rw[k]; };
        inv_r[d] = 1.0 / R;
        dp[d] = pr(kc) - pr(0);
    }
    if (!rc) {
        rc = densities(nd, nf);
        // the middle of the oil band
        const size_t k = (size_t)(fy / 2) * fx + fx / 2;
        if (!rc) *rho_bulk = ro[k] + rw[k];
    }
    lbm_batch_destroy(b);
    if (rc) return rc;
    // least squares dp = sigma / R + c
    double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
    for (int d = 0; d < nd; d++) {
        sx += inv_r[d];
        sy += dp[d];
        sxx += inv_r[d] * inv_r[d];
        sxy += inv_r[d] * dp[d];
    }
    const double den = nd * sxx - sx * sx;
    if (!(den > 0.0)) return cfail(LBM_EINVAL, "Laplace fit: degenerate radii");
    *sigma = (nd * sxy - sx * sy) / den;
    if (!(*sigma > 0.0)) return cfail(LBM_EINVAL, "Laplace fit: non-positive surface tension %g", *sigma);
    return LBM_OK;
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    return dev;
}

// The default table: 13 signed potentials in [-0.6, 0.6], FP32, 20 000 steps.
int default_calibration(void* stream, Calib* out) {
    const int dev = current_device();
    if (dev < 0) return cfail(LBM_ECUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_calib[dev].r.empty()) {
        Calib c;
        for (int i = 0; i < 13; i++) c.r.push_back(-0.6 + 0.1 * i);
        c.theta.resize(c.r.size());
        const int rc = calibrate(c.r.data(), (int)c.r.size(), kCalibSteps, LBM_FP32, stream, c.theta.data());
        if (rc) return rc;
        for (size_t k = 0; k + 1 < c.theta.size(); k++)
            if (!(c.theta[k] > c.theta[k + 1]))
                return cfail(LBM_EINVAL, "calibration: contact angle not decreasing in the wall potential");
        g_calib[dev] = c;
    }
    *out = g_calib[dev];
    return LBM_OK;
}

int default_laplace(void* stream, Laplace* out) {
    const int dev = current_device();
    if (dev < 0) return cfail(LBM_ECUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!(g_laplace[dev].sigma > 0.0)) {
        Laplace l;
        const int rc = laplace(kLaplaceSteps, LBM_FP32, stream, &l.sigma, &l.rho_bulk);
        if (rc) return rc;
        g_laplace[dev] = l;
    }
    *out = g_laplace[dev];
    return LBM_OK;
}

// Wall potentials (rho_s^o, rho_s^w) whose calibrated contact angle is
// theta: linear interpolation of r(theta) in the table (theta descending
// in r), clipped to the calibrated range; r > 0 sets rho_s^w = r, r < 0
// sets rho_s^o = -r.
void potentials_for(const Calib& c, double theta, double* rw) {
    const int n = (int)c.r.size();
    // the table ascending in theta: index k -> n - 1 - k
    auto th = [&](int k) { return c.theta[n - 1 - k]; };
    auto rr = [&](int k) { return c.r[n - 1 - k]; };
    double r;
    if (theta <= th(0)) r = rr(0);
    else if (theta >= th(n - 1)) r = rr(n - 1);
    else {
        int k = 0;
        while (k + 1 < n && th(k + 1) < theta) k++;
        const double t = (theta - th(k)) / (th(k + 1) - th(k));
        r = rr(k) + t * (rr(k + 1) - rr(k));
    }
    rw[0] = std::max(-r, 0.0);
    rw[1] = std::max(r, 0.0);
}

}  // namespace

extern "C" {

int lbm_channel_shape(const lbm_channel_spec* s, int32_t* nx, int32_t* ny) {
    Geom g;
    if (!s || !nx || !ny) return cfail(LBM_EINVAL, "NULL argument");
    if (!geom_of(*s, &g)) return cfail(LBM_EINVAL, "channel spec out of range");
    *nx = g.nx;
    *ny = g.ny;
    return LBM_OK;
}

int lbm_channel_geometry(const lbm_channel_spec* s, uint8_t* mask, double* rho_init) {
    Geom g;
    if (!s) return cfail(LBM_EINVAL, "NULL argument");
    if (!geom_of(*s, &g)) return cfail(LBM_EINVAL, "channel spec out of range");
    fill(g, mask, rho_init);
    return LBM_OK;
}

int lbm_planar_critical_balance_hysteresis(double theta_front_deg, double theta_rear_deg, double area, double h0,
                                           double amp, double lam, double x_rest, double* balance) {
    if (!balance) return cfail(LBM_EINVAL, "NULL argument");
    if (!(theta_front_deg > 0.0 && theta_front_deg < 180.0) || !(theta_rear_deg > 0.0 && theta_rear_deg < 180.0) ||
        !(area > 0.0) || !(h0 > 0.0) || !(amp >= 0.0 && amp < h0) || !(lam > 0.0) || !std::isfinite(x_rest))
        return cfail(LBM_EINVAL, "planar balance: argument out of range");
    return planar_balance2(theta_front_deg, theta_rear_deg, area, h0, amp, lam, x_rest, balance);
}

int lbm_meniscus_angles(const double* rho, int32_t nx, int32_t ny, double h0, double amp, double lam, double* out) {
    if (!rho || !out || nx < 8 || ny < 8 || !(h0 > 0.0) || !(amp >= 0.0 && amp < h0) || !(lam > 0.0))
        return cfail(LBM_EINVAL, "bad argument");
    const size_t n = (size_t)nx * ny;
    const double yc = (ny - 1) / 2.0, k = 2.0 * kPi / lam;
    std::vector<double> frac(n, 0.0);
    for (int y = 1; y < ny - 1; y++)
        for (int x = 0; x < nx; x++) {
            if (std::fabs(y - yc) > h0 - amp * std::cos(k * x)) continue;
            const size_t q = (size_t)y * nx + x;
            const double a = rho[q], b = rho[n + q];
            frac[q] = a + b > 0.0 ? a / (a + b) : 0.0;
        }
    // the slug's ends on the centre row
    const size_t row = (size_t)(ny / 2) * nx;
    int i0 = -1, i1 = -1;
    for (int x = 0; x < nx; x++)
        if (frac[row + x] > 0.5) {
            if (i0 < 0) i0 = x;
            i1 = x;
        }
    if (i0 <= 0 || i1 >= nx - 1) return cfail(LBM_EINVAL, "meniscus angles: no slug inside the period on the centre row");
    for (int side = 0; side < 2; side++) {
        double th, xc, r;
        if (!meniscus_angle(frac, nx, ny, h0, amp, lam, side ? i1 : i0, side == 1, &th, &xc, &r))
            return cfail(LBM_EINVAL, "meniscus angles: too few interface points on the %s meniscus", side ? "front" : "rear");
        out[side] = th;
        out[2 + side] = xc;
        out[4 + side] = r;
    }
    return LBM_OK;
}

int lbm_contact_angle(const double* rho, int32_t nx, int32_t ny, int32_t y_lo, int32_t y_hi, int32_t right,
                      double* theta) {
    if (!rho || !theta || nx < 3 || ny < 3 || y_lo < 0 || y_hi >= ny || y_hi - y_lo < 8)
        return cfail(LBM_EINVAL, "bad argument");
    if (!contact_angle(rho, nx, ny, y_lo, y_hi, right != 0, theta))
        return cfail(LBM_EINVAL, "contact angle: fewer than three interface points");
    return LBM_OK;
}

int lbm_slug_area(const double* rho, const uint8_t* mask, int32_t nx, int32_t ny, double* out) {
    if (!rho || !mask || !out || nx < 1 || ny < 1) return cfail(LBM_EINVAL, "bad argument");
    const size_t n = (size_t)nx * ny;
    auto frac = [&](size_t k) {
        const double t = rho[k] + rho[n + k];
        return t > 0.0 ? rho[k] / t : 0.0;
    };
    double half = 0.0, paper = 0.0;
    for (int x = 0; x < nx; x++) {
        int fluid = 0, rich = 0, above90 = 0;
        for (int y = 0; y < ny; y++) {
            const size_t k = (size_t)y * nx + x;
            if (mask[k]) continue;
            const double q = frac(k);
            fluid++;
            rich += q > 0.5;
            above90 += q > 0.9;
        }
        half += rich;
        if (rich == fluid && fluid > 0) paper += fluid;     // bulk column
        else if (rich > 0) paper += above90;                // a meniscus crosses it
    }
    out[0] = half;
    out[1] = paper;
    return LBM_OK;
}

int lbm_wall_potentials(const double* r, const double* theta, int32_t n, double theta_deg, double* rho_wall) {
    if (!r || !theta || !rho_wall || n < 2 || !std::isfinite(theta_deg)) return cfail(LBM_EINVAL, "bad argument");
    Calib c;
    c.r.assign(r, r + n);
    c.theta.assign(theta, theta + n);
    for (int k = 0; k < n; k++)
        if (!std::isfinite(c.r[k]) || !std::isfinite(c.theta[k]))
            return cfail(LBM_EINVAL, "calibration table: entry %d is not finite", k);
    for (int k = 0; k + 1 < n; k++)
        if (!(c.r[k] < c.r[k + 1]) || !(c.theta[k] > c.theta[k + 1]))
            return cfail(LBM_EINVAL, "calibration table: r must ascend and theta descend");
    potentials_for(c, theta_deg, rho_wall);
    return LBM_OK;
}

int lbm_planar_critical_balance(double theta_deg, double area, double h0, double amp, double lam, double x_rest,
                                double* balance) {
    if (!balance) return cfail(LBM_EINVAL, "NULL argument");
    if (!(theta_deg > 0.0 && theta_deg < 180.0) || !(area > 0.0) || !(h0 > 0.0) || !(amp >= 0.0 && amp < h0) ||
        !(lam > 0.0) || !std::isfinite(x_rest))
        return cfail(LBM_EINVAL, "planar balance: argument out of range");
    return planar_balance(theta_deg, area, h0, amp, lam, x_rest, balance);
}

int lbm_wetting_calibrate(const double* r, int32_t n, int64_t steps, int32_t precision, void* cuda_stream,
                          double* theta) {
    if (!r || !theta || n < 2 || steps < 1) return cfail(LBM_EINVAL, "bad argument");
    for (int i = 0; i < n; i++)
        if (!std::isfinite(r[i]) || std::fabs(r[i]) > 2.0) return cfail(LBM_EINVAL, "r[%d] out of range", i);
    return calibrate(r, n, steps, precision, cuda_stream, theta);
}

int lbm_surface_tension(int64_t steps, int32_t precision, void* cuda_stream, double* sigma, double* rho_bulk) {
    if (!sigma || !rho_bulk || steps < 1) return cfail(LBM_EINVAL, "bad argument");
    return laplace(steps, precision, cuda_stream, sigma, rho_bulk);
}

int lbm_critical_pressure_channels(const lbm_channel_spec* specs, int32_t n, const lbm_channel_opts* o,
                                   lbm_channel_result* out) {
    if (!specs || !o || !out || n < 1) return cfail(LBM_EINVAL, "bad argument");
    std::vector<Geom> geo(n);
    for (int i = 0; i < n; i++)
        if (!geom_of(specs[i], &geo[i])) return cfail(LBM_EINVAL, "spec %d out of range", i);
    if (o->use_surrogate && !o->surrogate) return cfail(LBM_EINVAL, "use_surrogate needs a surrogate network");
    // wettability table
    Calib cal;
    if (o->calib_n > 0) {
        if (!o->calib_r || !o->calib_theta || o->calib_n < 2) return cfail(LBM_EINVAL, "bad calibration table");
        cal.r.assign(o->calib_r, o->calib_r + o->calib_n);
        cal.theta.assign(o->calib_theta, o->calib_theta + o->calib_n);
        for (int k = 0; k < o->calib_n; k++)
            if (!std::isfinite(cal.r[k]) || !std::isfinite(cal.theta[k]))
                return cfail(LBM_EINVAL, "calibration table: entry %d is not finite", k);
        for (int k = 0; k + 1 < o->calib_n; k++)
            if (!(cal.r[k] < cal.r[k + 1]) || !(cal.theta[k] > cal.theta[k + 1]))
                return cfail(LBM_EINVAL, "calibration table: r must ascend and theta descend");
    } else {
        const int rc = default_calibration(o->cuda_stream, &cal);
        if (rc) return rc;
    }
    // surface tension and bulk density of the Bond number
    Laplace lap;
    if (o->sigma > 0.0 && o->rho_bulk > 0.0) {
        lap.sigma = o->sigma;
        lap.rho_bulk = o->rho_bulk;
    } else {
        const int rc = default_laplace(o->cuda_stream, &lap);
        if (rc) return rc;
    }
    // instances and starting brackets
    std::vector<std::vector<uint8_t>> masks(n);
    std::vector<std::vector<double>> rhos(n);
    std::vector<lbm_instance> inst(n);
    std::vector<double> lo(n), hi(n);
    std::vector<float> feat;
    for (int i = 0; i < n; i++) {
        const Geom& g = geo[i];
        const lbm_channel_spec& s = specs[i];
        const size_t nn = (size_t)g.nx * g.ny;
        masks[i].resize(nn);
        rhos[i].resize(2 * nn);
        fill(g, masks[i].data(), rhos[i].data());
        lbm_channel_result& r = out[i];
        std::memset(&r, 0, sizeof r);
        r.nx = g.nx;
        r.ny = g.ny;
        potentials_for(cal, s.theta_deg, r.rho_wall);
        const double nu_w = (1.0 - 0.5) / 3.0;
        r.tau[0] = std::max(3.0 * s.visc_ratio * nu_w + 0.5, kTauMin);
        r.tau[1] = 1.0;
        lbm_instance& I = inst[i];
        std::memset(&I, 0, sizeof I);
        I.nx = g.nx;
        I.ny = g.ny;
        I.periodic_x = 1;
        I.periodic_y = 0;
        I.tau[0] = r.tau[0];
        I.tau[1] = r.tau[1];
        I.G = kG;
        I.rho_wall[0] = r.rho_wall[0];
        I.rho_wall[1] = r.rho_wall[1];
        I.mask = masks[i].data();
        I.rho_init = rhos[i].data();
        I.disp_threshold = 0.5 * g.lam;
        I.collision = o->collision;
        // planar balance of the initial fill: oil area between the contact
        // chords, rest at the rear end
        const double k = 2.0 * kPi / g.lam;
        const double area = 2.0 * g.h0 * (2.0 * g.half) -
                            2.0 * g.amp / k * (std::sin(k * (g.centre + g.half)) - std::sin(k * (g.centre - g.half)));
        double bal = 0.0;
        const int rc = planar_balance(s.theta_deg, area, g.h0, g.amp, g.lam, g.centre - g.half, &bal);
        if (rc) return cfail(rc, "spec %d: %s", i, g_chan_err.c_str());
        // every slug resists with the same capillary balance: rho g L = n_slugs sigma bal
        r.g_analytic = g.slugs * (lap.sigma * bal / (lap.rho_bulk * g.nx));
        if (o->use_surrogate) {
            const double neck = 2.0 * (g.h0 - g.amp);
            const double x[5] = {s.amp_ratio, s.slug_len_over_lambda, std::cos(s.theta_deg * kPi / 180.0),
                                 std::log(s.visc_ratio), 1.0 / neck};
            for (int q = 0; q < 5; q++) {
                const double sd = o->feature_std[q] != 0.0f ? (double)o->feature_std[q] : 1.0;
                feat.push_back((float)((x[q] - (double)o->feature_mean[q]) / sd));
            }
        } else {
            const double flo = o->bracket_lo > 0.0 ? o->bracket_lo : 0.5;
            const double fhi = o->bracket_hi > flo ? o->bracket_hi : 2.0;
            lo[i] = flo * r.g_analytic;
            hi[i] = fhi * r.g_analytic;
            if (!(lo[i] > 0.0)) {
                // no capillary resistance in the planar balance: start from a
                // bracket around a small force and let the bracket checks widen it
                lo[i] = 1e-7;
                hi[i] = 4e-7;
            }
        }
    }
    if (o->use_surrogate) {
        std::vector<float> y(2 * (size_t)n);
        const int rc = lbm_mlp_forward(o->surrogate, feat.data(), n, y.data());
        if (rc) return cfail(rc, "surrogate forward: %s", lbm_mlp_last_error());
        const double ks = o->k_sigma > 0.0 ? o->k_sigma : 2.0;
        for (int i = 0; i < n; i++) {
            const double mu = (double)y[2 * i], ls = (double)y[2 * i + 1];
            const double half = std::max(ks * std::exp(0.5 * ls), 0.5 * std::log(kSurrogateFloor));
            lo[i] = std::exp(mu - half);
            hi[i] = std::exp(mu + half);
        }
    }
    for (int i = 0; i < n; i++) {
        out[i].g_start_lo = lo[i];
        out[i].g_start_hi = hi[i];
    }
    lbm_batch_t* b = nullptr;
    int rc = lbm_batch_create(inst.data(), n, o->precision, 3, o->cuda_stream, &b);
    if (rc) return batch_error("channel batch", rc, nullptr);
    lbm_bisect_opts bo;
    std::memset(&bo, 0, sizeof bo);
    bo.rel_bracket = o->rel_bracket > 0.0 ? o->rel_bracket : 0.02;
    bo.t_eq = o->t_eq;
    bo.t_obs = o->t_obs;
    bo.max_probes = o->max_probes > 0 ? o->max_probes : 24;
    bo.check_bracket = 1;
    bo.timeout_s = o->timeout_s;
    std::vector<lbm_crit_result> res(n);
    rc = lbm_critical_pressure_batch(b, lo.data(), hi.data(), &bo, res.data());
    if (rc && rc != LBM_ETIMEOUT) {
        const int e = batch_error("bisection", rc, b);
        lbm_batch_destroy(b);
        return e;
    }
    const int status = rc;
    lbm_batch_destroy(b);
    for (int i = 0; i < n; i++) {
        const Geom& g = geo[i];
        lbm_channel_result& r = out[i];
        r.g_lo = res[i].g_lo;
        r.g_hi = res[i].g_hi;
        r.probes = res[i].probes;
        r.status = res[i].status;
        // Eq. (Bo_number): Bo = rho g L D / sigma, L the periodic length, D
        // the neck half-width
        const double D = g.h0 - g.amp;
        r.bo_lo = lap.rho_bulk * r.g_lo * g.nx * D / lap.sigma;
        r.bo_hi = lap.rho_bulk * r.g_hi * g.nx * D / lap.sigma;
        r.sigma = lap.sigma;
        r.rho_bulk = lap.rho_bulk;
    }
    if (status) return cfail(status, "bisection stopped by timeout_s");
    return LBM_OK;
}

const char* lbm_channel_last_error(void) { return g_chan_err.c_str(); }

}  // extern "C"
