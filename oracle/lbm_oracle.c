/*
 * Plain FP64 CPU oracle of the coupled lattice Boltzmann model of
 * arXiv 2102.12663 (Sec. 2.3).  TEST INFRASTRUCTURE ONLY: the CUDA library
 * never links, loads or calls this file.
 *
 * One time step n -> n+1 is done with two lattices (read f, write fn) in the
 * order the paper gives: moments (Eq. 9, Eq. 13), buoyancy force (Eq. 17),
 * flow BGK collision with Guo's incompressible equilibrium (Eqs. 6-8), Darcy
 * drag in porous cells (Eq. 4), thermal BGK collision (Eqs. 11-12), then
 * streaming with link-wise boundary rules.
 *
 * Readings where the paper is silent or garbled (all listed in the design
 * notes, with reasons):
 *   - sigma = 5/12, lambda = 1/3, gamma = 1/12 (Eq. 7 fixes only two relations);
 *   - Eq. 17 applied to every axis link: F_i = (1/2) e_i . F for i = 1..4, so
 *     sum_i e_i F_i = F for gravity in any direction, plus an optional uniform
 *     drive used by the closed-form test flows;
 *   - Eq. 11 read as the standard BGK update;
 *   - no-slip walls: halfway bounce-back (Bouzidi's scheme at q = 1/2); on
 *     request, Bouzidi's linear interpolated rule on the curved cold wall
 *     (the cornea circle), with q from the exact link-circle intersection;
 *   - inlet: moving-wall bounce-back; outlet: pressure anti-bounce-back;
 *   - thermal Dirichlet walls: anti-bounce-back ("extrapolation" at q = 1/2);
 *   - TM: porous cells with an implicit mid-step Darcy drag.
 * Build with -ffp-contract=off: no fused multiply-add anywhere.
 */
#include "lbm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* D2Q9 velocities; i = 2, 4 is the vertical pair, as Eq. 17 requires. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* weights omega_i of Eq. 8 */
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* free constants of Eq. 7: lambda + gamma = sigma, lambda + 2 gamma = 1/2 */
static const double SIGMA = 5.0 / 12.0;
static const double LAMBDA = 1.0 / 3.0;
static const double GAMMA = 1.0 / 12.0;

static int g_threads = 1;
void orc_set_threads(int32_t n) { g_threads = n < 1 ? 1 : n; }
int32_t orc_get_threads(void) { return g_threads; }

static int is_active(uint8_t t) { return t == ORC_FLUID || t == ORC_POROUS; }

/* SplitMix64 (Steele, Lea & Flood 2014): advance the state by the golden
 * gamma and return the mixed value. */
uint64_t orc_splitmix64(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The builder's own analytic eye (the paper's Fig. 1 is not in the text; the
 * dimensions of Tab. 1 do not fit a 2:1 grid).  Cell centres sit at integer
 * coordinates; x runs across the chamber, y along the optical axis.
 *   - solid outer ring (adiabatic);
 *   - iris/lens band y < band (hot wall) between the two angle points, sclera
 *     (adiabatic) outside them;
 *   - ciliary inlet: the top band row over an inlet_w-wide gap at the pupil
 *     centre, parabolic inflow along +y;
 *   - cornea: circular arc over the chord y = band - 1/2 between the angle
 *     points, sagitta h = a tan(alpha/2) so that the arc meets the chord at the
 *     chamber angle alpha; cells outside the arc are cornea (cold wall);
 *   - trabecular meshwork: a tm_w-wide box either side of each angle point,
 *     tm_h rows high, made porous where it lies outside the arc, with a
 *     one-cell outlet column behind it.
 * Mirror-symmetric about x = (nx - 1) / 2.  Returns 0, or -1 on a geometry
 * that does not fit the grid. */
int orc_eye_mask(int32_t nx, int32_t ny, double angle_deg, int32_t band,
                 int32_t inlet_w, int32_t tm_w, int32_t tm_h,
                 uint8_t* type, orc_geom* geom)
{
    if (nx < 16 || ny < 8 || !(angle_deg > 0.0 && angle_deg < 180.0)) return -1;
    if (band <= 0) band = (int32_t)floor(ny / 10.0 + 0.5);
    if (inlet_w <= 0) {
        inlet_w = (int32_t)floor(4.0 * nx / 160.0 + 0.5);
        if (inlet_w < 2) inlet_w = 2;
    }
    if ((nx - inlet_w) % 2 != 0) inlet_w += 1;
    if (tm_w <= 0) {
        tm_w = (int32_t)floor(6.0 * nx / 160.0 + 0.5);
        if (tm_w < 2) tm_w = 2;
    }
    if (tm_h <= 0) {
        tm_h = (int32_t)floor(10.0 * nx / 160.0 + 0.5);
        if (tm_h < 2) tm_h = 2;
    }
    const int32_t xa = tm_w + 2; /* first chamber column at the left angle */
    const double a = 0.5 * nx - xa;       /* half chord */
    const double xc = 0.5 * (nx - 1);
    const double ych = band - 0.5;        /* chord on the iris surface */
    const double h = a * tan(angle_deg * M_PI / 360.0);
    const double R = (a * a + h * h) / (2.0 * h);
    const double yc = ych + h - R;
    const int32_t xin0 = (nx - inlet_w) / 2;
    if (band < 2 || a <= tm_w + 1 || ych + h >= ny - 1.5 || band + tm_h >= ny - 1 ||
        inlet_w >= 2 * a - 2)
        return -1;
    for (int32_t y = 0; y < ny; ++y) {
        for (int32_t x = 0; x < nx; ++x) {
            int32_t xm = x < nx - 1 - x ? x : nx - 1 - x;
            uint8_t t;
            if (x == 0 || y == 0 || x == nx - 1 || y == ny - 1) {
                t = ORC_ADIABATIC;
            } else if (y < band) {
                if (y == band - 1 && x >= xin0 && x < xin0 + inlet_w) t = ORC_INLET;
                else if (xm >= xa) t = ORC_HOT;
                else t = ORC_ADIABATIC;
            } else {
                double dx = x - xc, dy = y - yc;
                int in_tm_rows = y < band + tm_h;
                if (dx * dx + dy * dy < R * R) t = ORC_FLUID;
                else if (in_tm_rows && xm >= xa - tm_w && xm < xa + tm_w) t = ORC_POROUS;
                else if (in_tm_rows && xm == xa - tm_w - 1) t = ORC_OUTLET;
                else if (xm >= xa) t = ORC_COLD;
                else t = ORC_ADIABATIC;
            }
            type[(int64_t)y * nx + x] = t;
        }
    }
    geom->nx = nx;
    geom->ny = ny;
    geom->periodic_x = 0;
    geom->periodic_y = 0;
    geom->inlet_dir_x = 0;
    geom->inlet_dir_y = 1;
    geom->inlet_profile = 1;
    geom->inlet_lo = xin0;
    geom->inlet_width = inlet_w;
    geom->eye_normals = 1;
    geom->outlet_axis = 0;
    geom->arc_xc = xc;
    geom->arc_yc = yc;
    geom->arc_r = R;
    return 0;
}

/* Eq. 8 */
static double S_i(int i, double ux, double uy)
{
    double eu = EX[i] * ux + EY[i] * uy;
    double usq = ux * ux + uy * uy;
    return W[i] * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
}

/* Eq. 7 with c = 1 */
void orc_feq(double p, double ux, double uy, double feq[9])
{
    feq[0] = -4.0 * SIGMA * p + S_i(0, ux, uy);
    for (int i = 1; i <= 4; ++i) feq[i] = LAMBDA * p + S_i(i, ux, uy);
    for (int i = 5; i <= 8; ++i) feq[i] = GAMMA * p + S_i(i, ux, uy);
}

/* Eq. 9 with c = 1: u = sum_i e_i f_i, p = [sum_{i>=1} f_i + S_0(u)] / (4 sigma) */
void orc_moments(const double f[9], double* p, double* ux, double* uy)
{
    double sx = 0.0, sy = 0.0, s = 0.0;
    for (int i = 0; i < 9; ++i) {
        sx += EX[i] * f[i];
        sy += EY[i] * f[i];
    }
    for (int i = 1; i < 9; ++i) s += f[i];
    *ux = sx;
    *uy = sy;
    *p = (s + S_i(0, sx, sy)) / (4.0 * SIGMA);
}

/* Eq. 13 */
static double temperature(const double g[4]) { return g[0] + g[1] + g[2] + g[3]; }

/* Body force per unit mass: uniform drive minus the Boussinesq term of Eq. 16. */
static void body_force(const orc_params* P, double Tm, double* Fx, double* Fy)
{
    double gb = P->g_beta * (Tm - P->T0);
    *Fx = P->drive[0] - gb * P->g_dir[0];
    *Fy = P->drive[1] - gb * P->g_dir[1];
}

/* Collision of one cell: Eq. 6 (flow, forcing of Eq. 17), Eq. 4 (Darcy drag in
 * porous cells, implicit in the post-collision momentum), Eqs. 11-12 (heat). */
void orc_collide(const orc_params* P, int porous, const double f[9],
                 const double g[4], double fs[9], double gs[4])
{
    double p, ux, uy, feq[9], F[9];
    orc_moments(f, &p, &ux, &uy);
    orc_feq(p, ux, uy, feq);
    double Tm = temperature(g);
    double Fx, Fy;
    body_force(P, Tm, &Fx, &Fy);
    for (int i = 0; i < 9; ++i) F[i] = 0.0;
    for (int i = 1; i <= 4; ++i) F[i] = 0.5 * (EX[i] * Fx + EY[i] * Fy);
    double omega = 1.0 / P->tau;
    for (int i = 0; i < 9; ++i) fs[i] = f[i] - omega * (f[i] - feq[i]) + F[i];
    if (porous) {
        /* Darcy drag of Eq. 4, F_D = -(nu/K) u_m, taken at the mid-step velocity
         * u_m = u + (F + F_D)/2 (the velocity whose face flux the streaming
         * conserves), solved implicitly: u_m = (u + F/2) / (1 + nu/(2K)).
         * nu from Eq. 10.  The drag enters f through its first moment only. */
        double nu = (2.0 * P->tau - 1.0) / 6.0;
        double cK = nu / P->K;
        double den = 1.0 + 0.5 * cK;
        double umx = (ux + 0.5 * Fx) / den;
        double umy = (uy + 0.5 * Fy) / den;
        double FDx = -cK * umx;
        double FDy = -cK * umy;
        for (int i = 1; i < 9; ++i) fs[i] += 3.0 * W[i] * (EX[i] * FDx + EY[i] * FDy);
    }
    double omegaT = 1.0 / P->tau_T;
    double Tq = 0.25 * Tm;
    for (int i = 1; i <= 4; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double teq = Tq * (1.0 + 2.0 * eu); /* Eq. 12 */
        gs[i - 1] = g[i - 1] - omegaT * (g[i - 1] - teq);
    }
}

/* neighbour of (x, y) along e_i; returns -1 outside a non-periodic edge */
static int64_t neighbour(const orc_geom* G, int x, int y, int i)
{
    int xn = x + EX[i], yn = y + EY[i];
    if (G->periodic_x) xn = (xn + G->nx) % G->nx;
    if (G->periodic_y) yn = (yn + G->ny) % G->ny;
    if (xn < 0 || xn >= G->nx || yn < 0 || yn >= G->ny) return -1;
    return (int64_t)yn * G->nx + xn;
}

static void inlet_velocity(const orc_geom* G, const orc_params* P, int64_t cell,
                           double* ux, double* uy)
{
    int x = (int)(cell % G->nx), y = (int)(cell / G->nx);
    double shape = 1.0;
    if (G->inlet_profile == 1) {
        int c = G->inlet_dir_x == 0 ? x : y;
        double s = ((double)(c - G->inlet_lo) + 0.5) / (double)G->inlet_width;
        shape = 4.0 * s * (1.0 - s);
    }
    double u = P->u_in_max * shape;
    *ux = u * G->inlet_dir_x;
    *uy = u * G->inlet_dir_y;
}

static void gather(const double* f, const double* T, int64_t N, int64_t c,
                   double fc[9], double gc[4])
{
    for (int i = 0; i < 9; ++i) fc[i] = f[i * N + c];
    for (int i = 0; i < 4; ++i) gc[i] = T[i * N + c];
}

/* Fraction q of the link from cell centre (x, y) along e_i at which it
 * leaves the circle of centre (arc_xc, arc_yc) and radius arc_r: the positive
 * root t of |P + t e_i - C|^2 = R^2 (P inside, so c < 0), written with the
 * half coefficient: a = |e_i|^2, bh = (P - C) . e_i, c = |P - C|^2 - R^2,
 * t = (-bh + sqrt(bh^2 - a c)) / a. */
double orc_link_q(const orc_geom* G, int32_t x, int32_t y, int32_t i)
{
    const double dx = x - G->arc_xc, dy = y - G->arc_yc;
    const double a = (double)(EX[i] * EX[i] + EY[i] * EY[i]);
    const double bh = dx * EX[i] + dy * EY[i];
    const double c = dx * dx + dy * dy - G->arc_r * G->arc_r;
    return (-bh + sqrt(bh * bh - a * c)) / a;
}

/* Post-collision populations of the active cell c (its own collision, as in
 * orc_step). */
static void post_collision(const orc_params* P, const uint8_t* type, const double* f,
                           const double* T, int64_t N, int64_t c, double fs[9])
{
    double fc[9], gc[4], gs[4];
    for (int i = 0; i < 9; ++i) fc[i] = f[i * N + c];
    for (int i = 0; i < 4; ++i) gc[i] = T[i * N + c];
    orc_collide(P, type[c] == ORC_POROUS && P->tm_model == 0, fc, gc, fs, gs);
}

void orc_step(const orc_geom* G, const orc_params* P, const uint8_t* type,
              const double* f, const double* T, double* fn, double* Tn,
              double* q_in_out, double* q_out_out)
{
    const int nx = G->nx, ny = G->ny;
    const int64_t N = (int64_t)nx * ny;
    double q_in = 0.0, q_out = 0.0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) reduction(+ : q_in, q_out) schedule(static)
#endif
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t c = (int64_t)y * nx + x;
            if (!is_active(type[c])) continue;
            double fc[9], gc[4], fs[9], gs[4], p, ux, uy;
            gather(f, T, N, c, fc, gc);
            orc_moments(fc, &p, &ux, &uy);
            double usq = ux * ux + uy * uy;
            double Tm = temperature(gc);
            /* the lumped TM of Sec. 2.3 resolves no Darcy flow inside the TM block */
            orc_collide(P, type[c] == ORC_POROUS && P->tm_model == 0, fc, gc, fs, gs);
            fn[c] = fs[0];
            for (int i = 1; i < 9; ++i) {
                int64_t nb = neighbour(G, x, y, i);
                uint8_t tn = nb < 0 ? ORC_ADIABATIC : type[nb];
                int o = OPP[i];
                if (is_active(tn)) {
                    fn[i * N + nb] = fs[i];
                } else if (tn == ORC_INLET) {
                    double uix, uiy;
                    inlet_velocity(G, P, nb, &uix, &uiy);
                    double v = fs[i] - 6.0 * W[i] * (EX[i] * uix + EY[i] * uiy);
                    fn[o * N + c] = v;
                    q_in += v - fs[i];
                } else if (tn == ORC_OUTLET && P->tm_model == 1) {
                    /* lumped TM (Sec. 2.3): the seepage velocity, directed out
                     * of the domain along the outlet axis, as a moving wall */
                    double uwx = G->outlet_axis == 0 ? P->u_seep * EX[i] : 0.0;
                    double uwy = G->outlet_axis == 1 ? P->u_seep * EY[i] : 0.0;
                    double v = fs[i] - 6.0 * W[i] * (EX[i] * uwx + EY[i] * uwy);
                    fn[o * N + c] = v;
                    q_out += fs[i] - v;
                } else if (tn == ORC_OUTLET) {
                    double eu = EX[i] * ux + EY[i] * uy;
                    double kappa = i <= 4 ? LAMBDA : GAMMA;
                    double v = -fs[i] + 2.0 * (kappa * P->p_out + W[i] * (4.5 * eu * eu - 1.5 * usq));
                    fn[o * N + c] = v;
                    q_out += fs[i] - v;
                } else if (tn == ORC_COLD && P->bouzidi && G->arc_r > 0.0 &&
                           type[c] == ORC_FLUID) {
                    /* Bouzidi's linear interpolated bounce-back on the curved
                     * cornea, the wall at fraction q of the link:
                     *   q < 1/2: f_o(x) = 2q f*_i(x) + (1 - 2q) f*_i(x - e_i),
                     *   q > 1/2: f_o(x) = f*_i(x) / (2q) + (2q - 1)/(2q) f*_o(x);
                     * halfway at q = 1/2 and where x - e_i is not active. */
                    double q = orc_link_q(G, x, y, i);
                    int64_t up = neighbour(G, x, y, o);
                    if (q < 0.5 && up >= 0 && is_active(type[up])) {
                        double fu[9];
                        post_collision(P, type, f, T, N, up, fu);
                        fn[o * N + c] = (2.0 * q) * fs[i] + (1.0 - 2.0 * q) * fu[i];
                    } else if (q > 0.5) {
                        fn[o * N + c] = (1.0 / (2.0 * q)) * fs[i] + ((2.0 * q - 1.0) / (2.0 * q)) * fs[o];
                    } else {
                        fn[o * N + c] = fs[i];
                    }
                } else {
                    fn[o * N + c] = fs[i]; /* halfway bounce-back */
                }
            }
            for (int i = 1; i <= 4; ++i) {
                int64_t nb = neighbour(G, x, y, i);
                uint8_t tn = nb < 0 ? ORC_ADIABATIC : type[nb];
                int o = OPP[i];
                double v = gs[i - 1];
                if (is_active(tn)) {
                    Tn[(i - 1) * N + nb] = v;
                    continue;
                }
                switch (tn) {
                case ORC_COLD: v = -gs[i - 1] + 0.5 * P->T_cold; break;
                case ORC_HOT: v = -gs[i - 1] + 0.5 * P->T_hot; break;
                case ORC_INLET: v = -gs[i - 1] + 0.5 * P->T_in; break;
                case ORC_OUTLET: v = -gs[i - 1] + 0.5 * Tm; break;
                default: break; /* adiabatic: bounce-back, zero flux */
                }
                Tn[(o - 1) * N + c] = v;
            }
        }
    }
    if (q_in_out) *q_in_out = q_in;
    if (q_out_out) *q_out_out = q_out;
}

void orc_init(const orc_geom* G, const orc_params* P, const uint8_t* type,
              double* f, double* T)
{
    const int64_t N = (int64_t)G->nx * G->ny;
    double feq[9];
    orc_feq(P->p_out, 0.0, 0.0, feq);
    for (int64_t c = 0; c < N; ++c) {
        int act = is_active(type[c]);
        for (int i = 0; i < 9; ++i) f[i * N + c] = act ? feq[i] : 0.0;
        double noise = 0.0;
        if (act && P->noise_amp != 0.0) {
            uint64_t h = orc_splitmix64(P->seed ^ (uint64_t)c);
            double u01 = (double)(h >> 11) * 0x1.0p-53;
            noise = P->noise_amp * (2.0 * u01 - 1.0);
        }
        for (int i = 0; i < 4; ++i) T[i * N + c] = act ? 0.25 * (P->T0 + noise) : 0.0;
    }
}

/* unit normal of the wall of tissue `tt` seen from fluid cell (x, y) */
static void wall_normal(const orc_geom* G, const uint8_t* type, int x, int y,
                        uint8_t tt, double* nxo, double* nyo)
{
    double ax, ay;
    if (G->eye_normals && tt == ORC_COLD) {
        ax = x - G->arc_xc;
        ay = y - G->arc_yc;
    } else if (G->eye_normals && tt == ORC_HOT) {
        ax = 0.0;
        ay = 1.0;
    } else {
        ax = 0.0;
        ay = 0.0;
        for (int i = 1; i < 9; ++i) {
            int64_t nb = neighbour(G, x, y, i);
            if (nb >= 0 && type[nb] == tt) {
                ax += EX[i];
                ay += EY[i];
            }
        }
    }
    double r = sqrt(ax * ax + ay * ay);
    *nxo = r > 0.0 ? ax / r : 0.0;
    *nyo = r > 0.0 ? ay / r : 0.0;
}

/* |t . sigma . n| with sigma = -(1 - 1/(2 tau)) Pi_neq, Pi_neq = sum e e (f - feq) */
static double wall_shear(const orc_params* P, const double fc[9], const double feq[9],
                         double nx_, double ny_)
{
    double pxx = 0.0, pxy = 0.0, pyy = 0.0;
    for (int i = 0; i < 9; ++i) {
        double d = fc[i] - feq[i];
        pxx += EX[i] * EX[i] * d;
        pxy += EX[i] * EY[i] * d;
        pyy += EY[i] * EY[i] * d;
    }
    double k = -(1.0 - 1.0 / (2.0 * P->tau));
    double sxx = k * pxx, sxy = k * pxy, syy = k * pyy;
    double tx = -ny_, ty = nx_;
    return fabs(tx * (sxx * nx_ + sxy * ny_) + ty * (sxy * nx_ + syy * ny_));
}

void orc_observe(const orc_geom* G, const orc_params* P, const uint8_t* type,
                 const double* f, const double* T, const double* u_snap, orc_obs* o)
{
    const int nx = G->nx, ny = G->ny;
    const int64_t N = (int64_t)nx * ny;
    double sum_p = 0.0, n_fluid = 0.0, mass = 0.0, peak = 0.0, resid = 0.0;
    double wc = 0.0, nc = 0.0, wi = 0.0, ni = 0.0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t c = (int64_t)y * nx + x;
            if (!is_active(type[c])) continue;
            double fc[9], gc[4], p, ux, uy;
            gather(f, T, N, c, fc, gc);
            orc_moments(fc, &p, &ux, &uy);
            double m = 0.0;
            for (int i = 1; i < 9; ++i) m += fc[i];
            mass += m;
            double sp = sqrt(ux * ux + uy * uy);
            if (sp > peak) peak = sp;
            if (u_snap) {
                double dx = ux - u_snap[c], dy = uy - u_snap[N + c];
                double d = sqrt(dx * dx + dy * dy);
                if (d > resid) resid = d;
            }
            if (type[c] != ORC_FLUID) continue;
            sum_p += p;
            n_fluid += 1.0;
            int hit_cold = 0, hit_hot = 0;
            for (int i = 1; i < 9; ++i) {
                int64_t nb = neighbour(G, x, y, i);
                if (nb < 0) continue;
                if (type[nb] == ORC_COLD) hit_cold = 1;
                if (type[nb] == ORC_HOT) hit_hot = 1;
            }
            if (hit_cold || hit_hot) {
                double feq[9], nxw, nyw;
                orc_feq(p, ux, uy, feq);
                if (hit_cold) {
                    wall_normal(G, type, x, y, ORC_COLD, &nxw, &nyw);
                    wc += wall_shear(P, fc, feq, nxw, nyw);
                    nc += 1.0;
                }
                if (hit_hot) {
                    wall_normal(G, type, x, y, ORC_HOT, &nxw, &nyw);
                    wi += wall_shear(P, fc, feq, nxw, nyw);
                    ni += 1.0;
                }
            }
        }
    }
    o->iop = n_fluid > 0.0 ? sum_p / n_fluid : 0.0;
    o->q_in = 0.0;
    o->q_out = 0.0;
    o->mass = mass;
    o->peak = peak;
    o->wss_cornea = nc > 0.0 ? wc / nc : 0.0;
    o->wss_iris = ni > 0.0 ? wi / ni : 0.0;
    o->residual = u_snap ? resid : -1.0;
    o->n_fluid = n_fluid;
    o->n_cornea = nc;
    o->n_iris = ni;
}

/* Lumped TM of Sec. 2.3: Darcy's law (Eq. 4) across a meshwork of thickness
 * h_tm with a linear pressure profile, u_s = (K/mu) (p_IOP - p_0) / h_tm, in
 * kinematic lattice units u_s = K (iop - p_out) / (nu h_tm), nu from Eq. 10. */
double orc_seepage_velocity(const orc_params* P, double iop, double h_tm)
{
    double nu = (2.0 * P->tau - 1.0) / 6.0;
    return P->K * (iop - P->p_out) / (nu * h_tm);
}

void orc_fields(const orc_geom* G, const uint8_t* type, const double* f,
                const double* T, double* u, double* p, double* Tf)
{
    const int64_t N = (int64_t)G->nx * G->ny;
    for (int64_t c = 0; c < N; ++c) {
        if (!is_active(type[c])) {
            u[c] = u[N + c] = p[c] = Tf[c] = 0.0;
            continue;
        }
        double fc[9], gc[4], pp, ux, uy;
        gather(f, T, N, c, fc, gc);
        orc_moments(fc, &pp, &ux, &uy);
        u[c] = ux;
        u[N + c] = uy;
        p[c] = pp;
        Tf[c] = temperature(gc);
    }
}

void orc_run(const orc_geom* G, const orc_params* P, const uint8_t* type,
             double* f, double* T, double* f2, double* T2, int64_t nsteps)
{
    const int64_t N = (int64_t)G->nx * G->ny;
    double *a = f, *b = f2, *ta = T, *tb = T2;
    memcpy(f2, f, sizeof(double) * 9 * N);
    memcpy(T2, T, sizeof(double) * 4 * N);
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_step(G, P, type, a, ta, b, tb, NULL, NULL);
        double* t = a; a = b; b = t;
        t = ta; ta = tb; tb = t;
    }
    if (a != f) {
        memcpy(f, a, sizeof(double) * 9 * N);
        memcpy(T, ta, sizeof(double) * 4 * N);
    }
}

/* ---- vortex measures (Eq. 18, Tab. 3) ------------------------------------
 * omega_z = (1/2)(du_y/dx - du_x/dy) at every fluid cell.  Each derivative is
 * the difference of the two axis neighbours' values over their distance.  An
 * active neighbour contributes its velocity at distance 1; any other one
 * (a wall, inlet or outlet cell, or beyond a non-periodic edge) contributes
 * the no-slip wall value 0 halfway along the link, at distance 1/2.
 * I = 2 * sum omega_z over the fluid cells (cell area 1), and the same with
 * |omega_z|.
 * Stream function psi with u_x = dpsi/dy: per column, the midpoint sum of
 * u_x from y = 0 (u_x = 0 at non-active cells).  Its largest and smallest
 * values over the fluid cells mark the vortex centres; ties go to the lowest
 * flat index y*nx + x. */
static double axis_value(const orc_geom* G, const uint8_t* type, const double* comp, int x,
                         int y, int dx, int dy, double* dist)
{
    int xn = x + dx, yn = y + dy;
    if (G->periodic_x) xn = (xn + G->nx) % G->nx;
    if (G->periodic_y) yn = (yn + G->ny) % G->ny;
    if (xn < 0 || xn >= G->nx || yn < 0 || yn >= G->ny ||
        !is_active(type[(int64_t)yn * G->nx + xn])) {
        *dist = 0.5;
        return 0.0;
    }
    *dist = 1.0;
    return comp[(int64_t)yn * G->nx + xn];
}

void orc_vortex(const orc_geom* G, const uint8_t* type, const double* u, orc_vortex_out* out)
{
    const int nx = G->nx, ny = G->ny;
    const int64_t N = (int64_t)nx * ny;
    const double* ux = u;
    const double* uy = u + N;
    double* psi = (double*)malloc(sizeof(double) * (size_t)N);
    for (int x = 0; x < nx; ++x) {
        double S = 0.0;
        for (int y = 0; y < ny; ++y) {
            const int64_t c = (int64_t)y * nx + x;
            const double v = is_active(type[c]) ? ux[c] : 0.0;
            psi[c] = S + 0.5 * v;
            S = S + v;
        }
    }
    memset(out, 0, sizeof(*out));
    int have = 0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t c = (int64_t)y * nx + x;
            if (type[c] != ORC_FLUID) continue;
            double hr, hl, hu, hd;
            const double vr = axis_value(G, type, uy, x, y, 1, 0, &hr);
            const double vl = axis_value(G, type, uy, x, y, -1, 0, &hl);
            const double vu = axis_value(G, type, ux, x, y, 0, 1, &hu);
            const double vd = axis_value(G, type, ux, x, y, 0, -1, &hd);
            const double duy_dx = (vr - vl) / (hr + hl);
            const double dux_dy = (vu - vd) / (hu + hd);
            const double omega = 0.5 * (duy_dx - dux_dy);
            out->intensity += 2.0 * omega;
            out->intensity_abs += 2.0 * fabs(omega);
            out->n_fluid += 1.0;
            if (!have || psi[c] > out->psi_max) {
                out->psi_max = psi[c];
                out->max_x = x;
                out->max_y = y;
            }
            if (!have || psi[c] < out->psi_min) {
                out->psi_min = psi[c];
                out->min_x = x;
                out->min_y = y;
            }
            have = 1;
        }
    }
    free(psi);
}
