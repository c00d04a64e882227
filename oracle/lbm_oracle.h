/*
 * Plain FP64 CPU oracle of the coupled lattice Boltzmann model of aqueous-humor
 * flow (arXiv 2102.12663, Sec. 2.3, Eqs. 6-17).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library: everything here is written
 * out again from the paper's equations.
 *
 * Arrays are row-major planes: cell (x, y) has index y*nx + x; population i of
 * that cell lives at f[i*nx*ny + idx] (i = 0..8) and thermal population i at
 * T[(i-1)*nx*ny + idx] (i = 1..4).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

/* cell types (numbering is an interface convention shared with the masks
 * that the tests generate) */
enum { ORC_FLUID = 0, ORC_POROUS = 1, ORC_COLD = 2, ORC_HOT = 3,
       ORC_ADIABATIC = 4, ORC_INLET = 5, ORC_OUTLET = 6 };

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    int32_t inlet_dir_x, inlet_dir_y; /* lattice direction of the inflow */
    int32_t inlet_profile;            /* 0 = plug, 1 = parabolic across the gap */
    int32_t inlet_lo, inlet_width;    /* gap start and width, measured along the
                                         axis perpendicular to the inflow */
    int32_t eye_normals;              /* 1: analytic eye wall normals */
    int32_t outlet_axis;              /* 0: outlets drain along x, 1: along y */
    double arc_xc, arc_yc;            /* centre of the cornea arc (eye only) */
    double arc_r;                     /* its radius; 0: no curved wall */
} orc_geom;

typedef struct {
    double tau, tau_T;     /* flow / thermal relaxation times (Eqs. 10, 14) */
    double g_beta;         /* g * beta, lattice units (Eq. 17) */
    double g_dir[2];       /* unit vector of gravity */
    double T_cold, T_hot;  /* cornea / iris-lens wall temperatures */
    double T0;             /* reference temperature of Eq. 5 */
    double T_in;           /* temperature of the secreted inflow */
    double u_in_max;       /* peak inflow speed */
    double K;              /* TM permeability, lattice units (cells^2) */
    double p_out;          /* pressure held at the outlet */
    double drive[2];       /* uniform body force (test flows) */
    double noise_amp;      /* amplitude of the seeded temperature noise */
    uint64_t seed;
    int32_t tm_model;      /* 0: porous TM cells with Darcy drag; 1: the lumped
                              TM of Sec. 2.3 (seepage-velocity outflow) */
    int32_t bouzidi;       /* 1: interpolated bounce-back on the curved cold
                              wall (the circle of orc_geom), 0: halfway */
    double u_seep;         /* lumped TM: current seepage speed out of the outlets */
} orc_params;

typedef struct {
    double iop;          /* mean p over fluid cells */
    double q_in, q_out;  /* boundary fluxes of the step (orc_step only) */
    double mass;         /* sum over active cells of f_1..f_8 */
    double peak;         /* max |u| over active cells */
    double wss_cornea, wss_iris;  /* mean wall shear stress, lattice units */
    double residual;     /* max |u - u_snap| over active cells, -1 if no snapshot */
    double n_fluid, n_cornea, n_iris;
} orc_obs;

uint64_t orc_splitmix64(uint64_t state);
int orc_eye_mask(int32_t nx, int32_t ny, double angle_deg, int32_t band,
                 int32_t inlet_w, int32_t tm_w, int32_t tm_h,
                 uint8_t* type, orc_geom* geom);
void orc_feq(double p, double ux, double uy, double feq[9]);
void orc_moments(const double f[9], double* p, double* ux, double* uy);
void orc_collide(const orc_params* P, int porous, const double f[9],
                 const double g[4], double fs[9], double gs[4]);
void orc_init(const orc_geom* G, const orc_params* P, const uint8_t* type,
              double* f, double* T);
void orc_step(const orc_geom* G, const orc_params* P, const uint8_t* type,
              const double* f, const double* T, double* fn, double* Tn,
              double* q_in, double* q_out);
void orc_observe(const orc_geom* G, const orc_params* P, const uint8_t* type,
                 const double* f, const double* T, const double* u_snap,
                 orc_obs* obs);
double orc_seepage_velocity(const orc_params* P, double iop, double h_tm);
double orc_link_q(const orc_geom* G, int32_t x, int32_t y, int32_t i);

/* Vortex measures of a velocity field (Eq. 18, Tab. 3).  u holds u_x in
 * u[0..N) and u_y in u[N..2N) (values at non-active cells are ignored). */
typedef struct {
    double intensity;      /* sum over fluid cells of 2 omega_z (cell area 1) */
    double intensity_abs;  /* sum over fluid cells of 2 |omega_z| */
    double psi_max, psi_min;         /* extrema of the stream function over fluid cells */
    int32_t max_x, max_y, min_x, min_y;
    double n_fluid;
} orc_vortex_out;
void orc_vortex(const orc_geom* G, const uint8_t* type, const double* u, orc_vortex_out* out);
void orc_fields(const orc_geom* G, const uint8_t* type, const double* f,
                const double* T, double* u, double* p, double* Tf);
void orc_run(const orc_geom* G, const orc_params* P, const uint8_t* type,
             double* f, double* T, double* f2, double* T2, int64_t nsteps);
void orc_set_threads(int32_t n);
int32_t orc_get_threads(void);

#endif
