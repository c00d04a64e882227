/*
 * lbm.h - C ABI of the GB300 (sm_103a) coupled lattice Boltzmann solver for
 * aqueous-humor flow in the anterior chamber (arXiv 2102.12663).
 *
 * Model (Sec. 2.3 of the paper): Guo's incompressible D2Q9 BGK model for flow
 * (Eqs. 6-10) with the Boussinesq buoyancy force of Eqs. 15-17, a D2Q4 BGK
 * model for heat convection and diffusion (Eqs. 11-14), Darcy resistance of the
 * trabecular meshwork (Eq. 4) in porous cells, halfway bounce-back walls
 * (Bouzidi's scheme at q = 1/2), a velocity inlet at the ciliary body, a
 * fixed-pressure outlet behind the meshwork, and fixed-temperature walls on
 * the cornea (Gamma_1) and iris/lens (Gamma_2).  Observables: IOP (Sec. 2.3,
 * "the pressure in AC is just IOP"; Sec. 3.1), inflow and outflow rates
 * (Sec. 3.1, Fig. 2), peak speed (Tab. 3) and the mean cornea and iris wall
 * shear stress (Sec. 3.6, Tabs. 8-9).
 *
 * Conventions for every entry point:
 *  - All quantities are lattice units (c = dx = dt = 1) unless a name ends in
 *    _pa (pascal) or _m / _s (SI).  Cell (x, y) has flat index y*nx + x; x runs
 *    across the chamber, y along the optical axis.
 *  - D2Q9 velocities e_0..e_8 = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
 *    (-1,-1) (1,-1); the D2Q4 heat lattice uses e_1..e_4.
 *  - Every call returns an lbm_status; nothing throws across the ABI.  On an
 *    error, lbm_last_error() returns a message for the calling thread.
 *  - Device memory belongs to the caller: each object lives inside one device
 *    buffer that the caller allocates (lbm_*_bytes gives the size), keeps
 *    alive until the object is destroyed, and frees afterwards.  The library
 *    itself calls no device allocator.  Host-side bookkeeping uses malloc.
 *  - Work is queued on the caller's CUDA stream (a cudaStream_t passed as
 *    void*, 0 = legacy default stream); calls that return data to the host
 *    synchronise that stream.
 *  - Handles are not thread-safe: one thread drives a handle at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = 1,         /* invalid argument; nothing was changed */
    LBM_ENOMEM = 2,         /* caller buffer too small or misaligned */
    LBM_ECUDA = 3,          /* a CUDA runtime call failed */
    LBM_ENOTCONVERGED = 4,  /* lbm_run_to_steady hit max_steps */
    LBM_EUNSTABLE = 5,      /* NaN detected in the observables */
    LBM_EBUSY = 6           /* object in use (batch slot taken, batch full) */
} lbm_status;

/* Storage precision of the populations.  Arithmetic is FP64 for LBM_F64 and
 * FP32 otherwise; reductions always accumulate in FP64.  The 16-bit forms
 * store the flow populations of Guo's model (which vanish at rest, so they are
 * already deviations from the rest weights) scaled by a power of two, and the
 * heat populations as deviations from T0/4. */
typedef enum lbm_precision {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F16DEV = 2,
    LBM_BF16DEV = 3
} lbm_precision;

typedef enum lbm_geom_kind {
    LBM_GEOM_EYE = 0,  /* the library's analytic eye (see lbm_build_mask) */
    LBM_GEOM_MASK = 1  /* caller-supplied cell-type mask */
} lbm_geom_kind;

/* Cell types of a mask (Sec. 2.1 regions: Omega_1 fluid, Omega_3 porous TM,
 * Gamma_1 cornea, Gamma_2 iris/lens, inlet at the ciliary body, outlet behind
 * the TM).  Walls are solid; inlet and outlet cells are boundary cells that
 * are never updated. */
typedef enum lbm_cell_type {
    LBM_CELL_FLUID = 0,
    LBM_CELL_POROUS = 1,
    LBM_CELL_COLD = 2,       /* cornea: no-slip, T = T_cold */
    LBM_CELL_HOT = 3,        /* iris / lens: no-slip, T = T_hot */
    LBM_CELL_ADIABATIC = 4,  /* sclera and outer box: no-slip, zero heat flux */
    LBM_CELL_INLET = 5,      /* prescribed inflow, T = T_in */
    LBM_CELL_OUTLET = 6      /* p = p_out, zero temperature gradient */
} lbm_cell_type;

/* Geometry of one problem (Sec. 2.1, Tab. 1).
 * EYE: nx, ny, chamber_angle_deg and optionally band_cells (iris/lens band
 *      height), inlet_cells (ciliary inlet width), tm_w, tm_h (trabecular
 *      meshwork block); 0 selects the default scaled from the 160 x 80 eye
 *      (band ny/10, inlet 4, TM 6 x 10 cells per 160 columns).
 * MASK: nx, ny, host_mask (ny*nx lbm_cell_type bytes, read during
 *      lbm_create_domain only), periodic_x / periodic_y (wrap-around edges;
 *      every non-periodic edge must hold no fluid or porous cell), and the
 *      inflow: lattice direction (inlet_dir_x, inlet_dir_y), inlet_profile 0
 *      (plug) or 1 (parabolic 4 s (1 - s) over inlet_width cells starting at
 *      inlet_lo, counted along the axis across the inflow). */
typedef struct lbm_geometry_desc {
    int32_t nx, ny;
    int32_t kind;
    int32_t band_cells, inlet_cells, tm_w, tm_h;
    int32_t periodic_x, periodic_y;
    int32_t inlet_dir_x, inlet_dir_y, inlet_profile, inlet_lo, inlet_width;
    double chamber_angle_deg;
    const uint8_t* host_mask;
} lbm_geometry_desc;

/* Summary of a built mask (lbm_build_mask). */
typedef struct lbm_geometry_info {
    int64_t n_cells, n_active, n_fluid, n_porous, n_inlet, n_outlet;
    int32_t inlet_dir_x, inlet_dir_y, inlet_profile, inlet_lo, inlet_width;
    int32_t eye_normals;     /* 1: analytic cornea / iris wall normals */
    int32_t outlet_axis;     /* outlets drain along x (0) or y (1): EYE 0, MASK the
                                inflow axis */
    int32_t reserved;
    double arc_xc, arc_yc;   /* centre of the cornea arc (EYE) */
    double arc_r;            /* its radius (EYE; 0 for MASK) */
} lbm_geometry_info;

/* Physical parameters (lattice units).  May change between steps.
 *  tau, tau_T   relaxation times, nu = (2 tau - 1)/6 (Eq. 10),
 *               theta = (2 tau_T - 1)/4 (Eq. 14); both must exceed 1/2.
 *  g_beta       gravity times thermal expansion (Eq. 17); g_dir its unit
 *               direction (upright eye (-1, 0), supine (0, -1)).
 *  T_cold, T_hot, T_in  cornea, iris/lens and inflow temperatures;
 *  T0           reference temperature of the Boussinesq term (Eq. 5).
 *  u_in_max     peak inflow speed of the inlet profile.
 *  K_tm         TM permeability in cells^2 (> 0); porosity is carried for
 *               reporting only (Tab. 5 labels).
 *  p_out        outlet pressure (Schlemm's canal).
 *  drive        uniform body force (test flows; 0 for the eye).
 *  noise_amp, seed  amplitude and seed of the initial temperature noise.
 *  dx_m, dt_s, rho0, p_sc_pa  unit conversion for the *_pa outputs:
 *               IOP_pa = p_sc_pa + rho0 (dx/dt)^2 (iop - p_out).
 *  tm_model     0: the trabecular meshwork is resolved as porous cells with
 *               Darcy drag (Eq. 4) and the outlets hold p_out;
 *               1: the paper's lumped meshwork (Sec. 2.3): no drag in the TM
 *               cells, and the outlets impose the seepage velocity
 *               u_s = K_tm (IOP - p_out) / (nu h_tm) (Darcy's law across a
 *               meshwork of thickness h_tm with a linear pressure profile),
 *               re-evaluated from the IOP after every steady-state check.
 *  h_tm         effective meshwork thickness in cells (tm_model 1; > 0).
 *  bouzidi      0: halfway bounce-back on every no-slip wall; 1: Bouzidi's
 *               linear interpolated bounce-back (the no-slip scheme the paper
 *               names, Sec. 2.3 ref. 36) on the links from fluid cells to the
 *               curved cornea of the analytic eye, with the wall at the exact
 *               fraction q of each link where it crosses the cornea circle:
 *               q < 1/2: f_o(x) = 2q f*_i(x) + (1 - 2q) f*_i(x - e_i);
 *               q > 1/2: f_o(x) = f*_i(x)/(2q) + (2q - 1)/(2q) f*_o(x)
 *               (halfway where x - e_i is not active).  No effect on MASK
 *               geometries.  The q < 1/2 rule is applied when the cell next
 *               reads its populations, so switching it mid-run moves the
 *               switch by one step on those links. */
typedef struct lbm_params {
    double tau, tau_T;
    double g_beta;
    double g_dir[2];
    double T_cold, T_hot, T0, T_in;
    double u_in_max;
    double K_tm, porosity;
    double p_out;
    double drive[2];
    double noise_amp;
    uint64_t seed;
    double dx_m, dt_s, rho0, p_sc_pa;
    int32_t tm_model;
    int32_t bouzidi;
    double h_tm;
} lbm_params;

/* Observables of the state at time `step` (pre-collision populations).
 * q_in / q_out are the boundary fluxes of the step step -> step+1. */
typedef struct lbm_observables {
    int64_t step;
    double iop, iop_pa;           /* mean pressure over fluid cells */
    double q_in, q_out;           /* inflow / outflow per step */
    double mass;                  /* sum of f_1..f_8 over active cells */
    double peak_speed;            /* max |u| over active cells */
    double wss_cornea, wss_iris;  /* mean wall shear stress, lattice units */
    double wss_cornea_pa, wss_iris_pa;
    double residual;              /* max |u - u_snapshot|, -1 without snapshot */
    int64_t n_fluid, n_cornea, n_iris;
    int32_t nan_flag;             /* non-zero if any pressure was NaN */
    int32_t reserved;
    double u_seep;                /* seepage speed at the outlets during the
                                     observed step (tm_model 1, else 0) */
} lbm_observables;

/* Launch shape of the fused step kernel: tiles of tile_w x (block_rows *
 * rows_per_thread) cells, one thread per column (FP64) or column pair (other
 * storages) and row group.  tile_w in {32, 64, 128, 256}, tile_w * block_rows
 * <= 256, tile area >= 128 cells.  The 16-bit storages with tile_w 256 or
 * 128 take eight or four columns per thread instead (32 threads per row,
 * block_rows <= 8): rows whose cells are all away from boundaries then move
 * each population plane as one 16- or 8-byte vector.  Plain steps of the
 * 16-bit storages, and of FP32 grids with many cells in row segments next
 * to a boundary, update those cells in separate blocks, one per thread
 * (lbm_get_edge_cell_count); tiles 256 x 4 measured fastest for the 16-bit
 * storages, 64 x 4 for FP32.
 *
 * stepping selects how lbm_step advances a domain (the zero default is one
 * launch per step; the dataflow launch is faster where the per-step launch
 * overhead is a large share of a step, e.g. 0.81 against 0.74 of HBM on a
 * 4096 x 2048 eye, and slower on much smaller or much larger grids):
 *   LBM_STEP_FLOW: one cooperative launch covers all the steps of the call.  No
 *     grid-wide barrier separates them: a tile starts step s as soon as it
 *     and its eight neighbour tiles have finished step s - 1 (each link
 *     reaches one cell).  The grid is the co-resident block count (capped at
 *     blocks_per_sm per SM when blocks_per_sm > 0).  The steps are issued in
 *     sweeps of sweep_steps steps (0 or 1: one step at a time, at most 8): a
 *     wavefront over the tile rows with step k + 1 of the sweep sweep_lag
 *     tile rows behind step k (0: 8 rows; otherwise at least 2).  Step k + 1
 *     then reads what step k wrote while it is still in L2.  Grids periodic
 *     in y sweep one step at a time.  Falls back to LBM_STEP_PER_LAUNCH on a
 *     device without cooperative launches.
 *   LBM_STEP_PER_LAUNCH: one launch per step, replayed from a CUDA graph of
 *     32 steps; blocks_per_sm > 0 selects a grid of that many blocks per SM,
 *     0 one block per tile.  With FP32 arithmetic, shapes with block_rows 1
 *     and tile_w >= 64 take a persistent kernel (grid capped at the blocks
 *     the device holds at once) whose warps stage population rows in shared
 *     memory by bulk tensor copies; its interior collision rounds differently
 *     in the last bit.  A domain of at least 4096 tiles launches the tiles
 *     that hold boundary cells first (the slower ones), which shortens the
 *     tail of each step; the results do not depend on the order.
 * The dataflow kernel (any sweep) and the per-step direct kernel give
 * bit-identical populations.  Observing steps and batches always take one
 * launch per step. */
enum { LBM_STEP_PER_LAUNCH = 0, LBM_STEP_FLOW = 1 };

typedef struct lbm_launch {
    int32_t tile_w, block_rows, rows_per_thread, blocks_per_sm;
    int32_t stepping;    /* LBM_STEP_PER_LAUNCH (0) or LBM_STEP_FLOW */
    int32_t sweep_steps; /* LBM_STEP_FLOW: steps per wavefront sweep, 0..8 */
    int32_t sweep_lag;   /* LBM_STEP_FLOW: tile rows between a sweep's steps */
} lbm_launch;

typedef struct lbm_domain lbm_domain;
typedef struct lbm_batch lbm_batch;

/* ---- geometry (host only; no GPU needed) ---------------------------------*/

/* Build the cell-type mask of a geometry into host_out (ny*nx bytes) and
 * summarise it in *info (either may be NULL).  The analytic eye: solid outer
 * ring; iris/lens band y < band_cells between the two chamber-angle points;
 * ciliary inlet = the band's top row over a centred gap; cornea = circular arc
 * over the chord y = band - 1/2 whose sagitta a tan(angle/2) sets the chamber
 * angle (Tab. 1, Sec. 3.5); a porous TM block at each angle point with a
 * one-cell outlet column behind it.  EINVAL if the geometry does not fit. */
lbm_status lbm_build_mask(const lbm_geometry_desc* desc, uint8_t* host_out,
                          lbm_geometry_info* info);

/* ---- one problem ---------------------------------------------------------*/

/* Bytes of device memory a domain needs (0 if desc is invalid). */
size_t lbm_domain_bytes(const lbm_geometry_desc* desc, int32_t precision);

/* Create a domain inside dev_buf (>= lbm_domain_bytes, 256-byte aligned,
 * caller-owned, must outlive the domain).  Builds and uploads the mask on
 * `stream`.  The state is initialised by the first lbm_set_params. */
lbm_status lbm_create_domain(const lbm_geometry_desc* desc, int32_t precision,
                             void* dev_buf, size_t bytes, void* stream,
                             lbm_domain** out);

/* Validate and install parameters (Tab. 2 quantities in lattice units).
 * EINVAL if tau or tau_T <= 1/2, K_tm <= 0, |g_dir| not 1 while g_beta != 0,
 * or any value is not finite.  The first call also resets the state. */
lbm_status lbm_set_params(lbm_domain* dom, const lbm_params* params);

/* Reset to t = 0: f_i = f_i^eq(p_out, u = 0) (Eq. 7) and T_i = (T0 + n)/4 in
 * active cells, n = noise_amp (2 U - 1) with U the top 53 bits of
 * SplitMix64(seed XOR cell index) / 2^53.  Drops the velocity snapshot. */
lbm_status lbm_reset_state(lbm_domain* dom);

/* Advance nsteps >= 0 time steps (Eq. 6 and Eq. 11 with all boundary rules),
 * asynchronously on the domain's stream. */
lbm_status lbm_step(lbm_domain* dom, int64_t nsteps);

/* Step until the largest change of |u| over check_every steps falls below tol
 * (the steady criterion max |du| < tol per check_every steps), or max_steps
 * have been taken.  *steps_out (may be NULL) receives the steps taken.
 * Returns ENOTCONVERGED at the cap and EUNSTABLE on a NaN.  The host reads
 * each check's observables from pinned memory while the next interval
 * already runs (except with the lumped meshwork, tm_model 1, whose seepage
 * speed needs each check before the next interval), so the loop may stop one
 * interval after the check that met the criterion; *steps_out includes it.
 * Returns with the stream synchronised.  Allocates a small pinned host
 * buffer on first use.  The last check's observables are then available from
 * lbm_last_observables. */
lbm_status lbm_run_to_steady(lbm_domain* dom, double tol, int32_t check_every,
                             int64_t max_steps, int64_t* steps_out);

/* Reduce the observables of the current state (FP64 accumulation) and copy
 * them to *out; synchronises the stream. */
lbm_status lbm_read_observables(lbm_domain* dom, lbm_observables* out);

/* Write the macroscopic fields of the current state to caller device buffers
 * (any may be NULL): dev_u = 2*nx*ny doubles (u_x plane then u_y), dev_p and
 * dev_T = nx*ny doubles each (Eq. 9, Eq. 13); zero outside active cells. */
lbm_status lbm_read_field(lbm_domain* dom, double* dev_u, double* dev_p, double* dev_T);

/* Copy the populations of the current state, in natural order, to caller
 * device buffers: dev_f = 9*nx*ny doubles (plane i holds f_i), dev_g = 4*nx*ny
 * doubles (T_1..T_4); zero outside active cells. */
lbm_status lbm_read_populations(lbm_domain* dom, double* dev_f, double* dev_g);

/* Overwrite the populations of active cells from caller device buffers laid
 * out as in lbm_read_populations (rounded to the storage precision). */
lbm_status lbm_write_populations(lbm_domain* dom, const double* dev_f, const double* dev_g);

/* Checkpoint: lbm_state_bytes host bytes hold the raw stored populations, the
 * step counter and the parameters; save synchronises the stream. */
size_t lbm_state_bytes(const lbm_domain* dom);
lbm_status lbm_save_state(lbm_domain* dom, void* host_buf, size_t bytes);
lbm_status lbm_load_state(lbm_domain* dom, const void* host_buf, size_t bytes);

/* Launch shape of this domain's kernels (see lbm_launch). */
lbm_status lbm_set_launch(lbm_domain* dom, const lbm_launch* launch);
lbm_status lbm_get_launch(const lbm_domain* dom, lbm_launch* launch);

/* Test hook of the dataflow stepping's failure path (the paper has no
 * counterpart): while tile >= 0, this domain's dataflow launches never report
 * that tile's progress, so every wait on it runs out of its bounded polls
 * (about a second), the launch aborts its other waits and completes, and the
 * next observable read returns LBM_ECUDA ("results are invalid").  The GPU
 * context stays usable.  -1 turns it off.  EINVAL for a tile out of range. */
lbm_status lbm_debug_stall_tile(lbm_domain* dom, int32_t tile);

/* Time step counter, geometry summary, number of tiles of the launch shape. */
int64_t lbm_get_step(const lbm_domain* dom);
lbm_status lbm_get_info(const lbm_domain* dom, lbm_geometry_info* info);
int64_t lbm_get_tile_count(const lbm_domain* dom);

/* Edge cells of the domain's plain steps at its launch shape: the active
 * cells that no interior cell pair of the pair or vector path covers, which
 * separate blocks update one per thread (the 16-bit storages always; FP32
 * grids when more than 8 % of their active cells lie in 64-cell row segments
 * next to a boundary).  0 when the rows update every cell themselves (FP64,
 * other FP32 grids, tiles 32 wide, odd grid widths); -1 for a null domain. */
int64_t lbm_get_edge_cell_count(const lbm_domain* dom);

/* Bytes of algorithmic HBM traffic of one step of this domain: 2 x 13
 * populations per active cell at the storage precision plus one mask byte per
 * tiled cell. */
double lbm_step_bytes(const lbm_domain* dom);

void lbm_destroy_domain(lbm_domain* dom);

/* ---- vortex measures (Eq. 18, Tab. 3) -------------------------------------
 * Vortex intensity I = 2 * integral over the chamber of the vorticity
 * omega_z = (1/2)(du_y/dx - du_x/dy), taken over the fluid cells (cell area
 * 1 in lattice units), and the vortex centres, read as the extrema of the
 * stream function psi (u_x = dpsi/dy).  The signed integral over a closed
 * no-slip chamber is a boundary circulation and nearly vanishes (Stokes'
 * theorem), so the integral of |omega_z| is returned beside it; Tab. 3's
 * growth of I with the temperature difference fits the latter.
 * Derivatives: centred differences of the axis neighbours; a neighbour that
 * is not fluid or porous contributes the no-slip value 0 at half a link.
 * psi: the midpoint sum of u_x up each column from y = 0.  Extrema ties go to
 * the lowest flat index y*nx + x. */
typedef struct lbm_vortex_info {
    double intensity;           /* sum of 2 omega_z over fluid cells, lattice units */
    double intensity_abs;       /* sum of 2 |omega_z| */
    double intensity_phys;      /* intensity x dx^2/dt in m^2/s (0 without dx_m, dt_s) */
    double intensity_abs_phys;
    double psi_max, psi_min;    /* stream-function extrema over fluid cells, lattice units */
    int32_t max_x, max_y;       /* cell of psi_max (-1 without fluid cells) */
    int32_t min_x, min_y;       /* cell of psi_min */
    double max_mm[2], min_mm[2];/* those cell centres in mm, ((x + 1/2) dx, (y + 1/2) dx) */
    int64_t n_fluid;
} lbm_vortex_info;

/* Vortex measures of the device velocity field dev_u (FP64, 2 x ny x nx: u_x
 * then u_y, the layout lbm_read_field writes; values at non-active cells are
 * ignored) on this domain's grid and mask.  Uses the domain's partials region
 * as scratch and synchronises the domain's stream.  EINVAL for a null
 * argument or a one-row grid of at most 32 cells (too small a partials
 * region). */
lbm_status lbm_vortex(lbm_domain* dom, const double* dev_u, lbm_vortex_info* out);

/* ---- batches: many problems, fused launches ---------------------------------
 * A batch advances many domains of one storage precision, of any sizes and
 * parameters, over the concatenated tile lists of its members: with dataflow
 * stepping one cooperative launch for all steps of a call, else a single
 * launch of the fused step per time step (and, for 32 or more steps, replays
 * of a CUDA graph of those launches).  Each member keeps its own state,
 * parameters and step counter; a member's results do not depend on which
 * other domains share the batch: populations are bit-identical to stepping it
 * alone with the same launch shape, and its observables are folded from its
 * own tiles in a fixed order.  While a domain belongs to a batch its work
 * runs on the batch's stream.  Device memory of the batch (member table,
 * tile list, neighbour lists, progress words, observables) belongs to the
 * caller: lbm_batch_bytes. */

/* Bytes for a batch of up to max_instances members holding max_tiles tiles
 * in total (sum of lbm_get_tile_count of the members at the batch's shape).
 * The per-step list also holds the members' edge-cell chunks (blocks that
 * update the cells next to a boundary, one per thread), up to max_tiles of
 * them.  Tiles beyond max_tiles make lbm_batch_add fail, chunks beyond it
 * the batch's next step, both with LBM_EBUSY. */
size_t lbm_batch_bytes(int32_t max_instances, int64_t max_tiles);

/* Create an empty batch.  launch (may be NULL) is the shape every member is
 * switched to when it joins. */
lbm_status lbm_batch_create(int32_t precision, int32_t max_instances, int64_t max_tiles,
                            const lbm_launch* launch, void* dev_buf, size_t bytes,
                            void* stream, lbm_batch** out);

/* Add a domain (same precision, parameters set) / remove it.  EBUSY when the
 * batch is full or its tile capacity would be exceeded.  Adding synchronises
 * the domain's own stream; removing synchronises the batch's stream and gives
 * the domain its own stream back. */
lbm_status lbm_batch_add(lbm_batch* b, lbm_domain* dom);
lbm_status lbm_batch_remove(lbm_batch* b, lbm_domain* dom);
int32_t lbm_batch_size(const lbm_batch* b);

/* Advance every member nsteps time steps (Eqs. 6 and 11 with all boundary
 * rules), asynchronously on the batch's stream: with the batch shape's
 * stepping LBM_STEP_FLOW one dataflow launch over all members (step by step;
 * sweep_steps is ignored), else one launch per step. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* One check interval of the steady-state loop for every member:
 * check_every - 1 plain steps, then one step with the fused FP64 observables
 * and residual against each member's previous snapshot (-1 on a member's
 * first check).  Synchronises the batch's stream; each member's observables
 * are then available from lbm_last_observables. */
lbm_status lbm_batch_check(lbm_batch* b, int32_t check_every);

/* Observables of the domain's last steady-state check: the last check
 * interval that lbm_run_to_steady processed (including an interval queued
 * ahead that ran after the converging check) or the last lbm_batch_check.
 * `step` is the step count of the observed state; the sums are the check
 * step's (FP32 partials per warp for the FP32-arithmetic storages, folded in
 * FP64).  A host copy: no device work.  EINVAL if no check has run. */
lbm_status lbm_last_observables(const lbm_domain* dom, lbm_observables* out);

/* Launch shape of the batch (switches every member). */
lbm_status lbm_batch_set_launch(lbm_batch* b, const lbm_launch* launch);
lbm_status lbm_batch_get_launch(const lbm_batch* b, lbm_launch* launch);

/* Autotuner: time a fixed set of candidate shapes (tile width, rows per
 * thread, persistent grids, stepping; the 16-bit storages add eight-cell
 * shapes) for steps_per_candidate steps each on the current members, keep the
 * fastest and report it in *chosen (may be NULL).  One-launch-per-step shapes
 * are timed twice: with the merged tile list in member order, and with the
 * tiles that hold boundary cells first; the faster order is kept with the
 * shape.  The timed steps are real steps of the members. */
lbm_status lbm_batch_tune(lbm_batch* b, int32_t steps_per_candidate, lbm_launch* chosen);

/* Algorithmic bytes of one batch step (sum of lbm_step_bytes of the members)
 * and the number of active cells updated per step. */
double lbm_batch_step_bytes(const lbm_batch* b);
int64_t lbm_batch_active_cells(const lbm_batch* b);

/* Destroy the batch (members become stand-alone domains again). */
void lbm_batch_destroy(lbm_batch* b);

/* ---- observables without caller-provided reduction scratch ----------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * may not allocate device memory once they are running, for instance a host
 * application that hands the library a fixed device budget at start-up, or a
 * latency-critical loop in which an allocation would stall the device.  It
 * returns the same observables as lbm_read_observables (FP64 sums, folded in
 * a different fixed order), but keeps its per-row partial sums in a device
 * array inside the library instead of the domain buffer: LBM_NOALLOC_MAX_ROWS
 * rows x 12 doubles (about 0.8 MB), held by every GPU that loads the library
 * until the process exits.  The first call on a device looks up that array's
 * device address with the device current; make that first call before any
 * stream capture.  The device current at the call must be the one that was
 * current when the domain was created, else the call returns LBM_EINVAL.  A
 * batch member may be read: while it belongs to a batch its work runs on the
 * batch's stream, so the read follows the batch's steps.  A grid with more
 * than LBM_NOALLOC_MAX_ROWS rows is rejected with LBM_EINVAL.  All calls on one device share the array and it
 * keeps the last call's contents: calls that overlap on the GPU (for example
 * on two streams with no ordering between them) race on it, calls on one
 * stream do not.  Synchronises the domain's stream. */
#define LBM_NOALLOC_MAX_ROWS 8192
lbm_status lbm_read_observables_noalloc(lbm_domain* dom, lbm_observables* out);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
