/*
 * cyl.h -- C ABI of the paper's 2D axisymmetric FDTD (libfdtd_gb300.so).
 *
 * Sec. III.A of the paper: with cylindrical symmetry about the shower axis
 * the phi derivatives vanish, H_r, H_z and E_phi vanish, and Maxwell's
 * equations reduce to Eqs. fdtd_Er, fdtd_Ez, fdtd_Hphi for (E_r, E_z, H_phi)
 * on an (r, z) grid.  This is the formulation the paper runs on its GPU
 * (Sec. IV, Table I); the 3D Cartesian path of fdtd.h is the main path.
 *
 * Grid: nr x nz cells of size d; nodes r = i d (i = 0..nr), z = j d (j =
 * 0..nz).  E_r sits at (i+1/2, j), E_z at (i, j+1/2), H_phi at (i+1/2, j+1/2).
 * One step: H_phi^{n+1/2} from E^n, then E^{n+1} from H_phi^{n+1/2} and the
 * current J_z^{n+1/2}, then the boundary, then the detectors.  On the axis
 * E_z takes Ampere's law over the disc of radius d/2: dE_z/dt = 4 H_phi(1/2)
 * / (eps d) - J_z / eps.  The outer wall (r = nr d) and the end caps (z = 0,
 * z = nz d) are PEC, or first-order Mur on their tangential E.
 *
 * Source (same reading as the 3D path): the shower's charge q(z_s), z_s =
 * z0 + v t, linear in a bin table, spread over rings with weights w_i (ring i
 * covers r in [(i-1/2) d, (i+1/2) d], the axis disc [0, d/2]), moving as a
 * cloud-in-cell line; J_z through face (i, j+1/2) is the charge that crossed
 * it per unit area and time.
 *
 * Status codes, ownership and threading as in fdtd.h (FDTD_OK, FDTD_ERR_*):
 * the library owns its device buffers, host inputs are copied, the stream is
 * borrowed, errors are sticky and returned by the next call.
 */
#ifndef CYL_GB300_H
#define CYL_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cyl_ctx *cyl_t;

/*
 * 4 <= nr <= 65534 and nz >= 4 cells of size d (metres), dt seconds, relative permittivity
 * eps_r, boundary FDTD_PEC (0) or FDTD_MUR1 (1).  dt above the 2D Courant
 * limit d sqrt(eps_r) / (c sqrt 2) returns FDTD_ERR_CFL.
 */
int cyl_create(cyl_t *out, int nr, int nz, double d, double dt, double eps_r, int boundary, void *stream);
void cyl_destroy(cyl_t h);

/*
 * Shower: q (host, n_bins doubles, coulombs) at z0 + b bin_dz, linear in
 * between and zero outside; speed v (m/s) along z with |v| dt <= 4 d; ring
 * weights w (host, nw doubles, nw <= nr+1; ring nr lies on the wall, whose
 * E_z the boundary sets).  Replaces any previous shower.
 */
int cyl_set_shower(cyl_t h, const double *q, int n_bins, double z0, double bin_dz, double v, const double *w,
                   int nw);

/*
 * Ring weights of the paper's radial Gaussian spread (Sec. III.B, lateral
 * charge density exp(-r^2 / (2 sigma_r^2)), sigma_r = 5 cm in the paper):
 * w[i] (host, n_rings doubles) is the share of the charge in ring i, which
 * covers r in [(i-1/2) d, (i+1/2) d] (the axis disc [0, d/2] for i = 0),
 * renormalised to sum 1 over the n_rings rings.  The longitudinal table of
 * the same model (Eq. showerModel) comes from fdtd_profile_gaussian (fdtd.h).
 * FDTD_ERR_ARG for a null pointer, n_rings < 1, d <= 0 or sigma_r <= 0.
 */
int cyl_rings_gaussian(int n_rings, double d, double sigma_r, double *w);

/*
 * Detectors at (r, z) metres (host, n*2 doubles), snapped to the nearest
 * node, 0 <= i < nr and 0 < j < nz (FDTD_ERR_ARG otherwise); trace slot s
 * holds (E_z, E_r) at step s+1 (E_z averaged over j +- 1/2, E_r over i +- 1/2,
 * E_r = 0 on the axis), for s < max_steps (FDTD_ERR_CAPACITY beyond).
 */
int cyl_set_probes(cyl_t h, const double *rz, int n, int max_steps);

/*
 * Advance n >= 0 steps asynchronously on the handle's stream.  The
 * wavefront kernels advance K steps per launch; the n mod K steps left over
 * run on the two-kernel path.  FDTD_ERR_CAPACITY if detectors are set and
 * the trace would overflow.
 */
int cyl_step(cyl_t h, int n);

/*
 * Kernel for the following steps: 0 = two kernels per step (H, then E with
 * the boundary; 36 bytes of DRAM per cell-update); 1..5 = one wavefront
 * launch per K steps (24 bytes per cell per launch): 1 = K 4 with 2 z columns
 * per lane, 2 = K 8 with 2, 3 = K 4 with 4, 4 = K 4 with 4 and registers
 * bounded for 4 blocks per SM, 5 = K 8 with 2 bounded the same way.
 * seg_rows = radial rows per warp segment (at most 1024), 0 picks it from the
 * grid and the SM count.  FDTD_ERR_ARG for another index.  The default
 * depends on the grid: 0 below 400000 cells (its steps are replayed from
 * captured graphs of 32 steps), 1 below 1600000 cells, 3 above.
 */
int cyl_set_kernel(cyl_t h, int which, int seg_rows);

/*
 * Autotuner of the wavefront kernel in use: it advances the simulation with
 * each candidate segment length (12 rows and up, in steps of 4 to 64, 8 to
 * 128 and 16 beyond, until the tiles fit one wave of the resident blocks; at
 * most 48 candidates), `launches` (1..8) launches each, times every launch
 * on the device and keeps the length of the fastest launch (cyl_kernel_info
 * reports it).  The steps are real steps of the simulation, recorded by the
 * detectors; the segment length decides how the work is cut, never what is
 * computed, so the fields and traces are those of any other length.  Returns
 * the steps it used in *steps_used (may be null): at most 48 x launches x K.
 * Nothing to do (0 steps) on the two-kernel path.  FDTD_ERR_CAPACITY, before
 * any step, if detectors are set and their trace has no room for those
 * steps; FDTD_ERR_ARG for launches outside 1..8.
 */
int cyl_tune(cyl_t h, int launches, int *steps_used);

/* The kernel in use, its steps per launch and rows per segment (any pointer may be null). */
int cyl_kernel_info(cyl_t h, int *which, int *steps_per_launch, int *seg_rows);

/* Name of the kernel in use (static string; "none" for a null handle). */
const char *cyl_kernel_name(cyl_t h);

/* Steps done since creation or the last reset. */
int cyl_steps_done(cyl_t h, int64_t *steps);

/* Synchronise and return the sticky status (FDTD_ERR_TIMEOUT if a bounded wait of a kernel gave up). */
int cyl_sync(cyl_t h);

/* Traces [n][max_steps][2] float32 to a host (on_device = 0) or device pointer.  Synchronises. */
int cyl_probes(cyl_t h, float *out, int on_device);

/*
 * One component, float32, compact: comp 0 = E_r [nr][nz+1], 1 = E_z
 * [nr+1][nz], 2 = H_phi [nr][nz] (z fastest).  cyl_fields reads, cyl_set_field
 * writes (host or device pointer).  Synchronise.
 */
int cyl_fields(cyl_t h, int comp, float *out, int on_device);
int cyl_set_field(cyl_t h, int comp, const float *in, int on_device);

/* Zero the fields and traces, keep shower and detectors; steps = 0. */
int cyl_reset(cyl_t h);

/* Kernel launches so far (timing-independent bookkeeping). */
int cyl_launch_count(cyl_t h, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* CYL_GB300_H */
