/*
 * fdtd.h -- C ABI of the GB300 near-field FDTD library (libfdtd_gb300.so).
 *
 * The library integrates Maxwell's curl equations (Sec. III.A of Hu, Chen &
 * Chen, "A GPU-based Calculation Method for Near Field Effects of Cherenkov
 * Radiation Induced by Ultra High Energy Cosmic Neutrinos") on a 3D Cartesian
 * Yee grid in a uniform lossless dielectric (ice: eps_r = 3.17), driven by the
 * current of the net charge excess of a particle shower moving along the z
 * axis (Sec. III.B, eq. showerModel and the snapshot charge density n(z,r)),
 * with an absorbing boundary, and records E(t) at detector points placed
 * around the shower (Sec. III.B, "Simulation Setup": all detectors in one run).
 *
 * Conventions
 *   - A grid of nx*ny*nz cells has nodes 0..n per axis; node (i,j,k) sits at
 *     (i dx, j dx, k dx) metres.  Yee positions:
 *       Ex(i+1/2,j,k)  Ey(i,j+1/2,k)  Ez(i,j,k+1/2)
 *       Hx(i,j+1/2,k+1/2)  Hy(i+1/2,j,k+1/2)  Hz(i+1/2,j+1/2,k).
 *   - Field snapshots use the node grid (nz+1, ny+1, nx+1), x fastest, float32;
 *     entry (i,j,k) holds the component at the position listed above.  Entries
 *     outside a component's range, and the H components normal to an outer
 *     face lying on that face (they drive no updated E), read as zero.
 *   - The shower axis is the node line (nx/2, ny/2) (integer division).
 *   - One step n -> n+1: H^{n+1/2} from E^n, then E^{n+1} from H^{n+1/2} and
 *     J^{n+1/2}, then the boundary, then the detectors read E^{n+1}.
 *     E^0 = 0 and H^{-1/2} = 0 after fdtd_create / fdtd_reset.
 *
 * Ownership: the library allocates and owns every device buffer it uses; host
 * inputs are copied during the call; output buffers belong to the caller.  The
 * CUDA stream passed to fdtd_create is borrowed, never destroyed.
 *
 * Errors: every int-returning call returns FDTD_OK (0) or a negative
 * FDTD_ERR_* code and never throws.  Argument errors are detected on the host
 * before any device work.  A CUDA error seen during asynchronous work is kept
 * in the handle and returned by the next call (sticky).
 *
 * Threading: a handle may be used from one host thread at a time.
 */
#ifndef FDTD_GB300_H
#define FDTD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_ctx *fdtd_t;

enum fdtd_boundary {
    FDTD_PEC = 0,  /* tangential E = 0 on the six outer faces */
    FDTD_MUR1 = 1, /* first-order Mur on the tangential E of each face (edges PEC) */
    FDTD_CPML = 2  /* Roden-Gedney CPML of npml cells backed by PEC */
};

enum fdtd_status {
    FDTD_OK = 0,
    FDTD_ERR_ARG = -1,      /* bad argument (null pointer, size, range, state) */
    FDTD_ERR_CFL = -2,      /* dt above the 3D Courant limit dx sqrt(eps_r)/(c sqrt 3) */
    FDTD_ERR_OOM = -3,      /* device allocation failed */
    FDTD_ERR_UNSTABLE = -4, /* a non-finite field value was found */
    FDTD_ERR_CUDA = -5,     /* a CUDA runtime call failed (no device, launch error, ...) */
    FDTD_ERR_TIMEOUT = -6,  /* a bounded device-side wait gave up */
    FDTD_ERR_CAPACITY = -7  /* stepping past the detector trace capacity */
};

/* Field component ids for fdtd_fields / fdtd_set_field. */
enum fdtd_component { FDTD_EX = 0, FDTD_EY, FDTD_EZ, FDTD_HX, FDTD_HY, FDTD_HZ };

/*
 * Create a simulation of nx*ny*nz cells (each >= 4) of size dx metres with time
 * step dt seconds in a medium of relative permittivity eps_r (mu_r = 1,
 * sigma = 0; Sec. III.A with sigma = 0).  boundary is an fdtd_boundary; npml is
 * the CPML depth in cells (>= 1, each n >= 2 npml + 4; ignored otherwise).
 * cuda_stream is a cudaStream_t (NULL: the legacy default stream).  dt must not
 * exceed the Courant limit (FDTD_ERR_CFL).  Fields start at zero.  On error
 * *out is set to NULL.
 */
int fdtd_create(fdtd_t *out, int nx, int ny, int nz, double dx, double dt, double eps_r,
                int boundary, int npml, void *cuda_stream);

/* Release every resource of the handle (NULL is allowed).  Synchronises the stream. */
void fdtd_destroy(fdtd_t h);

/*
 * The moving charge excess (Sec. III.B; Sec. I for the 20 % excess).  q_profile
 * (host, n_bins >= 2 doubles) holds the charge Q in coulombs at the sample
 * points z0 + b*bin_dz metres, b = 0..n_bins-1; Q(z) between samples is linear
 * and zero outside the table.  The charge moves along `axis` (only 2 = z is
 * supported) at speed v m/s and is at z0 at step 0: z_s^n = z0 + v n dt.
 * lateral_w (host, (2L+1)^2 doubles, row dj = -L..L, column di = -L..L) spreads
 * it over the nodes (nx/2 + di, ny/2 + dj); the footprint must lie inside the
 * non-PML interior with one node of margin.  Each step the charge
 * qbar = Q(z_s^{n+1/2}) is carried from z_s^n to z_s^{n+1} with linear (CIC)
 * weights along z, and the current on edge (i,j,k+1/2) is the charge crossing
 * it: J = -(dx/dt) qbar w_ij / dx^3 [C_k(z_s^{n+1}) - C_k(z_s^n)], C_k the
 * weight on nodes <= k of the untruncated line.  The current is applied on the
 * Ez edges outside the PML (all edges otherwise); a change of qbar between steps
 * is charge created or removed at rest.  Replaces any previous shower.
 */
int fdtd_set_shower(fdtd_t h, const double *q_profile, int n_bins, double z0, double bin_dz,
                    int axis, double v, const double *lateral_w, int L);

/* Remove the shower (no current). */
int fdtd_clear_shower(fdtd_t h);

/*
 * Detectors (Sec. III.B: fixed (theta, R) positions, recorded as time evolves).
 * xyz_m (host, n*3 doubles) are positions in metres, snapped to the nearest
 * node, which must lie inside the non-PML interior with one node of margin
 * (FDTD_ERR_ARG otherwise).  max_steps is the trace capacity: trace slot s
 * holds the reading of E^{s+1}, for s < max_steps; stepping beyond it returns
 * FDTD_ERR_CAPACITY.  Each reading is (Ez, E_r) at the node: Ex, Ey, Ez are
 * averaged over their two samples around the node and E_r = (X Ex + Y Ey)/r
 * about the shower axis (0 on the axis).  Traces restart at zero.
 */
int fdtd_set_probes(fdtd_t h, const double *xyz_m, int n, int max_steps);

/* Nodes the detectors were snapped to, n*3 ints (host). */
int fdtd_probe_nodes(fdtd_t h, int *ijk);

/* Advance n >= 0 steps, asynchronously on the handle's stream. */
int fdtd_step(fdtd_t h, int n);

/* Synchronise the stream and return the sticky status. */
int fdtd_sync(fdtd_t h);

/* Steps done since creation / the last reset. */
int fdtd_steps_done(fdtd_t h, int64_t *steps);

/*
 * Copy the traces, float32 [n_probes][max_steps][2] (Ez, E_r), to `out`: a host
 * pointer (on_device = 0) or a device pointer (on_device = 1).  Synchronises.
 */
int fdtd_probes(fdtd_t h, float *out, int on_device);

/* Snapshot of one component (fdtd_component) on the node grid (see top). Synchronises. */
int fdtd_fields(fdtd_t h, int comp, float *out, int on_device);

/* Overwrite one component from a node-grid array; entries outside the
   component's updated range are ignored (kept zero). Synchronises. */
int fdtd_set_field(fdtd_t h, int comp, const float *in, int on_device);

/* Zero fields, CPML memory and traces; keep shower and detectors; steps = 0.
   Clears a sticky FDTD_ERR_UNSTABLE (the non-finite values are gone); any
   other sticky error stays. */
int fdtd_reset(fdtd_t h);

/*
 * Field energy W = 1/2 eps sum |E|^2 dx^3 + 1/2 mu0 sum |H|^2 dx^3 (double,
 * computed on the device in FP64 over the updated entries), and a stability
 * check: returns FDTD_ERR_UNSTABLE (and still fills *energy) if any field value
 * is not finite.  Synchronises.
 */
int fdtd_energy(fdtd_t h, double *energy);

/*
 * The paper has no counterpart to this call: it is a diagnostic of the
 * scheme, the same energy and stability check as fdtd_energy, for six field
 * arrays that the caller owns on the device, with no handle and no device
 * memory allocated by the call.  It serves callers that cannot allocate: one
 * whose device memory is already taken by its own field arrays (a handle
 * would add two full field sets), or one that must not allocate while it runs
 * because an allocator or a memory budget outside this library owns the rest
 * of the device.
 *
 * d_fields: device pointer to Ex, Ey, Ez, Hx, Hy, Hz back to back, each
 *   (nz+1)(ny+1)(nx+1) float32 in the node layout of fdtd_fields (x fastest);
 *   entries a component does not use should be zero (as fdtd_fields writes).
 * nx, ny, nz >= 1 cells; dx > 0 metres; eps_r > 0.
 * nblocks: partial sums of the first pass, 1 .. FDTD_ENERGY_SCRATCH_BLOCKS,
 *   or 0 for four per SM (capped at that maximum); a larger value returns
 *   FDTD_ERR_CAPACITY.
 * stream: cudaStream_t to run on (NULL: the default stream); the call
 *   synchronises it.
 * energy: host out, W = 1/2 eps sum |E|^2 dx^3 + 1/2 mu0 sum |H|^2 dx^3.
 * Returns FDTD_ERR_UNSTABLE (energy still written) if a value is not finite,
 * FDTD_ERR_ARG on a null pointer or bad size, FDTD_ERR_CUDA on a CUDA error.
 *
 * Scratch: a fixed array of 3 FDTD_ENERGY_SCRATCH_BLOCKS + 3 doubles (24.6 KB)
 * compiled into the library.  Every slot a call reads is written earlier in
 * the same call, so nothing has to start at zero.  All calls on a device share
 * it: calls that overlap in time (other threads, other streams) race and must
 * be serialised by the caller.  The first call on a device (with that device
 * current) looks the array up (cudaGetSymbolAddress, which may load the
 * module); make that first call before any stream capture begins.  The
 * address is kept per device and context: after a device reset (a new primary
 * context) the next call looks it up again, so it also belongs before any
 * capture.
 */
#define FDTD_ENERGY_SCRATCH_BLOCKS 1024
int fdtd_energy_noalloc(const float *d_fields, int nx, int ny, int nz, double dx, double eps_r,
                        int nblocks, void *stream, double *energy);

/*
 * Checkpoint: the full state (fields, CPML memory, step counter, traces) as an
 * opaque host blob.  With buf == NULL, *bytes receives the size needed.
 * Loading into a handle created with the same grid, boundary and detectors
 * resumes bit-for-bit.
 */
int fdtd_save_state(fdtd_t h, void *buf, size_t *bytes);
int fdtd_load_state(fdtd_t h, const void *buf, size_t bytes);

/*
 * Instrumentation.  fdtd_timing_begin(h, max_launches) records a CUDA event pair
 * around each launch of the main field-update kernel(s) on the handle's stream;
 * fdtd_timing_end(h, &ms, &launches) synchronises and returns their summed
 * device time and count.  fdtd_launch_count returns the number of kernels the
 * handle has launched since creation.
 */
int fdtd_timing_begin(fdtd_t h, int max_launches);
int fdtd_timing_end(fdtd_t h, double *total_ms, int *launches);
int fdtd_launch_count(fdtd_t h, int64_t *launches);

/* Cell-updates of one launch of the timed kernel(s): the whole grid (the
   unfused path 0 times its H sweep and its E sweep as separate launches),
   twice the grid on path 2 (two steps per launch). */
int fdtd_timed_cells(fdtd_t h, int64_t *cells);

/* Name of the field-update path in use (static string). */
const char *fdtd_kernel_name(fdtd_t h);

/*
 * Select the field-update path (all compute the same update, Sec. III.A):
 *   2 = two steps per pass (temporal blocking of the leapfrog): each tile
 *       recomputes the first step on a two-cell halo, so a pass reads the
 *       fields once and writes them once for two steps; CPML and detectors
 *       included; a last odd step of fdtd_step runs on path 1.  PEC and CPML
 *       grids only (FDTD_ERR_ARG on a Mur grid); the default there from
 *       FDTD_TWO_STEP_MIN_CELLS cells, about 12.6 million (on smaller grids
 *       its blocks are too few to hide their start-up: measured 22 against
 *       28 Gcell/s for path 1 on 96 x 96 x 384, CPML 10, and 52.5 against
 *       50.7 on 128 x 128 x 512, where path 1 is faster with thousands of
 *       detectors in one tile; 69.5 against 52.2 on 160 x 160 x 640);
 *   1 = one pass per step: TMA-staged vector-tile z-march over the whole
 *       grid, CPML included (the default on Mur grids and smaller grids);
 *   0 = one H sweep then one E sweep (the reference path; the adjoint uses
 *       its per-cell code).
 * Returns FDTD_ERR_ARG for a path the handle cannot run.
 */
int fdtd_set_kernel(fdtd_t h, int which);

/*
 * Watchdog of the stepping path: every `every` steps (FDTD_WATCHDOG_DEFAULT_STEPS
 * after fdtd_create; 0 turns it off) a small kernel scans every field component
 * on every eighth z plane and the last one for non-finite values.  An unstable
 * run (Sec. III.A: the leapfrog is stable only below the Courant limit) or a
 * non-finite value anywhere in the grid spreads one plane per step, so it is
 * seen within every + 4 steps; the next fdtd_sync, fdtd_probes or other call
 * that synchronises then returns FDTD_ERR_UNSTABLE, and the status is sticky
 * (fdtd_reset clears it).  Cost: 1/8 of the field bytes every `every` steps
 * (0.1 % of a step at the default).  FDTD_ERR_ARG for every < 0.
 */
#define FDTD_WATCHDOG_DEFAULT_STEPS 64
#define FDTD_TWO_STEP_MIN_CELLS (3LL << 22)
int fdtd_set_watchdog(fdtd_t h, int every);

/* Human-readable text of a status code (static string). */
const char *fdtd_strerror(int status);

/* ---- adjoint ------------------------------------------------------------- */

/*
 * The step of Sec. III.A is linear in (E^n, H^{n-1/2}) and in the source; on
 * the Yee grid its curls satisfy C_H = C_E^T on the E cells the update
 * changes, so its transpose is the same leapfrog with (kE, kH) replaced by
 * (-kH, -kE) and no source; on a Mur grid the transpose of the face update
 * E'_b = E_1^n + m (E'_1 - E_b^n) is folded in (the face cells' adjoint
 * feeds their inward neighbours before the curls, and takes the transposed
 * curl of the new adjoint H after them); on a CPML grid the layer memory
 * psi' = b psi + a d of every difference d gets its adjoint, kept in the
 * handle's psi memory like the forward's.
 *
 * fdtd_adjoint_step applies n >= 0 transposed steps to the handle's fields
 * (asynchronous; the step counter is not changed; fields and CPML memory
 * hold the adjoint state).
 *
 * fdtd_adjoint_gradient returns dL/dq_b, the derivative of a loss of the
 * detector traces with respect to the shower's charge table (Sec. III.B),
 * for the first n_steps steps from zero fields.  dl_dtrace is a device
 * pointer laid out like the traces, float32 [n_probes][max_steps][2], holding
 * dL/d(trace) (slots >= n_steps are not read).  grad_q (n_bins doubles) is a
 * host (on_device = 0) or device pointer.  The adjoint state lives in the
 * handle's field memory: the call leaves the handle reset (fields zero, step
 * counter 0, CPML memory zero, traces kept).  Needs a shower, detectors,
 * 1 <= n_steps <= max_steps (FDTD_ERR_ARG otherwise).  Synchronises.
 */
int fdtd_adjoint_step(fdtd_t h, int n);
int fdtd_adjoint_gradient(fdtd_t h, const float *dl_dtrace, int n_steps, double *grad_q, int on_device);

/* ---- host-side shower tables (Sec. III.B) ------------------------------ */

/* Eq. showerModel: out[b] = q_max exp(-(z_b - z_peak)^2 / (2 l^2)), z_b = z0 + b bin_dz. */
int fdtd_profile_gaussian(double z0, double bin_dz, int n_bins, double z_peak, double l,
                          double q_max, double *out);

/* Eq. nkg_formula (Greisen profile) with the age s = 3t/(t + 2 ln(E0/Ec)):
   out[b] = -e frac N_e(t_b), t_b = b bin_dz / X0 (X0 in metres). */
int fdtd_profile_greisen(double bin_dz, int n_bins, double E0, double Ec, double X0,
                         double frac, double *out);

/* Sum of Gaisser-Hillas subshowers (an elongated multi-peak profile):
   out[b] = -e frac sum_s N_s(z_b), z_b = z0 + b bin_dz. */
int fdtd_profile_gaisser_hillas(double z0, double bin_dz, int n_bins, int n_sub,
                                const double *z1, const double *zmax, const double *lambda,
                                const double *nmax, double frac, double *out);

/* Lateral weights, (2L+1)^2, normalised to sum 1: a Gaussian of sigma cells, or
   the NKG density with Moliere radius r_m and age s averaged over nsub^2
   points per cell and cut at r_cut metres. */
int fdtd_lateral_gaussian(int L, double sigma_cells, double *w);
int fdtd_lateral_nkg(int L, double dx, double r_m, double s, int nsub, double r_cut, double *w);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_GB300_H */
