/*
 * batch.h -- many simulations advanced together (libfdtd_gb300.so).
 *
 * A batch borrows n simulation handles (fdtd.h) on one device, each with its
 * own grid, boundary, shower (Sec. III.B) and detectors, and advances all of
 * them with one persistent kernel per launch: every step of Sec. III.A of a
 * simulation is a set of work items on a shared queue -- (simulation, tile
 * of 128 columns x 8 rows, z chunk) items, each the one-pass H and E update
 * of that tile with the shower's current, then pieces of the Mur faces and
 * the detector readout -- and an item waits only for the items of its own
 * simulation it depends on (per-simulation completion counts, no grid-wide
 * barrier inside a launch); every wait is bounded (FDTD_ERR_TIMEOUT if one
 * gives up).  The kernel is a cooperative launch of one block per SM; the
 * launch, with the reset of its counters, is captured once in a CUDA graph
 * and replayed.  A tile is
 * updated by the same code as the handle's one-pass tile path
 * (fdtd_set_kernel 1), and the faces and detectors by that of its own Mur and
 * readout kernels, so a batched step gives the numbers of fdtd_step on the
 * handle with path 1 selected, bit for bit.
 * The persistent kernel takes PEC and Mur grids.  Simulations large enough
 * to keep the GPU busy with their own kernels can instead step alone
 * (fdtd_batch_set_solo), as does a grid with CPML layers or one the tile path
 * cannot run: after the persistent launches, their handle's
 * selected path is issued on eight internal streams (largest grid first, each
 * to the least loaded stream), so several run at once and each gets exactly
 * what fdtd_step on the handle gives.
 *
 * The handles stay owned by the caller and must outlive the batch; stepping
 * a handle on its own between batch steps is allowed (the batch re-reads the
 * handle's step count and field set before each launch).  Status codes as in
 * fdtd.h; errors are sticky per batch.
 */
#ifndef BATCH_GB300_H
#define BATCH_GB300_H

#include "fdtd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_batch *fdtd_batch_t;

/* n >= 1 distinct handles on the current device; the batch works on its own stream. */
int fdtd_batch_create(fdtd_batch_t *out, const fdtd_t *sims, int n);
void fdtd_batch_destroy(fdtd_batch_t b);

/*
 * Advance every simulation n >= 0 steps (asynchronous with respect to the
 * host; ordered after earlier work on the handles' streams and before later
 * work on them).  FDTD_ERR_CAPACITY if a simulation's trace would overflow.
 */
int fdtd_batch_step(fdtd_batch_t b, int n);

/*
 * Synchronise (the solo streams included) and return the sticky status of
 * the batch.  A bounded wait that gives up inside a simulation stepping
 * alone is recorded on that handle, as for fdtd_step: fdtd_sync on the
 * handle reports it.
 */
int fdtd_batch_sync(fdtd_batch_t b);

/*
 * Launch configuration: z planes per chunk of a tile item (>= 1; the planes
 * between a CPML grid's z layers are cut into chunks of about this many, the
 * layers are chunks of their own; fewer planes per chunk where a long chunk's
 * coefficient table would crowd out the stage ring; default 256), steps per
 * persistent launch (1 .. 64; default 8).
 */
int fdtd_batch_set_config(fdtd_batch_t b, int chunk_planes, int steps_per_launch);
int fdtd_batch_get_config(fdtd_batch_t b, int *chunk_planes, int *steps_per_launch);

/*
 * Autotuner: first the solo threshold (none, every simulation alone, or a
 * power of two between the smallest and the largest grid), then the chunk
 * length of the persistent kernel's tile items (64 .. 512 planes).  It runs
 * trial_steps >= 1 steps of the batch itself with each candidate, times each
 * on the device, keeps the fastest and returns the steps it used in
 * *steps_used.  The trial steps are real steps of every simulation (a
 * candidate decides which code path steps a simulation, never what that
 * path computes).
 */
int fdtd_batch_tune(fdtd_batch_t b, int trial_steps, int *steps_used);

/*
 * Simulations of at least min_cells cells step alone, with their handle's
 * selected path, on the batch's internal streams; the rest share the
 * persistent kernel, CPML grids excepted (they always step alone).
 * min_cells = -1 (the default): every PEC and Mur grid shares it.
 * FDTD_ERR_ARG for min_cells < -1.  fdtd_batch_get_solo returns the
 * threshold and the number of simulations that step alone (either pointer
 * may be null).
 */
int fdtd_batch_set_solo(fdtd_batch_t b, long long min_cells);
int fdtd_batch_get_solo(fdtd_batch_t b, long long *min_cells, int *n_solo);

/*
 * Bound of every wait of the persistent kernel (for the items an item
 * depends on, and the grid barrier that ends a launch), in SM clock cycles
 * (0: the default, FDTD_BATCH_DEFAULT_WAIT_CYCLES, about two seconds).
 * A wait that runs out records the failure on the device and the kernel
 * returns; fdtd_batch_sync then reports FDTD_ERR_TIMEOUT for the batch and
 * for every simulation that shared the persistent kernel (left part-way
 * through a step, so its handle cannot be stepped again: the status is
 * sticky), and later persistent launches of the batch return at once.  A
 * small limit makes a wait give up while the items it waits for are still at
 * work, which is how the timeout path is tested.  FDTD_ERR_ARG for
 * cycles < 0.
 */
#define FDTD_BATCH_DEFAULT_WAIT_CYCLES (4LL << 30)
int fdtd_batch_set_wait_limit(fdtd_batch_t b, long long cycles);

/* Whether launches are replayed from a captured graph (1) or issued directly (0). */
int fdtd_batch_graph_mode(fdtd_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* BATCH_GB300_H */
