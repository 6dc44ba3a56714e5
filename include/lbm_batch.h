/*
 * lbm_batch.h - many independent D2Q37 lattices stepped together.
 *
 * A batch holds lattices of uneven sizes and parameters (each with its own
 * walls, tau, g and FP32 shift) that share one precision.  n steps of the
 * whole batch are captured once into a CUDA graph and replayed with one graph
 * launch.  Two ways to launch a step are candidates:
 *  - one kernel launch whose blocks walk a single work list of tiles spanning
 *    every lattice (each tile runs the fused propagate, bc and collide of
 *    Sect. 2 / eq. 1 on its lattice, with that lattice's constants staged in
 *    shared memory); nine tile shapes;
 *  - one launch of the single-lattice step kernel per lattice (its constants
 *    in the kernel parameters), the lattices spread over eight streams that
 *    the graph runs concurrently, each lattice's steps in order;
 *  - (LBM_FP32_SHIFTED batches whose lattices each hold fewer than 2^31
 *    elements) one kernel launch per group of up to 64 lattices whose blocks
 *    walk the group's tiles, with every lattice's constants in a table passed
 *    as the kernel's parameters (no shared-memory staging); three tile
 *    shapes.  For other batches these candidates run the shared-memory tile
 *    kernel of the same shape.
 * lbm_batch_autotune times every candidate on the batch itself and keeps the
 * fastest.  The paper has no batched mode; the per-lattice step is the one of
 * include/lbm.h (same readings, layout and population order).  The
 * candidates agree to rounding: each is its own compiled kernel, and float
 * multiply-add contraction may differ between them.
 *
 * OWNERSHIP.  The caller owns every lattice buffer (two per lattice, in the
 * state layout of include/lbm.h) and the stream.  The batch allocates its
 * own device tables (lattice parameters, tile offsets, and for every tile
 * shape the lattice of each tile: 4 bytes per tile, about 1 MB per shape for
 * 33 M sites), eight streams for the per-lattice launches, and its CUDA
 * graphs; lbm_batch_destroy releases them.
 *
 * ERRORS.  As in include/lbm.h: LBM_OK or a negative LBM_ERR_* code, with a
 * message from lbm_batch_last_error().
 */
#ifndef LBM_BATCH_H
#define LBM_BATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_lattice_desc {
  int32_t lx, ly;        /* lx >= 3, ly >= 6                                   */
  double tau;            /* > 0.5                                              */
  double g;              /* gravity magnitude along -y                         */
  double t_top, t_bottom;
  double rho0;           /* FP32 shift density                                 */
  void* f_a;             /* current state after creation                       */
  void* f_b;             /* second buffer; both lbm_state_bytes() bytes        */
} lbm_lattice_desc;

typedef struct lbm_batch lbm_batch;

/* Number of launch candidates lbm_batch_autotune chooses from (the nine tile
 * shapes of the shared-memory tile kernel, then the per-lattice launches,
 * then the three tile shapes of the parameter-table kernel), the block shape
 * of candidate `i` (threads along x and y), its sites per thread along y (a
 * tile covers bx x (by * rows) sites), whether it launches the single-lattice
 * kernel once per lattice (1) or not (0), and its kind (LBM_BATCH_*).
 * LBM_ERR_INVALID for a bad i. */
enum { LBM_BATCH_SHARED_TILES = 0, LBM_BATCH_PER_LATTICE = 1, LBM_BATCH_PARAM_TILES = 2 };
int lbm_batch_tile_count(void);
int lbm_batch_tile_shape(int i, int* bx, int* by);
int lbm_batch_tile_rows(int i);
int lbm_batch_tile_per_lattice(int i);
int lbm_batch_tile_kind(int i);

/* Create a batch of n >= 1 lattices in `precision` (LBM_FP64 or
 * LBM_FP32_SHIFTED).  descs is a host array of n entries.  stream: cudaStream_t. */
int lbm_batch_create(lbm_batch** out, int n, const lbm_lattice_desc* descs, int precision,
                     void* stream);

/* Synchronise the batch's stream, then release its device tables, streams
 * and graphs (the caller's lattice buffers are untouched).  NULL is
 * accepted. */
void lbm_batch_destroy(lbm_batch* b);

/* Message of the last failed call on b (never NULL; owned by the batch;
 * "null batch" for b == NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Lattice i := f^eq(rho, u, T) (device fields [ly_i][lx_i]). */
int lbm_batch_init(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy,
                   const double* T);

/* Select launch candidate `tile` (0 .. lbm_batch_tile_count()-1). */
int lbm_batch_set_tile(lbm_batch* b, int tile);

/* Time every launch candidate over `steps` batch steps each (after one
 * untimed step), keep the fastest and return its index in *best (and, if
 * times_ms is not NULL, each candidate's time per step in
 * times_ms[lbm_batch_tile_count()]).  The lattices
 * advance by (steps + 1) x lbm_batch_tile_count() steps: re-initialise
 * afterwards.  Synchronises the stream. */
int lbm_batch_autotune(lbm_batch* b, int steps, int* best, double* times_ms);

/* Advance every lattice by n >= 0 steps with one CUDA graph launch (the graph
 * of n steps is captured on first use and cached). */
int lbm_batch_step(lbm_batch* b, int n);

/* Advance every lattice by n >= 0 steps with ONE persistent cooperative
 * launch: blocks stride over the tile list (32 x 4 blocks, 8 rows per
 * thread) and meet at a grid barrier between steps.  LBM_FP32_SHIFTED
 * batches of at most 64 lattices whose lattices each hold fewer than 2^31
 * elements run the parameter-table kernel (every lattice's constants in the
 * kernel parameters; after the tiles, the blocks stride over the wall-row
 * sites); other batches stage each tile's constants in shared memory.  Every barrier wait is bounded (2 s of global time or
 * 2^24 polls); if a wait gives up, the kernel sets a status flag and all
 * blocks return, and lbm_batch_status() reports LBM_ERR_TIMEOUT.  Same
 * results as lbm_batch_step up to rounding (the loads use the L2-coherent
 * path because each step reads what other blocks wrote in the step
 * before). */
int lbm_batch_step_persistent(lbm_batch* b, int n);

/* Self-test of the bounded wait: launches a two-block kernel whose grid
 * barrier expects a third block that never comes.  Returns LBM_ERR_TIMEOUT
 * when the wait gave up after `budget_ms` (1..10000) as designed, LBM_OK if it
 * did not time out (a failure of the self-test), or another error.  Clears
 * the barrier state afterwards; the batch stays usable. */
int lbm_batch_barrier_selftest(lbm_batch* b, int budget_ms);

/* Device pointer of the buffer holding lattice i's current state. */
void* lbm_batch_current(const lbm_batch* b, int i);

/* eq. (2) fields of lattice i's current state (device [ly_i][lx_i]). */
int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy, double* T);

/* Total physical sites of the batch (sum of lx_i * ly_i). */
long long lbm_batch_sites(const lbm_batch* b);

/* Synchronise and report the first asynchronous error: a CUDA error
 * (LBM_ERR_CUDA) or a timed-out persistent-step barrier (LBM_ERR_TIMEOUT). */
int lbm_batch_status(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_BATCH_H */
