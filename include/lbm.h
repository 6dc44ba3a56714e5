/*
 * lbm.h - C ABI of the GB300 D2Q37 thermal lattice Boltzmann library (liblbm.so).
 *
 * The library runs the time step of the D2Q37 thermal LB model of
 * Calore et al., "Performance and portability of accelerated lattice
 * Boltzmann applications with OpenACC" (arXiv 1703.00186):
 *   eq. (1)  f_l(x, t+1) = f_l(x - c_l, t) - (1/tau) (f_l(x - c_l, t) - f_l^eq),
 *   eq. (2)  rho = sum_l f_l,  rho u = sum_l c_l f_l,  D rho T = sum_l |c_l - u|^2 f_l,
 * executed as propagate, then bc, then collide (Sect. 2), fused into one
 * CUDA kernel per step for sm_103a.
 *
 * Model readings where the paper is silent:
 *  - Velocity set: the 37 integer vectors xi with |xi_x|,|xi_y| <= 3 and
 *    |xi|^2 in {0,1,2,4,5,8,9,10}; c_l = r xi_l, with r and the shell weights
 *    solved from the order-8 Gaussian isotropy conditions.
 *  - Equilibrium: 4th-order Hermite expansion of the Maxwellian about T = 1.
 *  - Collide: plain BGK, omega = 1/tau; gravity g along -y as the equilibrium
 *    shift u' = u + tau g, T' = T + tau (1 - tau) g^2 / 2.
 *  - Walls (bc, Sect. 2): top and bottom rows; after propagate, the 26 slots
 *    per column and wall whose pull source lies beyond the wall are set to
 *    M(x) q_l, where M(x) is the mass that crossed that wall and lands in
 *    column x (summed in the order: population l ascending, then source row
 *    ascending, round-to-nearest, no contraction) and q_l = phi_l / sum phi
 *    over the 26 slots, phi_l = f^eq_l(1, 0, T_wall), rounded once from an
 *    exact value.  Left/right edges are periodic.
 *
 * POPULATION ORDER.  l = 0 is xi = (0,0).  For k = 0..17, l = 2k+1 is +R_k and
 * l = 2k+2 is -R_k with R = (1,0) (0,1) (1,1) (-1,1) (2,0) (0,2) (2,1) (1,2)
 * (-1,2) (-2,1) (2,2) (-2,2) (3,0) (0,3) (3,1) (1,3) (-1,3) (-3,1).
 *
 * STATE LAYOUT.  A lattice state is one contiguous device buffer of
 * 37 planes; plane l holds rows y = -3 .. ly+2 (three halo rows below and
 * above the ly physical rows), each row lx elements, x fastest:
 *     f[(l * (ly + 6) + (y + 3)) * lx + x]
 * (the structure-of-arrays layout of Sect. 4, Fig. "streamscheme").
 * Element type: double (LBM_FP64, LBM_FP64_DF), or float holding
 * f_l - w_l rho0 (LBM_FP32_SHIFTED).  Halo rows are never read as data and never written
 * by a step: they may hold anything, NaN included.
 * Macroscopic fields are double arrays of ly rows of lx, x fastest.
 *
 * OWNERSHIP.  The caller owns every lattice and field buffer (device memory
 * unless stated otherwise) and the CUDA stream.  A context allocates one
 * small device block of its own (status word and flags, freed by
 * lbm_destroy); a batch allocates its own tables (include/lbm_batch.h).
 * All work is enqueued asynchronously on the context's stream; a call
 * returns once its work is enqueued.
 *
 * ERRORS.  Every int-returning call returns LBM_OK (0) or a negative code;
 * lbm_last_error() gives a message.  Invalid arguments are rejected before
 * any work is enqueued.  Errors of asynchronous work appear at a later call
 * or at lbm_status().  No call throws or aborts.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_NPOP 37
#define LBM_HALO 3

enum {
  LBM_OK = 0,
  LBM_ERR_INVALID = -1,   /* bad argument (NULL, out of range, bad mode)     */
  LBM_ERR_SIZE = -2,      /* buffer size does not match the lattice          */
  LBM_ERR_CUDA = -3,      /* a CUDA runtime call failed                      */
  LBM_ERR_NONFINITE = -4, /* reserved: state check found NaN/Inf             */
  LBM_ERR_TIMEOUT = -5,   /* a bounded device wait gave up                   */
  LBM_ERR_STATE = -6      /* call not valid in the object's current state    */
};

/* Storage and arithmetic of the step:
 *   LBM_FP64         float64 populations, float64 arithmetic; the moment sums
 *                    of eq. (2) are formed exactly (96-bit fixed point on the
 *                    integer pipe) and rounded once, which is at least as
 *                    accurate as float64 additions;
 *   LBM_FP32_SHIFTED float32 deviations f_l - w_l rho0; moment sums with an
 *                    error of at most 2^-35 per term, double-float density
 *                    and temperature terms, float32 polynomial, and a
 *                    correction that makes the collide conserve mass and
 *                    energy and add exactly rho g to the momentum;
 *   LBM_FP64_DF      float64 populations; the collide runs in double-float
 *                    arithmetic (two float32 words, about 48 significant
 *                    bits) on the FP32 pipe, whose issue rate on GB300 is 64
 *                    times the FP64 rate.  Propagate and bc are identical
 *                    (bit-exact); every other call treats the state as
 *                    LBM_FP64, except that lbm_adjoint_step evaluates the
 *                    equilibrium's cotangent sums in double-float too. */
enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1, LBM_FP64_DF = 2 };
enum {
  LBM_FLAG_PERIODIC_Y = 1,   /* test mode: no walls, y periodic */
  /* Regularised collide (LBM_FP64 only): the populations are projected onto
   * the velocity polynomials of degree <= 4 (the tensor Hermite polynomials of
   * order <= 4, weight w) before relaxing, f <- f^eq + (1 - omega) Pi(f - f^eq):
   * the "projection onto a basis of Hermite polynomials" of Sect. 2.  Mass,
   * momentum and energy change exactly as in plain BGK.  The adjoint calls
   * refuse contexts with this flag. */
  LBM_FLAG_REGULARIZED = 2,
  /* LBM_FP32_SHIFTED steps stage each tile's pull sources in shared memory
   * with TMA loads instead of per-thread loads, where lx is a multiple of 4,
   * y has walls and the buffers are 16-byte aligned (otherwise the flag is
   * ignored).  Bit-identical results.  Measured slower than the default on
   * GB300 (the per-tile block barrier costs more issue slots than the load
   * latency it hides); kept for comparison. */
  LBM_FLAG_TMA_LOADS = 4,
  /* Arithmetic of the LBM_FP32_SHIFTED collide (at most one of the two; the
   * storage, every other call and the adjoint are unchanged):
   *   (neither)                 the default: split moment sums, double-float
   *                             density and temperature terms, float32
   *                             coefficients and polynomial, and the
   *                             conserved-moment correction (see LBM_FP32_SHIFTED);
   *   LBM_FLAG_FP32_F64_TERMS   the conserved-moment sums of eq. (2) exact
   *                             (rounded once to float64) on the populations
   *                             w_l rho0 + d_l, the site fields and every
   *                             temperature-dependent equilibrium term (the
   *                             per-shell coefficients and the zeroth-order
   *                             deviation w (rho A0 - rho0)) in float64, each
   *                             rounded once to float32; the cu-dependent
   *                             polynomial and the relaxation in float32; no
   *                             correction;
   *   LBM_FLAG_FP32_F64_COLLIDE the LBM_FP64 collide on the decoded
   *                             populations, re-encoded to float32: the error
   *                             of the float32 storage alone. */
  LBM_FLAG_FP32_F64_TERMS = 8,
  LBM_FLAG_FP32_F64_COLLIDE = 16
};

typedef struct lbm_params {
  int32_t lx;         /* physical columns, >= 3 (periodic)                    */
  int32_t ly;         /* physical rows, 6 <= ly <= 262140 (walls at both ends) */
  int32_t precision;  /* LBM_FP64, LBM_FP32_SHIFTED or LBM_FP64_DF             */
  int32_t flags;      /* LBM_FLAG_* bits                                      */
  double tau;         /* relaxation time, > 0.5 (eq. 1)                        */
  double g;           /* gravity magnitude, acting along -y                    */
  double t_top;       /* wall temperature of the top rows                      */
  double t_bottom;    /* wall temperature of the bottom rows                   */
  double rho0;        /* density of the FP32 shift f_l - w_l rho0              */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of one lattice state buffer: 37 * (ly + 6) * lx * element size.
 * Returns 0 for invalid parameters. */
size_t lbm_state_bytes(const lbm_params* p);

/* Create a context over two caller-owned device state buffers f_a, f_b of
 * `bytes` each (ping-pong; f_a holds the current state after creation).
 * `stream` is a cudaStream_t (NULL = legacy default stream).  Solves the
 * D2Q37 quadrature and the wall ratios on the host.  *out is NULL on error. */
int lbm_create(lbm_ctx** out, const lbm_params* p, void* f_a, void* f_b,
               size_t bytes, void* stream);

/* Release the context and its small device block; the caller's buffers are
 * untouched.  NULL is accepted. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last error on this context (never NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Change the stream used by later calls. */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Initial assignment of the populations (Sect. 2: "an initial assignment of
 * the populations"): current state := f^eq(rho, u, T) at every physical
 * site.  rho, ux, uy, T: device arrays [ly][lx]. */
int lbm_init(lbm_ctx* ctx, const double* rho, const double* ux,
             const double* uy, const double* T);

/* Advance n >= 0 time steps (Sect. 2: propagate, bc, collide; eq. 1).  Each
 * step is one fused kernel launch reading the current buffer and writing the
 * other; the buffers then swap roles. */
int lbm_step(lbm_ctx* ctx, int n);

/* The same n >= 0 steps as lbm_step, replayed as one CUDA graph launch on
 * the context's stream: the n step launches are captured once per (n,
 * current buffer) on a private stream, instantiated and cached in the
 * context (released by lbm_destroy).  For small lattices, whose steps are
 * shorter than their launch overhead.  Bit-identical results to lbm_step.
 * The first call for a given n captures; make it outside any stream capture
 * of the caller's own. */
int lbm_step_graph(lbm_ctx* ctx, int n);

/* One time step from state src into state dst (caller buffers in the
 * context's precision, must not alias), leaving the context's own buffers and
 * current state untouched.  Used to recompute checkpointed trajectories. */
int lbm_step_from(lbm_ctx* ctx, const void* src, void* dst);

/* x-slab decomposition (Sect. 4: the lattice split along x over devices in a
 * ring, each sub-lattice surrounded by three halo columns that the pbc step
 * refills from the neighbours' adjoining physical columns; bulk sites, which
 * read no halo column, overlap that exchange, Fig. "schedulingop").  A slab
 * of w physical columns is a lattice of lx = w + 6 columns: columns 0..2 and
 * w+3..w+5 are the halos, w+3 <= lx.
 *
 * lbm_step_columns: one time step from state src into state dst for the
 *   sites of columns x0 <= x < x1 only (every physical row); the other
 *   columns of dst are not written.  Column x pulls from columns x-3 .. x+3
 *   (periodic in lx), so a slab's physical columns 3 <= x < w+3 read only
 *   the slab and its halos.  0 <= x0 <= x1 <= lx; src and dst must not alias.
 * lbm_pack_columns: copy columns x0 .. x0+n-1 of every population's physical
 *   rows of state f into the contiguous buffer buf[37][ly][n] (element type of
 *   the context's precision), for a send.
 * lbm_unpack_columns: the inverse, from buf into those columns of f.
 *   0 <= x0, 0 <= n, x0 + n <= lx.  Device buffers; asynchronous on the
 *   context's stream. */
int lbm_step_columns(lbm_ctx* ctx, const void* src, void* dst, int x0, int x1);
int lbm_pack_columns(lbm_ctx* ctx, const void* f, int x0, int n, void* buf);
int lbm_unpack_columns(lbm_ctx* ctx, const void* buf, int x0, int n, void* f);

/* Device pointer of the buffer holding the current state. */
void* lbm_current(const lbm_ctx* ctx);

/* Make the context's other buffer the current state (no device work): after
 * a step written into it piecewise with lbm_step_columns, as lbm_step does
 * after each step. */
int lbm_swap(lbm_ctx* ctx);

/* Which kernel lbm_step runs for this context: LBM_PATH_TMA when the
 * LBM_FP32_SHIFTED step stages its pull sources with TMA loads (requested
 * with LBM_FLAG_TMA_LOADS and supported), LBM_PATH_PLAIN otherwise
 * (per-thread loads).  LBM_ERR_INVALID for a NULL context. */
enum { LBM_PATH_PLAIN = 0, LBM_PATH_TMA = 1 };
int lbm_step_path(const lbm_ctx* ctx);

/* Macroscopic fields of eq. (2) of the state f (NULL = current state), as
 * raw moments of the stored populations: rho, u = j / rho,
 * T = (E / rho - |u|^2) / D.  Outputs: device arrays [ly][lx]. */
int lbm_moments(lbm_ctx* ctx, const void* f, double* rho, double* ux,
                double* uy, double* T);

/* Measurement routines (Sect. 2: averages of physical observables taken every
 * several hundred or thousand steps).  LBM_NOBS quantities are averaged over x
 * for every physical row y:
 *   0 rho, 1 u_x, 2 u_y, 3 T, 4 T^2, 5 u_y T, 6 rho |u|^2 / 2, 7 rho u_y,
 * with eq. (2) fields and the hydrodynamic (mid-step) velocity
 * u = (sum c f - rho g_vec / 2) / rho, g_vec = (0, -g), of the stored state.
 * Output: device double array [LBM_NOBS][ly].
 * lbm_profiles: of state f (NULL = current); deterministic reduction. */
#define LBM_NOBS 8
int lbm_profiles(lbm_ctx* ctx, const void* f, double* out);

/* Advance n >= 0 steps like lbm_step, and after every `every`-th step
 * (steps every, 2 every, ...) store the row averages of the new state in the
 * next record of `out` (device double array [n / every][LBM_NOBS][ly]).  The
 * observing steps compute the averages in the step kernel itself from the
 * moments the collide already forms (exact warp sums, then one atomic add
 * per warp and quantity, so the order across warps is not fixed: results
 * agree with lbm_profiles to rounding).  LBM_FP64 contexts
 * without LBM_FLAG_REGULARIZED only; every >= 1.  *records (host, may be NULL)
 * receives the number of records written. */
int lbm_step_observe(lbm_ctx* ctx, int n, int every, double* out, int* records);

/* Checkpoint / restore: copy the current state to / from a caller buffer of
 * lbm_state_bytes() (device memory, or host memory the CUDA runtime can
 * address, e.g. pinned). */
int lbm_get_state(lbm_ctx* ctx, void* dst);
int lbm_set_state(lbm_ctx* ctx, const void* src);

/* propagate followed by bc only (Sect. 2, first two kernels), from state src
 * to state dst (both in the context's precision; must not alias).  The
 * current state is not changed. */
int lbm_propagate_bc(lbm_ctx* ctx, const void* src, void* dst);

/* One step of the discrete adjoint (transpose of the Jacobian of one step,
 * eq. 1 with propagate, bc and collide, linearised at state f_t):
 *   lam_out = P^T B^T C^T lam_in.
 * f_t: state in the context's precision (FP32 states are decoded and the
 * Jacobian of the float64 step is taken there).  LBM_FP64 contexts evaluate
 * it in float64; LBM_FP64_DF and LBM_FP32_SHIFTED contexts evaluate the
 * equilibrium's cotangent sums in double-float (about 48 bits), the rest in
 * float64.  lam_in, lam_out: double arrays in the FP64 state layout; must not
 * alias.  The halo rows of lam_out are used as scratch and hold no data
 * afterwards. */
int lbm_adjoint_step(lbm_ctx* ctx, const void* f_t, const double* lam_in,
                     double* lam_out);

/* The adjoint step without a context and without any device allocation.
 * The paper has no counterpart of this call.
 *
 * Who needs it: lbm_create allocates a small device block, so a caller that
 * cannot call cudaMalloc cannot create a context.  Such callers include a
 * host application whose device memory is all handed out by another allocator
 * (for example a framework's caching allocator that reserved the GPU up
 * front), and code that must not allocate after its set-up phase because
 * cudaMalloc can synchronise the device.  Its result equals that of
 * lbm_adjoint_step for a context with parameters *p up to rounding: this call
 * sums the equilibrium's cotangents pair by pair in float64 for every
 * precision, where the context call contracts w-weighted cotangent moments
 * (LBM_FP64) or sums in double-float (LBM_FP64_DF, LBM_FP32_SHIFTED).
 *
 * Arguments: f_t, lam_in and lam_out as for lbm_adjoint_step (caller-owned
 * device buffers, must not alias); stream is a cudaStream_t (NULL = legacy
 * default stream).  The lattice constants are derived on the host at every
 * call.
 *
 * Scratch: the per-wall-row sums that lbm_adjoint_step keeps in the halo rows
 * of lam_out go instead to one fixed array inside the library of
 * 6 x LBM_NOALLOC_MAX_LX doubles (768 KiB).  Every GPU that loads the library
 * holds this array until the process exits.  The halo rows of lam_out are
 * left untouched.
 *
 * Set-up: every call looks up the array's device address on the current
 * device (a host-side lookup, no device work), so the address stays right
 * after a device reset.  The first call on a device also loads the library's
 * device code there; make that first call before any stream capture.
 *
 * Errors: an error that earlier, unrelated calls left in the CUDA runtime's
 * last-error state is cleared before the launches, so LBM_ERR_CUDA reports
 * this call's own launch failures (and errors that the device context keeps
 * for every call).
 *
 * Sharing: every call shares the array, and the array keeps the last call's
 * contents.  Each call overwrites every entry it reads, so nothing needs
 * clearing.  Calls that overlap on the GPU (other streams, other host threads)
 * race and give wrong results; calls ordered on one stream are safe.
 *
 * Returns LBM_OK; LBM_ERR_SIZE if p->lx > LBM_NOALLOC_MAX_LX (no work done);
 * LBM_ERR_INVALID for bad parameters or pointers; LBM_ERR_CUDA if the address
 * lookup or a launch fails. */
#define LBM_NOALLOC_MAX_LX 16384
int lbm_adjoint_step_noalloc(const lbm_params* p, const void* f_t,
                             const double* lam_in, double* lam_out, void* stream);

/* Vector-Jacobian product of lbm_moments at state f:
 *   lam_out_l = d rho/d f_l g_rho + d u/d f_l . g_u + d T/d f_l g_T
 * (eq. 2).  Cotangent fields [ly][lx]; any of them may be NULL (zero).
 * lam_out: double array in the FP64 state layout. */
int lbm_moments_vjp(lbm_ctx* ctx, const void* f, const double* g_rho,
                    const double* g_ux, const double* g_uy, const double* g_T,
                    double* lam_out);

/* Vector-Jacobian product of lbm_init: for lam in the FP64 state layout,
 * g_x = sum_l lam_l d f^eq_l / d x at (rho, u, T) for x in {rho, ux, uy, T}.
 * Outputs [ly][lx]; any output may be NULL (not computed). */
int lbm_init_vjp(lbm_ctx* ctx, const double* rho, const double* ux,
                 const double* uy, const double* T, const double* lam,
                 double* g_rho, double* g_ux, double* g_uy, double* g_T);

/* Float32 cotangents for LBM_FP32_SHIFTED contexts.  The paper has no
 * counterpart of these calls: they make the discrete adjoint of the FP32-store
 * step as cheap as its storage allows.
 *
 * lbm_adjoint_step_f32: lam_out = P^T B^T C^T lam_in as lbm_adjoint_step, with
 * lam_in and lam_out float arrays in the FP32 state layout (37 planes of
 * (ly + 6) x lx, must not alias).  The site fields of f_t are formed as in
 * lbm_adjoint_step (exact moment sums, float64 rho, u, T) and rounded to
 * float32; every cotangent sum, the relaxation of the cotangents and the
 * transposed walls run in float32, so a result is within a few float32
 * roundings (relative 1e-6 of the site's largest cotangent) of the float64
 * adjoint of the decoded state.  The halo rows of lam_out are used as scratch
 * and hold no data afterwards.  LBM_ERR_INVALID for a context of another
 * precision or for bad buffers.
 *
 * lbm_moments_vjp_f32, lbm_init_vjp_f32: lbm_moments_vjp with a float32
 * lam_out (computed in float64, rounded once), and lbm_init_vjp reading a
 * float32 lam; any precision. */
int lbm_adjoint_step_f32(lbm_ctx* ctx, const void* f_t, const float* lam_in,
                         float* lam_out);
int lbm_moments_vjp_f32(lbm_ctx* ctx, const void* f, const double* g_rho,
                        const double* g_ux, const double* g_uy,
                        const double* g_T, float* lam_out);
int lbm_init_vjp_f32(lbm_ctx* ctx, const double* rho, const double* ux,
                     const double* uy, const double* T, const float* lam,
                     double* g_rho, double* g_ux, double* g_uy, double* g_T);

/* Check that every physical population of state f (NULL = current) is
 * finite.  Synchronises the stream; *ok = 1 if finite, else 0. */
int lbm_check_finite(lbm_ctx* ctx, const void* f, int* ok);

/* Synchronise the stream and return the first error of asynchronous work:
 * a CUDA error (LBM_ERR_CUDA) or the device status word (LBM_ERR_*). */
int lbm_status(lbm_ctx* ctx);

/* Copy of the float64 constants the context derived: r, the 37 weights w_l
 * and the wall ratios q_l of the bottom and top walls (zero where slot l is
 * not an unknown of that wall).  Any pointer may be NULL. */
int lbm_constants(const lbm_ctx* ctx, double* r, double* w37,
                  double* q_bottom37, double* q_top37);

/* The same constants without a context, for the lattice parameters *p: the
 * quadrature (velocity set and weights of the D2Q37 model, Sect. 2) and the
 * wall ratios of the thermal walls at p->t_bottom and p->t_top (bc, Sect. 2),
 * all derived on the host.  No device work and no allocation: callable on a
 * machine without a GPU.  Returns LBM_ERR_INVALID for invalid parameters (as
 * lbm_create would); any output pointer may be NULL. */
int lbm_model_constants(const lbm_params* p, double* r, double* w37,
                        double* q_bottom37, double* q_top37);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
