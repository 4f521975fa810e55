/*
 * lbmwet.h - C ABI of a GB300 (sm_103a) implementation of one time step of the pseudopotential
 * multiple-relaxation-time lattice Boltzmann method with contact angles on curved walls:
 * Q. Li, Y. Yu, K. H. Luo, "Implementation of contact angles in the pseudopotential lattice
 * Boltzmann simulations with curved boundaries", arXiv:1908.04443.
 *
 * One time step (Sec. II.A, Sec. III.B) is, per fluid node x:
 *   streaming with halfway bounce-back at walls        Eq. 3, Fig. 3
 *   rho = sum_a f_a                                      Eq. 4
 *   psi(rho) from the equation of state                  Eq. 6 with Eq. 18 (PR) or Carnahan-Starling
 *   virtual wall density rho_w at solid nodes next to fluid, improved scheme with limiter
 *                                                         Eqs. 16-17 (Sec. III.B); constant VD Sec. II.B
 *   F_m = -G psi(x) sum_a w_a psi(x + e_a) e_a            Eq. 5
 *   rho u = sum_a e_a f_a + F/2                          Eq. 4
 *   MRT collision with the consistency forcing            Eqs. 1, 2, 7
 *
 * Conventions for every entry point:
 *   - Grids are periodic in every direction; node (x, y, z) has linear index x + nx*(y + ny*z)
 *     (x fastest).  2D lattices use nz = 1.
 *   - Host pointers are read (or written) only during the call; the caller keeps ownership.
 *     Device memory is owned by the handle and freed by lbm_destroy, into the library's
 *     stream-ordered memory pool of the device (one per device), which keeps it for the next
 *     allocation instead of returning it to the driver; lbm_release_cached_memory returns it.
 *   - All device work is enqueued on the caller's CUDA stream given at lbm_init (NULL = the
 *     legacy default stream).  Calls that return host data synchronise that stream.
 *   - Calls return an lbm_status and never abort or throw.  lbm_last_error() gives a message.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Device-side numerical faults (a non-positive square-root argument in Eq. 6, a non-positive
 *     or non-finite density) set a sticky flag on the device; lbm_step and lbm_observables read
 *     it once per call and return LBM_ERR_UNSTABLE.  Nothing on the device traps, and its only
 *     waits (on the mbarriers of TMA copies) give up after a bounded number of polls: a copy that
 *     never lands sets another flag, which the same calls report as LBM_ERR_CUDA.
 */
#ifndef LBMWET_H
#define LBMWET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,       /* invalid argument or configuration                                */
    LBM_ERR_CUDA = 2,      /* a CUDA runtime call failed (message in lbm_last_error)           */
    LBM_ERR_OOM = 3,       /* device allocation failed                                          */
    LBM_ERR_UNSTABLE = 4,  /* the device flagged psi's square-root argument <= 0, rho <= 0 or NaN */
    LBM_ERR_STATE = 5      /* call not valid in the handle's current state                     */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Storage/compute precision of the distributions.
 * LBM_FP64:     f stored and computed in double.
 * LBM_FP32_DEV: f stored in float as deviations f_a - w_a rho_ref (w_a the equilibrium weights),
 *               computed in float; reductions of observables in double. */
typedef enum { LBM_FP64 = 0, LBM_FP32_DEV = 1 } lbm_precision;

/* Equations of state.  PR: Eq. 18 with Tc = 0.0778 a / (0.45724 b R).
 * CS: p = rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2, eta = b rho / 4. */
typedef enum { LBM_EOS_PR = 0, LBM_EOS_CS = 1 } lbm_eos_kind;

/* Wall schemes.  IVD: Eqs. 16-17 with the limiter rho_g <= rho_w <= rho_l (Sec. III.B), the
 * parameter in the unified form kappa >= 0 -> phi = 1 + kappa, kappa < 0 -> drho = -kappa.
 * VD: the constant virtual density rho_w_const of Benzi et al. (Sec. II.B).
 * SF: the solid-fluid interaction of Martys and Chen (Eq. 8): psi = 0 on solid nodes and the
 * adhesion force F_ads = -Gw rho(x) sum_a w_a s(x + e_a) e_a added to the force of every fluid
 * node (Gw < 0 wets, Gw > 0 repels); the consistency term of Eq. 7 keeps F_m of Eq. 5 alone.
 * GF (D2Q9 only): the curved geometric formulation (Sec. III.A, Eqs. 10-15) for a prescribed
 * angle theta_a: at each wall node P, the surface normal of Eq. 13 (eighth-order weights of
 * Eq. 14) rotated by +-(90 - theta_a) degrees (Eq. 15) gives two characteristic lines; each is
 * followed to the first mesh line it crosses (x or y one node from P), where the density is
 * interpolated linearly between the two fluid nodes of that mesh segment (a solid end is dropped;
 * a crossing with no fluid end is unused); rho_w = max of the two (theta_a <= 90) or min (Eq. 11),
 * or the mean of Eq. 17 when neither crossing is usable.  A wall node whose Eq. 13 sum vanishes
 * (a one-node-thin solid, for example) has no normal: lbm_init rejects such a mask. */
typedef enum { LBM_WALL_IVD = 0, LBM_WALL_VD = 1, LBM_WALL_SF = 2, LBM_WALL_GF = 3 } lbm_wall_kind;

/* Solid body used for the contact-angle observable.  BALL: a circle (2D) / sphere (3D) of
 * radius body_radius about body_center, wall at body_radius + 1/2 (halfway bounce-back).
 * PLANE: a flat wall at y = body_center[1] (the halfway position), liquid at larger y. */
typedef enum { LBM_BODY_NONE = 0, LBM_BODY_BALL = 1, LBM_BODY_PLANE = 2 } lbm_body_kind;

/* Step kernel (no counterpart in the paper: a choice of work decomposition).
 * D2Q9:
 *   TILE: one CTA per 32 x 8 tile with its halo ring, one node per thread.  YMARCH: persistent
 *   CTAs walking runs of rows of column blocks (124 own columns plus a 2-cell halo on each side),
 *   planned on the host so that every CTA pulls about the same number of rows; bit-identical to
 *   TILE.  PAIR (FP32 only): 32 x 16 tiles, two nodes per thread computed together with packed
 *   FP32x2 instructions; equal to TILE up to FP32 rounding (the operations are regrouped).  AUTO:
 *   PAIR in FP32, TILE in FP64.  A batch uses instance 0's choice for every instance, except that
 *   with AUTO each instance takes the kernel lbm_batch_autotune chose for its size class, where it
 *   has chosen one.  A y-march handle that records a trajectory for the adjoint steps with TILE
 *   from lbm_record on.
 * D3Q19 (every kernel marches z-planes through 32-plane chunks of x-y columns):
 *   ZTMA (FP32 only): 32 x 8 columns cut along z into the work items of lbm_d3q19_work_list, one
 *   CTA per item; the lead plane's 19 pull boxes are staged in shared memory by TMA, two planes in
 *   flight, two cells per thread in packed FP32x2 arithmetic; items on planes near a solid also
 *   stage node types and do the bounce-back and virtual-density work; columns cut by the grid's
 *   edge (ragged) run the z-pair march.  PAIR (FP32 only): the z-pair march, 32 x 4 columns, two planes
 *   per thread.  TILE: the scalar z-march (the only D3Q19 kernel in FP64).  AUTO: ZTMA in FP32
 *   (PAIR where the rows are not a multiple of 16 bytes), TILE in FP64.  The FP32 kernels agree up
 *   to FP32 rounding. */
typedef enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_TILE = 1, LBM_KERNEL_YMARCH = 2, LBM_KERNEL_PAIR = 3,
               LBM_KERNEL_ZTMA = 4 } lbm_step_kernel;

typedef struct {
    int32_t kind;      /* lbm_eos_kind                                       */
    double a, b, R;    /* EOS constants                                      */
    double T;          /* absolute temperature (> 0, below the critical one) */
    double omega;      /* PR acentric factor (Sec. IV.A uses 0.344)          */
} lbm_eos;

typedef struct {
    int32_t lattice;            /* lbm_lattice                                                    */
    int32_t precision;          /* lbm_precision                                                  */
    int32_t nx, ny, nz;         /* grid; nz = 1 for D2Q9; each >= 1                               */
    lbm_eos eos;
    double G;                   /* interaction strength of Eqs. 5-6 (the paper uses -1)           */
    double sigma;               /* consistency constant of Eq. 7                                  */
    /* MRT rates s = 1/tau (Lambda of Eq. 2).  D2Q9 uses s_rho, s_e, s_eps, s_j, s_q, s_nu;
     * D3Q19 also s_pi (3pi_xx, pi_ww) and s_m (m_x, m_y, m_z).  Each in (0, 2). */
    double s_rho, s_e, s_eps, s_j, s_q, s_nu, s_pi, s_m;
    double rho_l, rho_g;        /* limiter bounds (Sec. III.B); both <= 0 -> Maxwell construction */
    double rho_ref;             /* LBM_FP32_DEV offset of the stored deviations                  */
    double body_force[3];       /* constant body force added to F                               */
    int32_t wall_kind;          /* lbm_wall_kind                                                  */
    double kappa;               /* IVD parameter for every wall node (unless given per node)    */
    double rho_w_const;         /* VD constant virtual density                                   */
    int32_t body_kind;          /* lbm_body_kind (observables only)                              */
    double body_center[3];
    double body_radius;
    double drop_hint[3];        /* a point inside the drop: interface points are unwrapped to the
                                   periodic image nearest to it                                  */
    int32_t step_kernel;        /* lbm_step_kernel                                               */
    double Gw;                  /* SF adhesion parameter (Eq. 8)                                 */
    double theta_a;             /* GF prescribed contact angle, degrees in (0, 180)              */
} lbm_config;

typedef struct {
    double mass;            /* sum of rho over fluid nodes                                     */
    double rho_max, rho_min;/* fluid density extremes (Fig. 11)                                */
    double u_max;           /* maximum |u| over fluid nodes, u from Eq. 4 (Fig. 10)            */
    double theta_deg;       /* contact angle through the liquid; NaN if not measurable         */
    double drop_center[3];  /* fitted drop circle/sphere                                       */
    double drop_radius;
    int64_t n_interface;    /* interface points used by the fit                                */
    int64_t step;           /* time steps taken since lbm_init / lbm_set_state                 */
} lbm_obs;

typedef struct lbm_handle lbm_handle;

/* Coexistence densities of an EOS by the Maxwell equal-area rule (the target of the paper's
 * thermodynamic consistency, Sec. II.A; Sec. IV.A quotes rho_g ~ 0.38, rho_l ~ 6.5 for PR at
 * 0.86 Tc).  Host-only computation.  Errors: LBM_ERR_ARG if T is not below the critical
 * temperature or an argument is NULL. */
lbm_status lbm_coexistence(const lbm_eos* eos, double* rho_g, double* rho_l);

/* Critical temperature of an EOS with the given constants (T and omega ignored).  PR from the
 * definitions of a and b in Eq. 18; CS from dp/drho = d2p/drho2 = 0.  Host-only. */
lbm_status lbm_critical_temperature(const lbm_eos* eos, double* tc);

/* Create a simulation.
 *   cfg            configuration (copied).
 *   solid_mask     host, N = nx*ny*nz bytes, nonzero = solid.  Wall nodes are the solid nodes with
 *                  a fluid node among their lattice neighbours (Eq. 17 needs one).
 *   rho0           host, N doubles or NULL (uniform rho_g); values at solid nodes are ignored.
 *   u0             host, d*N doubles (component-major: u_x for all nodes, then u_y[, u_z]) or NULL.
 *   kappa_per_wall host, one IVD parameter per wall node in lbm_wall_nodes() order, or NULL to use
 *                  cfg->kappa everywhere (IVD only: LBM_ERR_ARG with the GF scheme).
 *   stream         cudaStream_t for all device work of this handle, or NULL.
 * The initial state is f = f^eq(rho0, u0) at fluid nodes (post-streaming, step 0).
 * Errors: LBM_ERR_ARG (bad sizes, rates, EOS, an all-solid grid; GF with D3Q19, theta_a outside
 * (0, 180) or a wall node without a normal), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_init(const lbm_config* cfg, const uint8_t* solid_mask, const double* rho0,
                    const double* u0, const double* kappa_per_wall, void* stream, lbm_handle** out);

/* Advance n >= 0 time steps (Eqs. 1-7 with halfway bounce-back).  Launches are asynchronous on
 * the handle's stream except for one 4-byte read of the device error flag at the end. */
lbm_status lbm_step(lbm_handle* h, int64_t n);

/* Enqueue n >= 0 time steps without reading the device error flag (no synchronisation).  A
 * fault flagged by these steps is reported by the next lbm_step, lbm_check or lbm_observables. */
lbm_status lbm_enqueue_steps(lbm_handle* h, int64_t n);

/* Synchronise the handle's stream and report the sticky device error flag (LBM_ERR_UNSTABLE). */
lbm_status lbm_check(lbm_handle* h);

/* Self-test of the device's bounded waits (no counterpart in the paper).  Every wait of the step
 * kernels on a shared-memory copy (an mbarrier) gives up after a fixed number of polls, flags
 * ERR_TIMEOUT and lets the kernel return, so a copy that never lands becomes an error status
 * (LBM_ERR_CUDA from the stepping call) instead of a hung GPU.  This call launches, on `stream`
 * (NULL: the legacy default stream), one CTA whose threads wait with `polls` polls (> 0) on an
 * mbarrier that nothing completes and no copy targets, and sets *timed_out to 1 if the waits gave
 * up and flagged the timeout (the expected outcome), 0 otherwise.  Synchronises the stream. */
lbm_status lbm_selftest_bounded_wait(void* stream, uint32_t polls, int32_t* timed_out);

/* Device memory pool (no counterpart in the paper).  Handles and batches allocate from a
 * stream-ordered pool per device (cudaMallocFromPoolAsync on their stream) whose release threshold
 * is unlimited: memory freed by lbm_destroy / lbm_batch_destroy stays reserved for later handles,
 * so repeated set-ups neither map fresh memory nor synchronise the device per buffer.
 * lbm_release_cached_memory synchronises the current device (frees pending in streams hold their
 * memory until then) and returns the unused part of every pool to the driver (memory of live
 * handles stays).  lbm_memory_stats gives the current device's pool: bytes reserved from the
 * driver and bytes in use by live allocations.  Errors: LBM_ERR_ARG (NULL argument),
 * LBM_ERR_CUDA. */
lbm_status lbm_release_cached_memory(void);
lbm_status lbm_memory_stats(int64_t* reserved_bytes, int64_t* used_bytes);

/* FP64 rate probe (no counterpart in the paper): the FP64 step kernels are bound by the device's
 * FP64 arithmetic, and their roofline needs its measured rate.  Launches, on `stream` (NULL: the
 * legacy default stream), a grid of 16 CTAs per SM whose threads run eight independent chains of
 * FP64 fused multiply-adds, times three launches after a warm-up with CUDA events and sets
 * *gflops to the best rate (2 flops per FMA).  Allocates 8 bytes of device memory for the call;
 * synchronises the stream.  Errors: LBM_ERR_ARG (NULL gflops), LBM_ERR_CUDA. */
lbm_status lbm_probe_fp64_rate(void* stream, double* gflops);

/* Memory-safety check, for tests (the paper has no counterpart).  Both distribution buffers and
 * the density / velocity fields of lbm_observables sit between two 4096-byte guard zones filled
 * with the byte 0xA5 when they are allocated; D2Q9 distribution rows also carry padding nodes
 * x in [nx, pitch), pitch = nx rounded up to 32, that lbm_init zeroes and no kernel writes.  Sets
 * *guard_bad to the number of guard bytes that no longer hold 0xA5 and *pad_bad to the number of
 * padding bytes of the distributions that are no longer 0: both 0 unless a kernel wrote outside
 * its buffers.  Copies the whole distribution buffers to the host (sized for test grids) and
 * synchronises the handle's stream.  Works on a batch instance (lbm_batch_handle). */
lbm_status lbm_check_guards(lbm_handle* h, int64_t* guard_bad, int64_t* pad_bad);

/* Observables of the current state: mass, fluid density extremes, maximum |u| (u from Eq. 4 with
 * the current force), and the contact angle (interface at (rho_l + rho_g)/2 fitted by a Kasa
 * circle/sphere, points within 3 nodes of a solid dropped).  Optionally copies the density
 * field (N doubles; 0 at solid nodes) and velocity (d*N doubles, component-major) to the host.
 * rho_host / u_host may be NULL.  Synchronises the stream. */
lbm_status lbm_observables(lbm_handle* h, lbm_obs* out, double* rho_host, double* u_host);

/* Device-resident form of the fields of lbm_observables: writes rho (N doubles) and u (d*N
 * doubles) into caller-owned DEVICE buffers (either may be NULL); no host copy, no sync. */
lbm_status lbm_fields_device(lbm_handle* h, double* rho_dev, double* u_dev);

/* Allocation-free form of the reductions of lbm_observables.  The paper has no counterpart: this
 * is for callers that must not call cudaMalloc - frameworks that route every device allocation
 * through their own allocator and memory budget, or latency-sensitive loops where cudaMalloc's
 * implicit device synchronisation is not acceptable.  It allocates nothing: the caller passes
 * the device fields (rho: N doubles, u: d*N doubles, component-major, e.g. filled by
 * lbm_fields_device into the caller's buffers) and receives the same lbm_obs as lbm_observables
 * (on the host; the call synchronises the handle's stream).  The per-block partial sums live in a
 * static device array inside the library, of fixed size (about 590 KB), present on every GPU
 * that loads the library until the process exits.
 *   - Maximum grid: 16,777,216 nodes (256^3); larger grids are rejected with LBM_ERR_ARG.
 *   - The first call on a device (with that device current) looks up the array's device address
 *     with cudaGetSymbolAddress; make that first call before any stream capture.
 *   - Every call shares the array, which keeps the last call's contents; each call writes every
 *     slot it reads, so nothing needs clearing.  Calls whose kernels overlap on the GPU (e.g. on
 *     different streams) race on the array: order them.
 * Errors: LBM_ERR_ARG (null pointer, grid too large), LBM_ERR_CUDA. */
lbm_status lbm_observables_noalloc(lbm_handle* h, const double* rho_dev, const double* u_dev, lbm_obs* out);

/* Wall nodes (linear indices, ascending) - the order of kappa_per_wall.  idx_out may be NULL
 * to query the count only. */
lbm_status lbm_wall_nodes(const lbm_handle* h, int64_t* idx_out, int64_t* count);

/* The post-streaming distributions f_a(x) of the current state as doubles, layout [a][node]
 * (q*N values; 0 at solid nodes).  Velocity order: D2Q9 e0=(0,0), (1,0), (0,1), (-1,0),
 * (0,-1), (1,1), (-1,1), (-1,-1), (1,-1); D3Q19 e0=0, +-x, +-y, +-z, then (1,1,0), (-1,-1,0),
 * (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1),
 * (0,-1,1).  Synchronises the stream. */
lbm_status lbm_get_state(lbm_handle* h, double* f_host);

/* Replace the state by post-streaming distributions in the layout of lbm_get_state (values at
 * solid nodes ignored); resets the step counter to `step`. */
lbm_status lbm_set_state(lbm_handle* h, const double* f_host, int64_t step);

/* Raw checkpoint of the stored state (storage precision) plus the step counter.  With
 * host_buf == NULL, *bytes receives the size; otherwise *bytes must be at least that size. */
lbm_status lbm_save_state(lbm_handle* h, void* host_buf, size_t* bytes);
lbm_status lbm_load_state(lbm_handle* h, const void* host_buf, size_t bytes);

/* Set the per-wall-node IVD parameter (one per wall node, lbm_wall_nodes() order).  LBM_ERR_ARG
 * for a handle of another wall scheme. */
lbm_status lbm_set_kappa(lbm_handle* h, const double* kappa_per_wall);

/* Resolved coexistence densities used by the limiter (after a Maxwell construction if asked). */
lbm_status lbm_limiter_bounds(const lbm_handle* h, double* rho_g, double* rho_l);

/* Grid of a handle: shape4 = {nx, ny, nz, d} (d = 2 for D2Q9, 3 for D3Q19), so that a caller can size
 * the host arrays of lbm_observables, lbm_get_state and lbm_set_state (N = nx*ny*nz nodes, Q = 9 or
 * 19 directions).  Errors: LBM_ERR_ARG (NULL argument). */
lbm_status lbm_grid_shape(const lbm_handle* h, int32_t* shape4);

/* Number of kernel launches this handle has issued (step kernels and others), for accounting. */
int64_t lbm_kernel_launches(const lbm_handle* h);

/* The work list of the TMA-staged D3Q19 z-march (LBM_KERNEL_ZTMA) for a solid mask: host code only
 * (no device, no handle), the list lbm_init builds for an FP32 D3Q19 handle on that kernel.  One
 * time step (Eqs. 1-7 with the Eq. 16-17 walls) is split into items, one CTA each: item i is the 5
 * int32 values items[5i .. 5i+4] = {bx, by, z0, z1, solid}: the column of cells x in [32 bx,
 * 32 bx + 32), y in [8 by, 8 by + 8) (clipped to the grid), planes z0 <= z < z1, and solid = 1 where
 * the item takes the path for planes within 3 planes of a solid near the column (node types,
 * bounce-back, virtual densities) or, for a column cut by the grid's edge, the z-pair march.  Every
 * (column, plane) lies in exactly one item; items run in ascending z0, then by, then bx.
 *   solid_mask: host, nz*ny*nx bytes (x fastest), nonzero = solid; read only during the call.
 *   items: host array of 5 * capacity int32, owned by the caller, or NULL to ask for the count.
 *   count: receives the number of items.
 * Errors: LBM_ERR_ARG (NULL mask or count, a size below 1, more than 2^31 / 19 nodes, or items
 * given with capacity below the count; nothing is written to items then). */
lbm_status lbm_d3q19_work_list(const uint8_t* solid_mask, int32_t nx, int32_t ny, int32_t nz, int32_t* items,
                               int64_t capacity, int64_t* count);

/* Step kernel the handle's lbm_step uses now (see lbm_step_kernel): LBM_KERNEL_TILE,
 * LBM_KERNEL_YMARCH or LBM_KERNEL_PAIR for D2Q9; LBM_KERNEL_ZTMA, LBM_KERNEL_PAIR or
 * LBM_KERNEL_TILE for D3Q19; LBM_KERNEL_AUTO for a NULL handle. */
int32_t lbm_step_kernel_used(const lbm_handle* h);

/* ---- Adjoint (D2Q9, IVD walls) -------------------------------------------------------------
 * Gradient of a loss of the final density, L(rho_T), with respect to the per-wall-node IVD
 * parameter kappa_j (Eq. 16 in the unified form of lbm_config.kappa), by the discrete adjoint of
 * the time step (Eqs. 1-7, 16-17, halfway bounce-back): reverse of the collision, of the force
 * of Eq. 5 through psi (Eq. 6), of the virtual wall density with its limiter (zero derivative
 * where the limiter clamps), and of the streaming.  The paper has no adjoint; this serves the
 * inverse problem of fitting wall wettability to an observed density field. */

/* Advance n_steps >= 1 steps from the current state, keeping a device checkpoint of the stored
 * state every ckpt_every steps (ceil(n_steps/ckpt_every) copies of the distributions).  Switches
 * the handle to per-wall-node kappa if it was using the scalar one.  Errors: LBM_ERR_ARG (D3Q19,
 * VD walls, bad counts), LBM_ERR_OOM, LBM_ERR_UNSTABLE. */
lbm_status lbm_record(lbm_handle* h, int64_t n_steps, int64_t ckpt_every);

/* dL/dkappa for the trajectory of the last lbm_record, whose final state must still be the
 * handle's state (else LBM_ERR_STATE).  drho_final_dev: DEVICE array of N doubles, dL/drho_T at
 * every node (ignored at solid nodes).  dkappa_host: host array, one double per wall node in
 * lbm_wall_nodes() order.  Recomputes each checkpoint segment's states, then runs the reverse
 * sweep (each segment replayed as a CUDA graph); allocates ckpt_every + 2 distribution buffers and 19 N
 * scalars of scratch for the
 * call.  Synchronises the stream. */
lbm_status lbm_adjoint(lbm_handle* h, const double* drho_final_dev, double* dkappa_host);

/* ---- Batches (no counterpart in the paper: many independent grids of one physics) ----------
 * A batch steps n grids with one persistent kernel launch per time step: a grid of CTAs sized to
 * the GPU walks a work list of (instance, tile) items covering every instance; the launches of
 * lbm_batch_step are captured in CUDA graphs of 16 steps like lbm_step's.  Instances share
 * lattice, precision and physics (EOS, G, sigma, rates, limiter bounds, rho_ref, body force,
 * wall scheme); grid size, kappa, per-wall-node kappa, body and drop hint may differ. */
typedef struct lbm_batch lbm_batch;

/* Create a batch of n >= 1 instances: cfgs[i], masks[i], rho0s[i] (array may be NULL, entries may
 * be NULL) and kappas_per_wall[i] (array or entries may be NULL) as in lbm_init.  The host scans of
 * the instances' masks (wall lists, tile flags) run in parallel on up to 16 host threads; the
 * stream is synchronised once for the whole batch.  Errors as lbm_init, plus LBM_ERR_ARG if the
 * instances' physics differ. */
lbm_status lbm_batch_init(int32_t n, const lbm_config* cfgs, const uint8_t* const* masks, const double* const* rho0s,
                          const double* const* kappas_per_wall, void* stream, lbm_batch** out);
/* Advance every instance n steps; reads the batch's device error flag once at the end. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n);
/* Enqueue n steps without reading the error flag (checked by the next lbm_batch_step). */
lbm_status lbm_batch_enqueue_steps(lbm_batch* b, int64_t n);
/* Observables of every instance (out_n has lbm_batch_size() entries). */
lbm_status lbm_batch_observables(lbm_batch* b, lbm_obs* out_n);
/* The same with, optionally, every instance's density and velocity fields copied to the host:
 * rho_hosts[i] (N_i doubles) and u_hosts[i] (d*N_i doubles, component-major) as in lbm_observables;
 * either array, or any entry, may be NULL.  All instances' fields, reductions and copies are enqueued
 * on the batch's stream and the stream is synchronised once (lbm_observables on each instance
 * synchronises per instance); the reduction results land in pinned memory owned by the batch.
 * Copies into pinned host buffers run asynchronously; the runtime completes a copy into pageable
 * memory before it returns.  lbm_batch_observables is this call without fields.  Errors:
 * LBM_ERR_ARG, LBM_ERR_UNSTABLE or LBM_ERR_CUDA for an instance whose device flag is set (its index
 * in the message), LBM_ERR_OOM. */
lbm_status lbm_batch_observables_fields(lbm_batch* b, lbm_obs* out_n, double* const* rho_hosts,
                                        double* const* u_hosts);
/* Handle of instance i, owned by the batch: valid for lbm_observables, lbm_fields_device,
 * lbm_get_state, lbm_set_state, lbm_save_state/lbm_load_state, lbm_wall_nodes; lbm_step and
 * lbm_enqueue_steps on it return LBM_ERR_STATE and lbm_destroy ignores it.  NULL if i is out of range. */
lbm_handle* lbm_batch_handle(lbm_batch* b, int32_t i);
int32_t lbm_batch_size(const lbm_batch* b);
int64_t lbm_batch_kernel_launches(const lbm_batch* b);
/* Step kernel of the batch: LBM_KERNEL_TILE, LBM_KERNEL_YMARCH or LBM_KERNEL_PAIR when every
 * instance uses the same one, LBM_KERNEL_AUTO when they differ (after lbm_batch_autotune) or for
 * NULL. */
int32_t lbm_batch_step_kernel_used(const lbm_batch* b);
/* Step kernel of instance i (LBM_KERNEL_AUTO if i is out of range). */
int32_t lbm_batch_instance_kernel(const lbm_batch* b, int32_t i);

/* Autotuner of the batch's kernels (no counterpart in the paper).  Groups the instances by size
 * class (floor(log2(nodes))) and, for each class, times every candidate on the class's own
 * instances from their current state: the pair kernel (FP32) with 4, 3 and 2 resident CTAs per
 * SM, the tile kernel and the y-march, 2 warm-up steps then trial_steps (>= 2, rounded up to even)
 * steps between CUDA events.  The state is saved before and restored after the trials, so the
 * simulation is unchanged.  Each class then steps with its fastest candidate when that is more
 * than 3 % faster than the first candidate (the kernel the batch runs untuned), else with the first:
 * instances of different choices form groups whose kernels run as parallel branches of the
 * captured steps, and a group of its own costs more than a near-tie gains.
 * The choices are kept per (device, lattice, precision, size class) for the process: a later
 * lbm_batch_init with LBM_KERNEL_AUTO uses them.  Synchronises the batch's stream.  Errors:
 * LBM_ERR_ARG (trial_steps < 2), LBM_ERR_CUDA, LBM_ERR_OOM. */
lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps);
/* Set the step kernel of every instance (kinds: n entries of LBM_KERNEL_TILE, LBM_KERNEL_YMARCH
 * or LBM_KERNEL_PAIR, the latter FP32 only), overriding lbm_batch_init's and the autotuner's
 * choice; instances of different kernels step as parallel groups.  Errors: LBM_ERR_ARG. */
lbm_status lbm_batch_set_kernels(lbm_batch* b, const int32_t* kinds);
/* Forget the choices lbm_batch_autotune made for this process (later batches use their defaults). */
void lbm_batch_autotune_forget(void);
/* Text report of the last lbm_batch_autotune (one line per class and candidate with its time and
 * rate, then the choice per class); owned by the batch, "" before any. */
const char* lbm_batch_tuning_report(const lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

void lbm_destroy(lbm_handle* h);

/* Message of the last failing call on h (or of the last failing lbm_init when h is NULL). */
const char* lbm_last_error(const lbm_handle* h);

const char* lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif /* LBMWET_H */
