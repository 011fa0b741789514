/*
 * sesc.h - C ABI of the GB300 implementation of the multi-level blended DG/FV
 * right-hand side for the compressible Euler equations (Markert, Gassner &
 * Walch, "A Sub-Element Adaptive Shock Capturing Approach for Discontinuous
 * Galerkin Methods", arXiv 2011.03338).
 *
 * Data layout (all entry points):
 *   state u[e][v][t], FP64, element-major: element e = ex + nx*(ey + ny*ez),
 *   variable v = 0..d+1 (rho, rho v_1..rho v_d, E), subcell t = ix + M*(iy + M*iz)
 *   (x fastest). Each value is the mean of the conserved variable over one of the
 *   M^d uniform subcells of the element (Sec. 2, eq. subcell-grid; appendix 3D
 *   extension: the element holds N^3 mean values).
 *   Coefficients c[e][2][S]: c[e][0][:] blending factors alpha, c[e][1][:]
 *   squeezing parameters beta, for levels n = M, M/2, ..., 2 (in that order),
 *   (M/n)^d sub-elements per level with x fastest; S = sum_n (M/n)^d
 *   (sesc_num_coeffs).
 *
 * Pointers: every array argument is DEVICE memory of the handle's device unless
 * stated otherwise. The caller owns all arrays it passes; the handle owns its
 * workspace. Calls are asynchronous on the given CUDA stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream). A handle is not thread-safe;
 * use it from one host thread and one stream at a time.
 *
 * Errors: argument errors are returned synchronously (SESC_EINVAL). Conditions
 * found on the device (a non-permissible mean value, a non-finite wave speed)
 * are recorded in the handle's status word and returned by sesc_status.
 */
#ifndef SESC_H_
#define SESC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sesc_handle sesc_handle;

enum {
  SESC_OK = 0,
  SESC_EINVAL = 1,            /* bad argument or configuration */
  SESC_ENOMEM = 2,            /* device allocation failed */
  SESC_ECUDA = 3,             /* a CUDA call or launch failed */
  SESC_ENONPERMISSIBLE = 4,   /* a mean value had rho <= 0 or p <= 0 (Sec. 3.1 permissible set) */
  SESC_ENONFINITE = 5,        /* a non-finite wave speed in the time-step reduction */
  SESC_ETOOLARGE = 6,         /* the problem does not fit the static scratch of sesc_rhs_static */
  SESC_ETIMEOUT = 7,          /* a bounded device-side wait gave up (a grid-wide barrier of a persistent
                                 batched launch, or an element's staging copy): output invalid */
  SESC_EBOUNDS = 8            /* bounds-checked build (libsesc_bounds.so) only: a computed index fell
                                 outside its buffer; it was replaced by 0 and the output is invalid */
};

enum { SESC_BC_PERIODIC = 0, SESC_BC_WALL = 1, SESC_BC_OUTFLOW = 2, SESC_BC_HALO = 3 };
enum { SESC_NODES_GAUSS = 0, SESC_NODES_LOBATTO = 1 };
enum { SESC_FP64 = 0, SESC_FP32_SPLIT = 1 };
enum { SESC_SCHEME_MULTI_LEVEL = 0, SESC_SCHEME_SINGLE_LEVEL = 1 };

/* Problem description. dim in {2, 3}; M (mean values per direction per element,
 * the paper's N, a power of two) in {4, 8}; nel[a] elements along direction a;
 * the box [xlo, xhi]; bc[2a], bc[2a+1] the low / high boundary of direction a
 * (periodic must be set on both sides; SESC_BC_HALO marks a side shared with
 * another part of a partitioned mesh, see sesc_pack_halo). gamma: ratio of specific heats
 * (eq. equation-of-state). tauA, tauS: indicator amplification / sensitivity
 * (eq. calc-blending-factor; paper: 100, 0.05). alphaH, alphaL, betaL: switching
 * thresholds (appendix, sketch of the multi-level algorithm; paper: 0.99, 0.01, 0.95;
 * 0 <= alphaL < alphaH <= 1, 0 <= betaL <= 1). cfl: CFL number of
 * eq. cfl-condition. node_family: collocation nodes (paper: Gauss-Legendre).
 * precision: SESC_FP64 (every operation in double precision) or SESC_FP32_SPLIT
 * (reconstruction, fluxes and operator passes in FP32 accumulated in FP32; the
 * indicator ratio, the squeezing formula, the permissibility checks of face
 * states, the conservative flux-difference assembly and the RK stage in FP64;
 * the state stays FP64). sesc_rhs_static supports SESC_FP64 only.
 * scheme: SESC_SCHEME_MULTI_LEVEL (the hierarchy FV, 2, 4, ..., M of Sec. 2.6) or
 * SESC_SCHEME_SINGLE_LEVEL (the single-level DG/FV blend of Sec. 2.5 and its 3D form
 * eq. dgfv-scheme-3d: one blending factor per element from eq. calc-blending-factor
 * at level M, intermediate levels off, inner subcell interfaces with the flux of the
 * raw subcell means, element faces with the blended states of eq. 3D-prolongation
 * and the flux blend of eq. 3D-blend-interface-fluxes). The adjoint entry points
 * support the multi-level scheme only. elem_size[a]: the element edge along a when
 * > 0 (a part of a partitioned mesh takes the whole mesh's, so that its factors
 * M / dx match to the last bit), else (xhi[a] - xlo[a]) / nel[a]. */
typedef struct {
  int32_t dim;
  int32_t M;
  int32_t nel[3];
  double xlo[3];
  double xhi[3];
  int32_t bc[6];
  double gamma, tauA, tauS, alphaH, alphaL, betaL, cfl;
  int32_t node_family;
  int32_t precision;
  int32_t scheme;
  double elem_size[3];
} sesc_config;

/* Create a handle on the current CUDA device: validates cfg, builds the level
 * operators (Sec. 2.2-2.5) and allocates the workspace (face states, interface
 * fluxes, coefficients, two RK stage buffers). Returns SESC_OK and *out, or an
 * error code with *out = NULL. */
int sesc_create(const sesc_config* cfg, sesc_handle** out);

/* Release the handle and its workspace (synchronises the device). NULL is a no-op. */
void sesc_destroy(sesc_handle* h);

/* Number of elements E and coefficients per element S of the handle. */
int64_t sesc_num_elements(const sesc_handle* h);
int64_t sesc_num_coeffs(const sesc_handle* h);

/* Blending indicator (Sec. 2.7 eq. calc-blending-factor, Sec. 2.4 eq.
 * calc-squeezing-parameter, and the multi-level loop of the appendix sketch,
 * steps I-II) for state u. Outputs (each nullable):
 *   coeffs   [E][2][S] snapped alpha and beta (levels never reached: alpha 0, beta 1)
 *   theta    [E][L][M^d] blending weights per subcell (eq. blending-weights), L =
 *            log2(M)+1 levels in the order 1, 2, 4, ..., M
 *   decision [E] byte: low nibble log2(n_min), high nibble log2(n_max), the
 *            lowest / highest level with a nonzero weight in the element
 *   abar     [E][M^d] weighted blending factor sum_n n theta^(n) (eq. order-estimate) */
int sesc_indicator(sesc_handle* h, const double* u, double* coeffs, double* theta,
                   uint8_t* decision, double* abar, void* stream);

/* Right-hand side dudt = R(u) of the multi-level blended scheme (Sec. 2.6 eqs.
 * multilevel-blending-scheme / multilevel-blending-discretizations, appendix
 * eq. dgfv-scheme-3d with the blended common interface fluxes). frozen:
 * nullable [E][2][S] coefficients to use instead of the indicator (alpha is used
 * as given, already snapped). coeffs_out: nullable [E][2][S] copy of the
 * coefficients used. dudt must not alias u. */
int sesc_rhs(sesc_handle* h, const double* u, double* dudt, const double* frozen,
             double* coeffs_out, void* stream);

/* One SSP-RK stage: uout = a*u0 + b*(us + dt*R(us)) (Shu-Osher form; SSP-RK3 uses
 * (a, b) = (0,1), (3/4,1/4), (1/3,2/3)). The time step is read from dt_dev
 * (device, one double) when it is not NULL, else `dt` is used. frozen: nullable
 * [E][2][S] coefficients used instead of the indicator (as in sesc_rhs);
 * coeffs_out: nullable [E][2][S] copy of the coefficients used. uout may alias
 * u0 but not us. */
int sesc_rk_stage(sesc_handle* h, const double* u0, const double* us, double* uout,
                  double a, double b, double dt, const double* dt_dev, const double* frozen,
                  double* coeffs_out, void* stream);

/* Adjoint (vector-Jacobian product) of the right-hand side with the blending
 * coefficients held fixed: u_bar = (dR/du)^T dudt_bar at state u. frozen: nullable
 * [E][2][S] coefficients; when NULL the indicator's coefficients at u are used and
 * held fixed. R is then a composition of linear maps and pointwise Euler / HLL
 * fluxes (Sec. 2.2-2.6); the Jacobians of the pointwise maps follow the branches
 * taken at u. Every adjoint value is summed in a fixed order (the result is the
 * same bit for bit from run to run). In a SESC_FP32_SPLIT handle the adjoint runs
 * in the same precision split as the forward: transposed operator passes and
 * Jacobians in FP32, the transposed flux differences with their blending weights
 * and the stage combination in FP64. Multi-level scheme only. u_bar must not alias
 * the inputs. */
int sesc_rhs_vjp(sesc_handle* h, const double* u, const double* frozen, const double* dudt_bar,
                 double* u_bar, void* stream);

/* Adjoint of one stage uout = a*u0 + b*(us + dt*R(us)) with fixed coefficients
 * (frozen, nullable as above) and fixed dt (dt_dev, if not NULL, is read once
 * with a synchronisation): us_bar = b*uout_bar + b*dt*(dR/dus)^T uout_bar
 * (overwritten); u0_bar += a*uout_bar when u0_bar is not NULL. Precision as
 * sesc_rhs_vjp. */
int sesc_rk_stage_vjp(sesc_handle* h, const double* us, const double* frozen, const double* uout_bar,
                      double a, double b, double dt, const double* dt_dev, double* us_bar,
                      double* u0_bar, void* stream);

/* Time step of eq. cfl-condition with the wave-speed estimate of eq.
 * euler-max-eigenvalue over all mean values: writes one double to dt_dev. */
int sesc_dt(sesc_handle* h, const double* u, double* dt_dev, void* stream);

/* One SSP-RK3 step: dt (written to dt_dev if not NULL) and three stages, with
 * the two stage buffers of the workspace. uout may alias u. */
int sesc_rk3_step(sesc_handle* h, const double* u, double* uout, double* dt_dev, void* stream);

/* Generalised stage uout = a*u0 + c*u2 + b*(us + g*dt*R(us)) (Shu-Osher form with a
 * second earlier state, for integrators such as SSP-RK(5,4)); dt from dt_dev when it
 * is not NULL. u0 / u2 may be NULL when a / c is 0. uout must not alias us. */
int sesc_rk_stage_ex(sesc_handle* h, const double* u0, double a, const double* u2, double c,
                     const double* us, double b, double g, double dt, const double* dt_dev,
                     double* uout, void* stream);

/* One step of the five-stage, fourth-order SSP Runge-Kutta method the paper
 * integrates with (SSP-RK(5,4), Spiteri & Ruuth), with the time step of eq.
 * cfl-condition (written to dt_dev if not NULL) and four stage buffers of the
 * workspace (two allocated by the first call). uout may alias u. */
int sesc_ssprk54_step(sesc_handle* h, const double* u, double* uout, double* dt_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Partitioned meshes. A mesh split into blocks of elements (one handle per block,
 * on one or several GPUs) exchanges, per RK stage, only what the paper's parallel
 * form exchanges between processes (appendix: 3D extension and multi-level
 * sketch, step IV): the face-centred mean values and level weights of the element
 * faces on the shared sides. A shared side has bc = SESC_BC_HALO. One stage of a
 * part then runs as: sesc_indicator(h, us, ...) (K1: coefficients and element-face
 * states); sesc_pack_halo for each halo side, the packed buffers sent to the
 * neighbours; sesc_set_halo for each halo side with the neighbour's packed buffer
 * of the opposite side; sesc_stage_finish (interface fluxes and update). Both parts
 * compute the flux of a shared face from the same two states, so the result equals
 * the unpartitioned mesh's bit for bit; the time step is the minimum of the parts'
 * sesc_dt. The adjoint, batch and allocation-free entry points reject halo sides.
 * ------------------------------------------------------------------------- */

/* Bytes of the packed face states of side `side` (2a + 0 low, 2a + 1 high side of
 * direction a): one row per element of that boundary layer, in transverse order,
 * each (d + 2 + L) x M^(d-1) values of the handle's compute type (FP64, or FP32 for
 * SESC_FP32_SPLIT). -1 for a bad side. */
int64_t sesc_halo_bytes(const sesc_handle* h, int side);

/* Pack the element-face states of side `side` left by the last sesc_indicator (or
 * RHS / stage call) into dst (device, sesc_halo_bytes bytes). Asynchronous. */
int sesc_pack_halo(sesc_handle* h, int side, void* dst, void* stream);

/* Use src (device, sesc_halo_bytes(h, side) bytes, the neighbour's packed states of
 * its opposite side, same transverse extent) as the ghost states of halo side
 * `side` in later flux evaluations. The pointer is kept (not copied): its contents
 * must be in place when the next sesc_stage_finish runs on the stream. */
int sesc_set_halo(sesc_handle* h, int side, const void* src);

/* Interface fluxes and update from the coefficients and face states of the last
 * sesc_indicator(h, us, ...): mode 0: out = R(us); mode 1: out = a*u0 + b*(us +
 * dt*R(us)) (dt from dt_dev when not NULL). Every halo side needs a halo set.
 * out must not alias us. */
int sesc_stage_finish(sesc_handle* h, const double* u0, const double* us, double* out, double a,
                      double b, double dt, const double* dt_dev, int mode, void* stream);

/* Synchronises the handle's device, copies 16 counters to host memory
 * `counters` (nullable) and returns the first device-side error recorded since
 * the last sesc_reset_status (SESC_OK if none). counters: [0] error bits
 * (1 non-permissible mean, 2 non-finite wave speed, 4 a timed-out wait: a grid
 * barrier of a batch, or the bulk copy that stages an element's means in shared
 * memory, whose element was then skipped; SESC_ETIMEOUT is returned; 8 an index
 * outside its buffer, bounds-checked build only: SESC_EBOUNDS), [1] squeezed
 * sub-elements (beta < 1), [2] DG face candidates replaced by the FV candidate, [3]
 * threshold-near elements (a raw blending factor within 1e-10 of alpha_H or
 * alpha_L, or a squeezing parameter within 1e-10 of beta_L: their level decisions
 * hang on the last bits), [4 + k] elements with n_min = 2^k, [8 + k] elements with
 * n_max = 2^k, [12] elements whose levels the certified FP32 pass of an FP64
 * handle's indicator decided (sesc_set_indicator_filter); summed over the indicator
 * evaluations since the reset. */
int sesc_status(sesc_handle* h, int64_t* counters);
int sesc_reset_status(sesc_handle* h, void* stream);

/* Bound of the wait for the bulk copy that stages an element's means in shared
 * memory (polls of its mbarrier, each a hardware-bounded try-wait). A kernel that
 * gives up records flag 4 of counters[0] and skips the element (sesc_status returns
 * SESC_ETIMEOUT; the output is invalid); the copy still gets a second bounded wait
 * to land first. Default 2^22. 0 makes every staged element give up (a test of
 * the error path). Returns SESC_EINVAL for polls < 0. */
int sesc_set_stage_cap(sesc_handle* h, int64_t polls);

/* Certified FP32 pass of the indicator of an FP64 handle (on by default; ignored by
 * FP32-split handles). The smoothness statistics of eq. L1-norm-slope enter the
 * blending factor of eq. calc-blending-factor only through a ratio that gives exactly
 * 1 or 0 outside the transition band [tau_S, tau_S + 1/tau_A]. The pass computes
 * them in FP32 with a forward error bound against the exact values from the FP64
 * means and decides a factor only where the bounded ratio lies outside the band; an
 * element with a factor left open, or with a level to squeeze, is evaluated in FP64
 * from the start. The coefficients, decisions and right-hand sides are therefore
 * the same bits with the pass on or off (on = 1, off = 0); counters[12] of
 * sesc_status counts the elements it decided. Returns SESC_EINVAL for h == NULL. */
int sesc_set_indicator_filter(sesc_handle* h, int on);

/* Element classes of the multi-level sketch (appendix; the paper's per-element level
 * bounds n_min / n_max skip levels with zero weight): synchronises the device and
 * writes counts[m], m = 0..15, the number of elements, summed over every indicator
 * evaluation since the last sesc_reset_status, whose set of levels carrying weight
 * is m (bit l set: level n = 2^l has a nonzero blending weight at some subcell of the
 * element; bit 0 the FV level). The work of the update kernel depends on that set;
 * the measurement weighs its operation counts with these. */
int sesc_level_counts(sesc_handle* h, int64_t* counts);

/* Kernel timing, for measurement. Kinds of kernel launches: */
enum {
  SESC_KERNEL_INDICATOR = 0,   /* K1: indicator, coefficients, element face states */
  SESC_KERNEL_FACE_FLUX = 1,   /* K2: interface fluxes at element faces (all directions) */
  SESC_KERNEL_UPDATE = 2,      /* K3: level right-hand sides, blend, RK stage */
  SESC_KERNEL_DT = 3,          /* time-step reduction */
  SESC_NUM_KERNEL_KINDS = 4
};

/* enable != 0: every later launch group of the handle is bracketed by a pair of
 * CUDA events on its stream (small overhead). sesc_kernel_times synchronises the
 * device, writes the summed device time in milliseconds (ms[kind]) and the
 * number of bracketed launch groups (launches[kind]) of each kind since the last
 * read, and releases the events. Both arrays have SESC_NUM_KERNEL_KINDS entries;
 * a face-flux group is one launch per direction. */
int sesc_set_timing(sesc_handle* h, int enable);
int sesc_kernel_times(sesc_handle* h, double* ms, int64_t* launches);

/* Allocation-free right-hand side (the paper has no counterpart; this is a
 * service of the library). Some callers cannot have a library allocate device
 * memory: programs that give out a fixed device-memory budget up front and
 * forbid allocations behind their back (a host simulation code, a plugin inside
 * another application), and callers on a time-critical path, where cudaMalloc
 * or cudaFree can synchronise the device and stall other streams. For them,
 * sesc_rhs_static computes the same dudt = R(u) as sesc_rhs (same kernels) for the
 * problem `cfg`, without a handle and without calling cudaMalloc, cudaFree or any
 * allocating routine: its scratch lives in one device array of
 * SESC_STATIC_SCRATCH_BYTES that every GPU which loads the library holds until the
 * process exits. The caller passes u and dudt (device, layout as above).
 * - Sizes: the face states, interface fluxes and coefficients must fit that array
 *   (about 2.9 KB per element in 2D with M = 8, i.e. up to about 11,000 elements,
 *   and 36.5 KB per element in 3D with M = 8, up to about 900 elements); larger
 *   problems return SESC_ETOOLARGE and nothing runs.
 * - The first call on a device sets up that device (looks up the array's device
 *   address, uploads the operator tables); make that first call before any CUDA
 *   stream capture. Host threads may make first calls concurrently: the set-up
 *   is serialised by a lock.
 * - Every call on a device uses the same array, which keeps the previous call's
 *   contents; calls whose kernels overlap on the GPU (other streams, other host
 *   threads) race on it. Serialise them.
 * - Device-side conditions (non-permissible means) are not reported; use a
 *   handle and sesc_status for that. */
#define SESC_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int sesc_rhs_static(const sesc_config* cfg, const double* u, double* dudt, void* stream);

/* ---------------------------------------------------------------------------
 * Batched ensembles of independent problems (the paper runs one problem at a
 * time; this is a service of the library for parameter studies and ensembles).
 * A batch holds nproblems configurations of any sizes, dimensions, M, node
 * families and precisions; their states are concatenated in one device array,
 * problem k at offsets[k] .. offsets[k+1]-1 (doubles, layout of each problem as
 * above, offsets from sesc_batch_offsets). Problems with equal (dim, M,
 * precision) form a group. A stage of a group is one persistent launch: the
 * indicator (K1) over all elements of the group's problems, a grid-wide barrier,
 * the interface fluxes (K2) over all their faces, a barrier, the update (K3); or,
 * per group as the autotuner or sesc_batch_set_fused chooses, three persistent
 * launches, one per phase. The wave speeds of the time step are one more launch
 * pair. Groups run on concurrent stream branches. Each problem keeps its own time step (eq.
 * cfl-condition over its own means), so every problem follows exactly the
 * arithmetic of a handle for that configuration. A batch is single-stream and not
 * thread-safe, like a handle.
 * ------------------------------------------------------------------------- */
typedef struct sesc_batch sesc_batch;

/* Kernel kinds of a batch group (index into the grid arrays below). */
enum {
  SESC_BATCH_KERNEL_INDICATOR = 0,
  SESC_BATCH_KERNEL_FACE_FLUX = 1,
  SESC_BATCH_KERNEL_UPDATE = 2,
  SESC_BATCH_KERNEL_DT = 3,
  SESC_BATCH_NUM_KERNEL_KINDS = 4
};

/* Create a batch on the current device: validates every configuration (as
 * sesc_create), allocates the workspace, the two stage buffers and the device
 * tables, uploads the operator tables, and sets every kernel's grid to all CTAs
 * resident (capped at its work items). Returns SESC_OK and *out, or an error code
 * with *out = NULL. Synchronises the device. */
int sesc_batch_create(const sesc_config* cfgs, int nproblems, sesc_batch** out);
/* Release the batch (synchronises the device). NULL is a no-op. */
void sesc_batch_destroy(sesc_batch* b);
/* offsets[nproblems + 1]: start of every problem in the concatenated state, in doubles. */
int sesc_batch_offsets(const sesc_batch* b, int64_t* offsets);
/* Number of groups, and the group of problem k (-1 if out of range). */
int sesc_batch_num_groups(const sesc_batch* b);
int sesc_batch_group_of(const sesc_batch* b, int k);

/* dudt = R(u) for every problem (as sesc_rhs with frozen = NULL). dudt must not alias u. */
int sesc_batch_rhs(sesc_batch* b, const double* u, double* dudt, void* stream);
/* Per-problem time steps; dt_dev (nullable) receives nproblems doubles. */
int sesc_batch_dt(sesc_batch* b, const double* u, double* dt_dev, void* stream);
/* One SSP-RK3 step of every problem with its own time step (as sesc_rk3_step);
 * dt_dev (nullable) receives the nproblems time steps. uout must not alias u.
 * With the graph mode on, the first call for a given (u, uout, dt_dev) captures
 * the whole step (memset, wave speeds, 3 x 3 phases per group, group branches)
 * into a CUDA graph on an internal stream and later calls with the same pointers
 * replay it on `stream`; other pointers capture anew. */
int sesc_batch_rk3_step(sesc_batch* b, const double* u, double* uout, double* dt_dev, void* stream);
/* enable != 0: turn the graph mode on; 0: off (drops the captured graph). */
int sesc_batch_use_graph(sesc_batch* b, int enable);

/* Grid sizes, [groups][SESC_BATCH_NUM_KERNEL_KINDS]: each CTA of a persistent
 * launch walks items (elements, face tasks or wave-speed tiles) with a stride of
 * the grid size, so the grid sets how many elements a CTA handles. set_grids
 * rejects values < 1 and drops a captured graph. */
int sesc_batch_grids(const sesc_batch* b, int32_t* grids);
int sesc_batch_set_grids(sesc_batch* b, const int32_t* grids);
/* Autotuner: runs one eager stage of state u, then for every group and kernel
 * kind times `reps` launches at each candidate grid (multiples of the SM count up
 * to all CTAs resident, and one CTA per item) and keeps the fastest; then times a
 * whole stage as one persistent launch at grids of 1, 2, 4 ... x the SM count up to
 * all CTAs resident against the three separate launches, and keeps the fastest
 * mode (the grid sets how many elements, faces and wave-speed tiles each CTA
 * walks). Blocking; drops a captured graph and clears the status counters. */
int sesc_batch_autotune(sesc_batch* b, const double* u, int reps, void* stream);

/* Stage mode per group: fused_grid[g] = the grid of the one-launch stage (all its
 * CTAs resident, a cooperative launch), or 0 when group g runs the three phases as
 * separate launches. set_fused rejects a grid above all CTAs resident and drops a
 * captured graph. */
int sesc_batch_fused(const sesc_batch* b, int32_t* fused_grid);
int sesc_batch_set_fused(sesc_batch* b, const int32_t* fused_grid);
/* Polls (128 ns apart) a CTA of the one-launch stage waits at a grid-wide barrier
 * before it gives up: the stage then ends early and sesc_batch_status reports
 * SESC_ETIMEOUT (its output is invalid). Default 2^24 (about 2 s). */
int sesc_batch_set_barrier_cap(sesc_batch* b, int64_t polls);

/* As sesc_status / sesc_reset_status for every problem: counters receives
 * [nproblems][16] (nullable); the return value reports the first error bit set
 * in any problem. */
int sesc_batch_status(sesc_batch* b, int64_t* counters);
int sesc_batch_reset_status(sesc_batch* b, void* stream);

/* Static description of an error code. */
const char* sesc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SESC_H_ */
