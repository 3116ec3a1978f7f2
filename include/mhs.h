/*
 * mhs.h -- C ABI of libmhs, a single-GPU (GB300, sm_103a) multigrid solver
 * for linear magnetohydrostatic (MHS) equilibria in the poloidal/toroidal
 * representation used by MacTaggart, Elsheikh, McLaughlin & Simitev,
 * "Non-symmetric magnetohydrostatic equilibria: a multigrid approach".
 *
 * The method (Sect. 2):
 *   1. P = 0 everywhere (Sect. 2.2, step 1);
 *   2. multigrid solve of eq. (lower_bound), P_xx + P_yy = -B_z on z = 0 with
 *      P = 0 on the edges of that plane (Sect. 2.2, step 2);
 *   3. multigrid solve of eq. (scalar_pot),
 *      [1 - xi(z)](P_xx + P_yy) + P_zz + alpha^2 P = 0, in the interior with
 *      P from step 2 on z = 0 and P = 0 on the top and side faces
 *      (Sect. 2.2, step 3; elliptic for xi < 1, Sect. 2.1);
 *   4. B = curl[curl(P e_z) + alpha P e_z] (eqs. b_iden, t):
 *      B_x = alpha P_y + P_xz, B_y = -alpha P_x + P_yz, B_z = -(P_xx + P_yy),
 *      by second-order finite differences (Sect. 2.2);
 *   5. p = p_b(z) - xi B_z^2/(2 mu0)                         (eq. pressure)
 *      rho = rho_b(z) + [xi' B_z^2/(2 mu0) + xi B.grad(B_z)/mu0]/g  (eq. density)
 *      with the background atmosphere of Sect. 3.
 *
 * Grid: nx*ny*nz vertex-centred nodes on [0,Lx] x [0,Ly] x [0,Lz] (z = 0 is
 * the photosphere), node (i,j,k) at (i Lx/(nx-1), j Ly/(ny-1), k Lz/(nz-1)).
 * Every array crossing this interface is a dense double array in
 * [nz][ny][nx] order (x fastest): element (i,j,k) at i + nx*(j + ny*k);
 * 2D arrays are [ny][nx].  A pointer may be a host pointer (pageable or
 * pinned) or a CUDA device pointer; the library detects which.  The caller
 * owns every buffer it passes; the library copies in and out and keeps no
 * pointer after the call returns.
 *
 * Errors: every call returns an mhs_status; no C++ exception crosses the
 * interface; a failed call leaves the handle usable (except after
 * MHS_ERR_CUDA caused by a sticky device fault).  mhs_last_error() returns a
 * thread-local message describing the last failure on the calling thread.
 *
 * Streams: all device work of a handle is ordered on its stream (default:
 * the legacy default stream).  Calls that return results to host memory
 * synchronise that stream before they return.  A handle must not be used by
 * two threads at once.
 */
#ifndef MHS_H
#define MHS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MHS_API __attribute__((visibility("default")))
#else
#define MHS_API
#endif

typedef struct mhs_ctx* mhs_handle;

typedef enum {
    MHS_OK = 0,
    MHS_ERR_INVALID_ARG = 1,     /* a size, length, pointer or option is out of range */
    MHS_ERR_NOT_ELLIPTIC = 2,    /* xi(z_k) >= 1 on an interior plane (Sect. 2.1), or alpha^2 not below
                                    the smallest eigenvalue bound of the discrete operator */
    MHS_ERR_OUT_OF_MEMORY = 3,   /* device or host allocation failed */
    MHS_ERR_CUDA = 4,            /* a CUDA runtime call failed; see mhs_last_error() */
    MHS_ERR_NO_CONVERGENCE = 5,  /* the residual did not reach the tolerance within the cycle limit */
    MHS_ERR_NONFINITE = 6,       /* B_z holds NaN/Inf, or a residual norm became non-finite */
    MHS_ERR_BAD_STATE = 7,       /* call order violated (solve before set_lower_bz, fields before solve) */
    MHS_ERR_TIMEOUT = 8,         /* a bounded wait expired */
    MHS_ERR_REJECTED = 9         /* a request exceeds the server's device-memory budget */
} mhs_status;

/* Height profile xi(z) of the cross-field current, F = xi(z) B_z / g
 * (Sect. 2.1, after eq. helm).  The families are those of Sect. 3.2. */
typedef enum {
    MHS_XI_NONE = 0,     /* xi = 0: linear force-free field (Sect. 3.1) */
    MHS_XI_EXP = 1,      /* xi = a exp(-kappa z)                 (xi_1 family) */
    MHS_XI_EXP_SIN = 2   /* xi = (a + b sin(omega z)) exp(-kappa z) (xi_2 family) */
} mhs_xi_kind;

typedef struct {
    int kind;            /* mhs_xi_kind */
    double a, kappa, b, omega;
} mhs_xi_params;

/* Background atmosphere (Sect. 3): T_b = 1 for z <= z1,
 * T_cor^((z - z1)/(z2 - z1)) for z1 < z <= z2, T_cor above; p_b = rho_b T_b;
 * dp_b/dz = -g p_b / T_b with p_b(0) = 1.  mu0 is the permeability in code
 * units (1/2 when B is measured in B0 = (2 mu0 p0)^(1/2) and p in p0). */
typedef struct {
    double g, mu0, T_cor, z1, z2;
} mhs_atmos_params;

typedef enum {
    MHS_FP64 = 0,        /* every multigrid operation in FP64 */
    MHS_MIXED = 1        /* FP32 V-cycles inside a defect-correction loop whose iterate and residual are
                            double-float (pairs of FP32 words, about 48 bits); P returned in FP64 */
} mhs_precision;

/* Solver options.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
    int nu1;             /* pre-smoothing red-black sweeps per level [2] */
    int nu2;             /* post-smoothing sweeps [2] */
    int max_cycles;      /* V-cycles (FP64 mode) or outer steps (mixed mode) per solve [100] */
    int inner_cycles;    /* FP32 V-cycles per outer step in mixed mode [1] */
    int flags;           /* MHS_FLAG_* bits */
    int cut64;           /* FP64: largest interior node count of a level solved, with all coarser levels, by
                            the one-CTA shared-memory sub-cycle [1200] */
    int cut32;           /* same for FP32 levels [4000] */
    int fused_min;       /* FP32 3D levels with at least this many interior nodes use the fused, TMA-staged
                            red-black sweep (one pass per sweep, HBM-bound); smaller, cache-resident levels use the
                            two colour passes, which have less latency [12000000] */
    int sep_coarse;      /* coarse-grid solve of the V-cycles: the first level below the finest with at most this
                            many interior nodes, whose sine transforms are fast (nx - 1 and ny - 1 powers of two)
                            or short (nx, ny <= 66), is solved exactly by the separable solver (sine transforms
                            in x and y, one tridiagonal system along z per mode) in the cycle's precision, and
                            the levels below it are never visited; the one-CTA sub-cycle handles the coarse end
                            when no level qualifies or when the sub-cycle cut-off lies above it.  -1: never
                            [300000] */
    int tile;            /* thread-block shape of the red-black point passes (threads along x, each owning an
                            x pair of nodes, x rows): 1 = 32 x 8, 2 = 64 x 4, 3 = 16 x 16, 4 = 32 x 16,
                            5 = 128 x 2 (results do not depend on it) [1] */
    int tma_rows;        /* rows of the tiles of the fused, TMA-staged FP32 sweep: 8 (64 x 8 tiles, 256 threads)
                            or 16 (64 x 16, 512 threads, fewer halo updates per node); results do not depend on
                            it [8] */
} mhs_solver_opts;

#define MHS_FLAG_WARM 1         /* start the interior solve from the resident P instead of P = 0 */
#define MHS_FLAG_BZ_MIMETIC 2   /* B_z = -(D_x D_x + D_y D_y) P with the first-difference operators,
                                   which makes the central-difference div B vanish to rounding */
#define MHS_FLAG_FUSED_SWEEP64 8 /* FP64 3D levels also use the fused out-of-place red-black sweep (one pass per
                                    sweep; FP32 levels do from fused_min interior nodes up); default: the two
                                    in-place colour passes, which spend no FP64 work on redundant halo updates */
#define MHS_FLAG_NO_FMG 32      /* start from P = 0 with plain V-cycles instead of a full-multigrid first cycle */
#define MHS_FLAG_ZLINE 64       /* smooth the interior levels by zebra z-line Gauss-Seidel (columns with i + j
                                   even, then odd, each solved exactly along z) instead of red-black point
                                   Gauss-Seidel: robust when 1 - xi(z) is small or h_z < h_x; same solution.
                                   Without this flag or MHS_FLAG_POINT the smoother is chosen from the problem:
                                   z-line when the anisotropy class (see mhs_autotune) is 5 or more */
#define MHS_FLAG_POINT 128      /* always smooth by red-black point Gauss-Seidel */
#define MHS_FLAG_SEPARABLE 256  /* solve the correction equation of each step with the exact separable solver
                                   (sine transforms in x and y, one tridiagonal system along z per mode; valid
                                   because xi depends on z only and the sides are Dirichlet) instead of a
                                   V-cycle; same discrete solution.  Mixed mode: FP32 solves inside the
                                   double-float loop, 2-3 steps.  FP64 mode: FP64 direct solves, 1-2 steps,
                                   when nx - 1 and ny - 1 are powers of two or nx, ny <= 66 (else V-cycles).
                                   Not in groups */
#define MHS_FLAG_LOWER_FP64 512 /* mixed mode: solve the lower-boundary problem (eq. lower_bound) by FP64 V-cycles,
                                   as in FP64 mode, instead of FP32 cycles in a double-float defect correction
                                   loop; the interior problem keeps the mixed-precision loop.  The double-float
                                   iterate (48-bit significand) bounds the relative residual of the
                                   lower-boundary problem near 5e-12 on 257^2 and 2e-11 on 513^2 nodes (the
                                   interior problem's, whose right-hand side is smoother, near 1e-13 and 8e-13);
                                   with this flag a mixed solve reaches 1e-12 on 257^3 and 2e-12 on 513 x 513 x 257
                                   nodes.  The lower boundary is a small part of the work (1 / nz of the
                                   unknowns).  Not in groups */
#define MHS_FLAG_NO_TMA 16      /* FP32 levels sweep with plain global loads instead of TMA-staged planes (same
                                   results; for comparison) */
#define MHS_FLAG_STAGED_TRANSFORMS 1024 /* separable solves of a level (the exact coarse-grid solves, MHS_OP_EXACT)
                                   launch one kernel per sine-transform pass instead of the per-plane kernels
                                   on thread-block clusters (same results bit for bit; for comparison) */
#define MHS_FLAG_NO_GRAPH 4     /* launch the solve kernel by kernel with host-side convergence checks instead of
                                   one captured CUDA graph (same kernels, same results; for profilers that cannot
                                   see kernels inside conditional graph nodes) */

typedef struct {
    int cycles_2d;       /* iterations of the lower-boundary solve: FP64 V-cycles (or separable direct steps)
                            when it runs in FP64, defect-correction steps in mixed mode */
    int cycles_3d;       /* the same for the interior solve */
    double rel_res_2d;   /* final ||b - A P||_2 / ||b||_2 of eq. (lower_bound) */
    double rel_res_3d;   /* same for eq. (scalar_pot), b = right-hand side after lifting the z = 0 data */
    double conv_factor;  /* geometric-mean residual reduction per interior cycle */
    double ms;           /* device time of the solve (CUDA events on the handle's stream) */
    int outer_iters_2d;  /* outer defect-correction steps of the lower-boundary solve (each: double-float
                            residual, inner_cycles FP32 V-cycles or one FP32 separable solve, correction);
                            0 when that problem runs in FP64 cycles (FP64 mode, MHS_FLAG_LOWER_FP64) */
    int outer_iters_3d;  /* the same for the interior solve (0 in FP64 mode) */
} mhs_solve_info;

/* Create a solver for an nx*ny*nz node grid on [0,Lx]x[0,Ly]x[0,Lz].
 * Each n must be odd, >= 5 and <= 16385 (nx, ny <= 4097); multigrid coarsens all three axes together
 * while every axis stays odd and >= 3 nodes, so n = 2^k m + 1 with small m
 * gives the deepest hierarchy.  Lengths must be > 0; xi == NULL means
 * xi = 0; atm == NULL means g = 1, mu0 = 1/2, T_cor = 150, z1 = 5, z2 = 10.
 * Allocates the whole device hierarchy (owned by the handle) and computes
 * the per-plane coefficients on the device.
 * Errors: MHS_ERR_INVALID_ARG, MHS_ERR_NOT_ELLIPTIC (xi(z_k) >= 1 on an
 * interior plane, Sect. 2.1), MHS_ERR_OUT_OF_MEMORY, MHS_ERR_CUDA. */
MHS_API mhs_status mhs_create(int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                      const mhs_xi_params* xi, const mhs_atmos_params* atm, mhs_handle* out);

/* Release every device and host resource of h (NULL is accepted). */
MHS_API void mhs_destroy(mhs_handle h);

/* Order all later device work of h on stream (a cudaStream_t; NULL = legacy default stream). */
MHS_API mhs_status mhs_set_stream(mhs_handle h, void* stream);

/* Replace the solver options (NULL restores the defaults). */
MHS_API mhs_status mhs_set_options(mhs_handle h, const mhs_solver_opts* opts);

/* Change alpha and the xi profile of an existing handle (same grid); the
 * per-plane coefficients are recomputed on the device.  Same errors as
 * mhs_create for these arguments. */
MHS_API mhs_status mhs_set_params(mhs_handle h, double alpha, const mhs_xi_params* xi, const mhs_atmos_params* atm);

/* Prescribe the normal field B_z on z = 0 (Sect. 2.2, eq. lower_bound):
 * bz is [ny][nx] doubles, host or device.  Only interior nodes enter the
 * lower-boundary equation.  Errors: MHS_ERR_INVALID_ARG (NULL),
 * MHS_ERR_NONFINITE (a NaN/Inf among the interior values), MHS_ERR_CUDA. */
MHS_API mhs_status mhs_set_lower_bz(mhs_handle h, const double* bz);

/* Steps 1-3 of Sect. 2.2: the lower-boundary and interior multigrid solves,
 * each until its relative residual ||b - A P||_2/||b||_2 falls below tol
 * (tol in (0, 1)).  mode is an mhs_precision.  info may be NULL.
 * Errors: MHS_ERR_BAD_STATE (no B_z yet), MHS_ERR_INVALID_ARG,
 * MHS_ERR_NO_CONVERGENCE (P is still the last iterate and usable),
 * MHS_ERR_NONFINITE, MHS_ERR_CUDA. */
MHS_API mhs_status mhs_solve(mhs_handle h, double tol, int mode, mhs_solve_info* info);

/* Batched solves (independent instances, any mix of grid sizes and
 * parameters): runs mhs_solve(hs[q], tol, mode, ...) for q < n with every
 * instance on its own internal stream, so that the instances' captured
 * solves overlap on the GPU, and returns when all have finished.  Each
 * instance runs exactly the kernels of its solo solve: results are bitwise
 * identical to solving it alone.  infos and statuses (each n entries) may be
 * NULL; statuses[q] receives the per-instance status.  The return value is
 * MHS_OK or the first failing instance's status.  Work already queued on a
 * handle's own stream is ordered before its batch solve.  Each handle may
 * appear once.  Errors: MHS_ERR_INVALID_ARG, MHS_ERR_BAD_STATE (an instance
 * without B_z), per-instance MHS_ERR_NO_CONVERGENCE / MHS_ERR_NONFINITE,
 * MHS_ERR_CUDA. */
MHS_API mhs_status mhs_batch_solve(mhs_handle* hs, int n, double tol, int mode, mhs_solve_info* infos,
                                   mhs_status* statuses);

/* ---- grouped solves ------------------------------------------------------
 * A group solves n independent instances (handles with any grids,
 * parameters and options) together: every multigrid operation on one
 * level is a single kernel launch for all instances that have that level,
 * and the whole solve (lower-boundary and interior problems, both with the
 * full-multigrid first cycle and V-cycles until each instance reaches the
 * tolerance) is one captured CUDA graph whose loops run while any instance
 * still iterates; converged instances drop out of the launches.  Each
 * instance runs the operations of its solo mhs_solve (its coarse-grid solve
 * included: the separable solve's stages are grouped launches too) with
 * arithmetic that does not depend on the decomposition, so its P is bitwise
 * identical to solving it alone.
 *
 * The instances, ordered by decreasing cycle working set (every level's
 * arrays in the cycle precision, plus the double-float state in mixed
 * mode), are packed into parts of at most part_bytes of working set (0:
 * half the L2 cache), so that a part holds instances of similar size; each
 * part is one graph, and the parts are launched round-robin on nstreams
 * streams (0: 16), so that several parts run at once.  An instance whose
 * working set exceeds a sixteenth of part_bytes takes a part of its own, and a
 * part that holds a single instance runs that instance's own solve, as
 * mhs_solve would, on a stream of its own, as in mhs_batch_solve: grouping
 * pays where launch latency dominates.  part_bytes = SIZE_MAX makes one part
 * of all instances.
 *
 * mhs_group_create snapshots the handles' options, cut-offs and smoother
 * choice (recreate the group after changing a member's options, or its
 * parameters when that moves it to another anisotropy class) and captures
 * the graphs.  The handles must outlive the group and must not be used for
 * other work while a group solve runs.  Not supported: MHS_FLAG_WARM,
 * MHS_FLAG_SEPARABLE, MHS_FLAG_LOWER_FP64 in mixed mode, inner_cycles other
 * than 1 (MHS_ERR_INVALID_ARG).
 * Errors: MHS_ERR_INVALID_ARG (n < 1, NULL or repeated handle, bad mode,
 * nstreams outside [0, 64]), MHS_ERR_OUT_OF_MEMORY, MHS_ERR_CUDA. */
typedef struct mhs_group* mhs_group_t;
MHS_API mhs_status mhs_group_create(mhs_handle* hs, int n, int mode, size_t part_bytes, int nstreams,
                                    mhs_group_t* out);
/* Solve every instance of the group to tol with its current B_z (set by
 * mhs_set_lower_bz, which must have returned for every member).  infos and
 * statuses (n entries each) may be NULL; infos[q].ms is the device time
 * of the part holding instance q.  Returns MHS_OK or the first failing instance's status
 * (MHS_ERR_NO_CONVERGENCE, MHS_ERR_NONFINITE); MHS_ERR_BAD_STATE when a
 * member has no B_z; MHS_ERR_CUDA. */
MHS_API mhs_status mhs_group_solve(mhs_group_t g, double tol, mhs_solve_info* infos, mhs_status* statuses);
MHS_API void mhs_group_destroy(mhs_group_t g);
/* eager != 0: later group solves launch the same kernels from the host, the
 * loops reading the continuation flags back after each cycle, instead of
 * the captured graph (same results; for profilers that cannot see kernels
 * inside conditional graph nodes).  Errors: MHS_ERR_INVALID_ARG. */
MHS_API mhs_status mhs_group_set_eager(mhs_group_t g, int eager);

/* ---- autotuner ----------------------------------------------------------
 * mhs_autotune picks the solver options for h's problem by timing whole
 * solves of its resident B_z to tol in the given mode (CUDA events, the
 * captured-graph path).  Coordinate descent from h's current options over
 * the smoother (red-black point or zebra z-line, MHS_FLAG_ZLINE), the sweep
 * counts (nu1, nu2), the level of the separable coarse-grid solve
 * (sep_coarse: every level that allows it, or none), the sub-cycle cut-off
 * (cut64 in FP64 mode, cut32 in mixed mode; one candidate per level), the
 * fused-sweep threshold of FP32
 * levels (fused_min, mixed mode) and the full-multigrid first cycle
 * (MHS_FLAG_NO_FMG); at most two rounds, a change kept when it saves at
 * least 3 %.  Each candidate costs one untimed solve (graph capture) plus
 * `repeats` timed solves (1..20), of which the fastest counts; candidates
 * that do not converge are dropped.  The winner is applied to h (as by
 * mhs_set_options) and stored in a process-wide table under the class
 * (nx, ny, nz, mode, anisotropy class), where mhs_tune_lookup finds it for
 * other handles of the class.  h's P afterwards is the solution of its last
 * timed solve.  The anisotropy class is floor(log2(max_k max(h_x,h_y)^2 /
 * ((1 - xi(z_k)) h_z^2))), at least 0: vertical over horizontal coupling.
 * Errors: MHS_ERR_BAD_STATE (no B_z), MHS_ERR_INVALID_ARG (tol, mode,
 * repeats), MHS_ERR_CUDA.  Thread-safe across handles. */
typedef struct {
    mhs_solver_opts opts;   /* chosen options (applied to the handle) */
    double ms;              /* fastest timed solve with them */
    double ms_start;        /* fastest timed solve with the options h had on entry */
    int candidates;         /* option sets timed */
    int aniso_class;        /* anisotropy class of the problem */
} mhs_tune_result;

MHS_API mhs_status mhs_autotune(mhs_handle h, double tol, int mode, int repeats, mhs_tune_result* out);
/* Options stored by mhs_autotune for the class of h's current problem in
 * `mode`: *found = 1 and *opts filled, or *found = 0 (opts untouched).
 * Errors: MHS_ERR_INVALID_ARG. */
MHS_API mhs_status mhs_tune_lookup(mhs_handle h, int mode, mhs_solver_opts* opts, int* found);
/* Forget every stored option set. */
MHS_API void mhs_tune_clear(void);

/* ---- request server (continuous batching) ----------------------------
 * A server owns a worker thread and a pool of resident solver hierarchies
 * (one pool per grid shape).  Submitted requests are admitted in arrival
 * order as soon as one of max_inflight slots and enough of the device-
 * memory budget are free; admitted requests run concurrently, each on its
 * own stream, while later requests keep arriving.  Idle hierarchies of
 * other shapes are released when the budget is short.  Each request runs
 * the kernels of a solo mhs_solve + mhs_fields, so its result does not
 * depend on what else is in flight. */
typedef struct mhs_server* mhs_server_t;

typedef struct {
    int nx, ny, nz;                 /* grid (as mhs_create) */
    double Lx, Ly, Lz, alpha;
    mhs_xi_params xi;
    mhs_atmos_params atm;           /* all-zero = defaults */
    double tol;                     /* relative residual target, (0, 1) */
    int mode;                       /* mhs_precision */
    const double* bz;               /* [ny][nx], host or device; copied during mhs_server_submit */
    double* phi;                    /* outputs [nz][ny][nx], host or device, any may be NULL; written */
    double *Bx, *By, *Bz, *p, *rho; /* asynchronously: keep them valid until the request completes */
} mhs_request;

typedef struct {
    long long completed, rejected, queued, running;
    double p50_ms, p99_ms, mean_ms;  /* latency from submission to completion, completed requests */
    double solves_per_s;             /* completed / (last completion - first submission) */
    size_t device_bytes;             /* bytes held by resident hierarchies */
    long long resident_hierarchies;
} mhs_server_stats_t;

/* Errors: MHS_ERR_INVALID_ARG (budget 0, max_inflight outside [1, 1024]), MHS_ERR_CUDA. */
MHS_API mhs_status mhs_server_create(size_t budget_bytes, int max_inflight, mhs_server_t* out);
/* Queue one request; *ticket identifies it.  B_z is copied and checked here
 * (MHS_ERR_NONFINITE for a NaN/Inf interior value, MHS_ERR_INVALID_ARG for
 * bad sizes).  A request whose hierarchy exceeds the whole budget completes
 * with status MHS_ERR_REJECTED. */
MHS_API mhs_status mhs_server_submit(mhs_server_t s, const mhs_request* req, long long* ticket);
/* Non-blocking completion check; on completion fills info, the request's
 * status and its latency, and forgets the ticket. */
MHS_API mhs_status mhs_server_poll(mhs_server_t s, long long ticket, int* done, mhs_solve_info* info,
                                   mhs_status* req_status, double* latency_ms);
/* Blocking wait (timeout_s <= 0: no limit; MHS_ERR_TIMEOUT when it expires). */
MHS_API mhs_status mhs_server_wait(mhs_server_t s, long long ticket, double timeout_s, mhs_solve_info* info,
                                   mhs_status* req_status, double* latency_ms);
MHS_API mhs_status mhs_server_stats(mhs_server_t s, mhs_server_stats_t* out);
/* Finish every queued and running request, then release the server. */
MHS_API void mhs_server_destroy(mhs_server_t s);

/* Copy P (the poloidal potential of eq. b_iden), [nz][ny][nx], to phi (host
 * or device).  Errors: MHS_ERR_BAD_STATE (no solve yet), MHS_ERR_INVALID_ARG. */
MHS_API mhs_status mhs_get_phi(mhs_handle h, double* phi);

/* Steps 4-5 (Sect. 2.2, eqs. b_iden, t, pressure, density): B_x, B_y, B_z,
 * p and rho on every node, each [nz][ny][nx] (host or device; any may be
 * NULL to skip it).  Central differences inside, second-order one-sided
 * differences on the first and last node of each axis.
 * Errors: MHS_ERR_BAD_STATE (no solve yet), MHS_ERR_CUDA. */
MHS_API mhs_status mhs_fields(mhs_handle h, double* Bx, double* By, double* Bz, double* p, double* rho);

/* ---- post-processing: the quantities of the paper's figures (Sect. 3) ----
 * mhs_current: the current density j = curl B / mu0 of the latest solve's B
 * (recomputed as by mhs_fields), with the same difference operators
 * (central inside, second-order one-sided on the first and last node of
 * each axis), its magnitude |j| and |B|; each [nz][ny][nx], host or device,
 * any may be NULL.  Errors: MHS_ERR_BAD_STATE (no solve yet), MHS_ERR_CUDA. */
MHS_API mhs_status mhs_current(mhs_handle h, double* jx, double* jy, double* jz, double* jmag, double* bmag);

/* mhs_trace: magnetic field lines of the latest solve's B.  From each of the
 * n seeds (x, y, z; node (i, j, k) sits at (i h_x, j h_y, k h_z)), classical
 * fourth-order Runge-Kutta steps of arc length ds along dr/ds = direction *
 * B/|B| (direction +1 or -1), B interpolated trilinearly in its cell (along
 * x, then y, then z), at most max_steps steps.  A step is taken only when
 * its four stage points and its end point lie in the closed box
 * [0,Lx]x[0,Ly]x[0,Lz] and |B| does not vanish at the stage points;
 * otherwise the line ends.  points: n x (max_steps + 1) x 3 doubles, the
 * seed first (entries past a line's end are left as they were); lengths: n
 * ints, the number of points of each line, 0 for a seed outside the box.
 * seeds, points and lengths may be host or device memory; host buffers are
 * staged through temporary device memory and the call then returns after
 * the copies.  The arithmetic is IEEE FP64 with every operation rounded
 * separately (no fused multiply-add), in a fixed order.
 * Errors: MHS_ERR_BAD_STATE (no solve yet), MHS_ERR_INVALID_ARG (n < 0,
 * max_steps < 0, ds <= 0, direction not +1/-1, NULL buffers, output over
 * 64 GB), MHS_ERR_CUDA. */
MHS_API mhs_status mhs_trace(mhs_handle h, const double* seeds, int n, double ds, int max_steps, int direction,
                             double* points, int* lengths);

/* mhs_trace_field: the same tracer on caller-supplied device arrays Bx, By,
 * Bz, dense [nz][ny][nx], on the box [0,Lx]x[0,Ly]x[0,Lz] (nx, ny, nz >= 2),
 * enqueued on `stream` (a cudaStream_t, NULL for the default stream).
 * Errors: MHS_ERR_INVALID_ARG (as mhs_trace, or B not in device memory),
 * MHS_ERR_CUDA. */
MHS_API mhs_status mhs_trace_field(int nx, int ny, int nz, double Lx, double Ly, double Lz, const double* Bx,
                                   const double* By, const double* Bz, const double* seeds, int n, double ds,
                                   int max_steps, int direction, double* points, int* lengths, void* stream);

/* Number of multigrid levels of the interior (dim = 3) or lower-boundary
 * (dim = 2) hierarchy, and the node counts of one level (level 0 finest). */
MHS_API mhs_status mhs_num_levels(mhs_handle h, int dim, int* nlevels);
MHS_API mhs_status mhs_level_shape(mhs_handle h, int dim, int level, int* nx, int* ny, int* nz);

/* Level-access hooks for operation-by-operation parity tests.  They expose
 * the very kernels the solver runs, on one level of the resident hierarchy.
 *   field: MHS_FIELD_U (iterate / correction), MHS_FIELD_F (right-hand side),
 *          MHS_FIELD_R (residual)
 *   prec:  MHS_FP64 or MHS_MIXED (the FP32 copy)
 * Arrays are dense doubles of the level's shape (converted to/from FP32 for
 * prec = MHS_MIXED), host or device.
 * Operations (op):
 *   MHS_OP_SMOOTH:   one red-black Gauss-Seidel sweep on u (colour (i+j+k)
 *                    even first, then odd) for A u = f                 (Sect. 4)
 *   MHS_OP_RESIDUAL: r = f - A u on interior nodes                      (Sect. 4)
 *   MHS_OP_RESTRICT: f[level+1] = full-weighting restriction of r[level] (Sect. 4)
 *   MHS_OP_PROLONG:  u[level] += (bi/tri)linear interpolation of u[level+1] (Sect. 4)
 *   MHS_OP_COARSE:   coarsest-level solve of A u = f (u from 0)
 *   MHS_OP_VCYCLE:   one V(nu1,nu2)-cycle on A u = f from level down
 *   MHS_OP_RESID_RESTRICT: f[level+1] = full-weighting restriction of
 *                    f - A u on level (residual and restriction in one pass,
 *                    the residual not stored; u[level+1] zeroed; as the
 *                    V-cycles run them)                                (Sect. 4)
 *   MHS_OP_EXACT:    u = A^{-1} f on the interior by the separable solver
 *                    (zero boundary values; the level's r and t are
 *                    scratch); levels whose sine transforms are fast
 *                    or short (see sep_coarse), else MHS_ERR_INVALID_ARG
 *   MHS_OP_RESTRICT_RED: MHS_OP_RESTRICT of a residual taken right after a
 *                    red-black sweep, which vanishes at the black nodes
 *                    (i+j+k odd): only the centre and the 12 edge neighbours
 *                    of each fine node under a coarse one are read (the
 *                    form the FP64 V-cycles use); r[level] must be +0 at
 *                    the black nodes, where the result then equals
 *                    MHS_OP_RESTRICT's
 * For the finest interior level, A includes the Dirichlet data held in u's
 * boundary entries.  Errors: MHS_ERR_INVALID_ARG, MHS_ERR_CUDA. */
#define MHS_FIELD_U 0
#define MHS_FIELD_F 1
#define MHS_FIELD_R 2
#define MHS_OP_SMOOTH 0
#define MHS_OP_RESIDUAL 1
#define MHS_OP_RESTRICT 2
#define MHS_OP_PROLONG 3
#define MHS_OP_COARSE 4
#define MHS_OP_VCYCLE 5
#define MHS_OP_EXACT 6
#define MHS_OP_RESID_RESTRICT 7
#define MHS_OP_RESTRICT_RED 8
MHS_API mhs_status mhs_level_write(mhs_handle h, int dim, int level, int field, int prec, const double* src);
MHS_API mhs_status mhs_level_read(mhs_handle h, int dim, int level, int field, int prec, double* dst);
MHS_API mhs_status mhs_level_op(mhs_handle h, int dim, int level, int op, int prec);

/* Per-operation device timing (CUDA events on the handle's stream), off by
 * default.  While enabled, every multigrid operation and field kernel of
 * the handle is bracketed by two events; mhs_kernel_timing() synchronises
 * the stream and returns, for one operation kind, the summed duration, the
 * number of timed launches and the algorithmic bytes and flops of those
 * launches (minimal traffic of the operation: each input read once, each
 * output written once).  Kinds are MHS_KT_*; mhs_kernel_timing_reset()
 * clears the totals. */
#define MHS_KT_SMOOTH64 0      /* red-black sweep, FP64 */
#define MHS_KT_SMOOTH32 1      /* red-black sweep, FP32 */
#define MHS_KT_RESID64 2       /* residual (+ norm partials), FP64 */
#define MHS_KT_RESID32 3       /* residual, FP32 */
#define MHS_KT_RESTRICT64 4
#define MHS_KT_RESTRICT32 5
#define MHS_KT_PROLONG64 6
#define MHS_KT_PROLONG32 7
#define MHS_KT_COARSE64 8      /* coarse-grid solve, FP64: the one-CTA sub-cycle or the separable solve of a level */
#define MHS_KT_COARSE32 9      /* the same in FP32 */
#define MHS_KT_RESID_MIXED 10  /* double-float outer residual rounded to the FP32 right-hand side */
#define MHS_KT_CORRECT 11      /* (hi, lo) += e32, the double-float iterate */
#define MHS_KT_FIELDS 12       /* B, p, rho */
#define MHS_KT_OTHER 13        /* set-up, copies, norms of the right-hand side */
#define MHS_KT_SEPARABLE 14    /* separable inner solve (sine transforms, mode tridiagonal solves) */
#define MHS_KT_COUNT 15
MHS_API mhs_status mhs_set_kernel_timing(mhs_handle h, int enable);
MHS_API mhs_status mhs_kernel_timing(mhs_handle h, int kind, double* total_ms, long long* launches,
                                     double* alg_bytes, double* alg_flops);
/* The same totals restricted to operations on the finest interior level. */
MHS_API mhs_status mhs_kernel_timing_finest(mhs_handle h, int kind, double* total_ms, long long* launches,
                                            double* alg_bytes, double* alg_flops);
MHS_API mhs_status mhs_kernel_timing_reset(mhs_handle h);
MHS_API const char* mhs_kernel_kind_name(int kind);

/* Allocation-free residual check (the paper has no counterpart; this is a
 * service for callers that may not allocate device memory: applications
 * whose device memory is owned entirely by their own pool allocator, and
 * loops that cannot afford the device-wide synchronisation that cudaMalloc
 * or cudaFree may imply).  It evaluates, for a caller-supplied potential P
 * whose six faces are Dirichlet data, the relative residual of the interior
 * problem of eq. (scalar_pot) with zero interior source:
 *   out[0] = ||b - A P||_2 over the interior nodes,
 *   out[1] = ||b||_2, b = the right-hand side after lifting the Dirichlet
 *            data (every face value of P enters the row of its interior
 *            neighbour, weighted by that row's coefficient),
 *   out[2] = out[0] / out[1] (0 when ||b|| = 0).
 * For a P returned by mhs_get_phi (faces zero except z = 0) this is the
 * quantity mhs_solve's stopping test and rel_res_3d report.
 * P: device pointer, dense [nz][ny][nx] doubles; out: device pointer to 3
 * doubles; stream: cudaStream_t (NULL = legacy default stream).  The call is
 * asynchronous on that stream and allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  Its scratch is one fixed
 * device array of about 176 KB inside the library, which every GPU that
 * loads the library holds until the process exits.  Limits: nx, ny, nz >= 3
 * and nz <= 4097; finite, positive lengths; finite alpha and xi parameters,
 * a known xi kind (MHS_ERR_INVALID_ARG otherwise); P and out must be device
 * pointers (MHS_ERR_INVALID_ARG otherwise).  The first call on each device
 * looks up the scratch array's device address (cudaGetSymbolAddress) and
 * caches it for the life of the process; make that first call before any
 * stream capture, and do not call this entry point on a device after a
 * cudaDeviceReset of that device (the cached address would be stale).
 * Every call shares the one scratch array: calls whose work overlaps on the
 * GPU (other streams, other threads) race on it, so serialise them. */
MHS_API mhs_status mhs_interior_residual_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz,
                                                 double alpha, const mhs_xi_params* xi, const double* P,
                                                 double* out, void* stream);

/* Human-readable name of a status code (static storage). */
MHS_API const char* mhs_status_string(mhs_status s);

/* Thread-local description of the last failure on the calling thread
 * (empty string if none).  Valid until the next failing call on that thread. */
MHS_API const char* mhs_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles; for launch accounting around a timed region). */
MHS_API long long mhs_kernel_launches(void);

/* Device arithmetic-rate probe (a measurement aid for the roofline of the
 * FP64 stencil kernels, which the FP64 pipe bounds on this part): the
 * sustained fused multiply-add rate of the current device in flop/s (two
 * flops per FMA), FP64 for precision = MHS_FP64, FP32 for MHS_MIXED.  Every
 * thread of a grid of 8 blocks of 256 threads per SM runs eight independent
 * FMA chains; one launch of about 10 ms (FP64) or 5 ms (FP32) is timed with
 * CUDA events on `stream` after one warm-up launch.  Synchronises the
 * stream.  Errors: MHS_ERR_INVALID_ARG, MHS_ERR_CUDA. */
MHS_API mhs_status mhs_probe_fma_rate(int precision, void* stream, double* flops_per_s);

/* Library version string (static storage). */
MHS_API const char* mhs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MHS_H */
