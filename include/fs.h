/*
 * fs.h -- C ABI of the fractional-step finite-volume / immersed-boundary
 * time step (Diff-FlowFSI, arXiv 2505.23940), B300 (sm_103a) CUDA library.
 *
 * Conventions for every function
 *   - Returns an int status: FS_OK (0) or a negative FS_ERR_* code.  The text
 *     of the last error of the calling thread is returned by fs_last_error().
 *     No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the grid's device;
 *     "host" pointers are ordinary CPU memory.  The library never takes
 *     ownership of a caller pointer and never frees one.
 *   - Work is enqueued on the stream given to fs_create_grid (or
 *     fs_set_stream).  Functions return without waiting for the GPU unless
 *     their comment says they synchronise.
 *
 * Discretisation (§2.3.1 of the paper): staggered (MAC) finite-volume grid,
 * pressure at cell centres, velocity component c on the faces normal to
 * direction c; 2nd-order central diffusion, 2nd-order central or 1st-order
 * upwind convection; Chorin projection (Eqs. 4-10).
 *
 * Field layout (every velocity array, state or adjoint): dense, x fastest,
 * index = i + ex * (j + ey * k).  Component c has extents (ex, ey, ez) equal
 * to the cell counts n, except along its own direction c where a
 * non-periodic direction stores n_c + 1 faces (faces 0 and n_c lie on the
 * boundary).  fs_field_extent() returns them.  Pressure arrays have extents n.
 * In 2-D, n[2] = 1 and there is no w component.
 */
#ifndef FS_H
#define FS_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FS_OK               0
#define FS_ERR_ARG         -1   /* invalid argument or combination (message says which) */
#define FS_ERR_CUDA        -2   /* a CUDA runtime call failed */
#define FS_ERR_DIVERGED    -3   /* NaN/Inf or |u| above the blow-up bound after a step */
#define FS_ERR_TIMEOUT     -4   /* a bounded device-side wait ran out */
#define FS_ERR_UNSUPPORTED -5   /* a valid request this library does not implement */
#define FS_ERR_STATE       -6   /* call out of order (e.g. forces before any step) */

/* ---- boundary types (Table 1 of the paper) ---------------------------- */
#define FS_BC_PERIODIC 0
#define FS_BC_NOSLIP   1   /* Dirichlet: wall velocity bc_val */
#define FS_BC_FREESLIP 2   /* no penetration, zero tangential stress */
#define FS_BC_INFLOW   3   /* Dirichlet velocity bc_val (x-low only) */
#define FS_BC_OUTFLOW  4   /* zero-gradient, flux-corrected (x-high only) */

#define FS_CENTRAL2 0      /* 2nd-order central convection */
#define FS_UPWIND1  1      /* 1st-order upwind convection */
#define FS_FE       0      /* forward Euler (the paper's runs) */
#define FS_RK3      1      /* SSP Runge-Kutta 3, projection at every stage */
#define FS_FP64     0      /* every step in FP64 */
#define FS_MIXED    1      /* FP32 stencils, transforms and IB transfers; FP64
                              tridiagonal / zero-mode solves, reductions, body ODE */
#define FS_PESKIN4  0      /* 4-point kernel of Eq. (22) */
#define FS_ROMA3    1      /* 3-point kernel of Roma, Peskin & Berger (1999) */

typedef struct fs_grid fs_grid;   /* opaque; owns plans, workspaces, IB buffers */

/* Grid description (§2.5: rectangular domain, uniform or stretched spacing).
 * x and z must be uniform; y may be stretched when it is not periodic.
 * Supported: 2-D with x periodic / inflow-outflow / walls and y periodic /
 * walls; 3-D with x and z periodic and y periodic / walls.  Periodic
 * directions need an even cell count; transform lengths need prime factors
 * <= 13. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int n[3];                /* cell counts (n[2] = 1 in 2-D) */
  const double* xf[3];     /* host: n[d] + 1 face coordinates per direction (xf[2] unused in 2-D) */
  int bc[3][2];            /* FS_BC_* at the low / high side of each direction */
  double bc_val[3][2][3];  /* velocity vector imposed at each side (NOSLIP wall velocity, INFLOW velocity) */
  double nu;               /* kinematic viscosity */
  double rho;              /* density */
  int conv_scheme;         /* FS_CENTRAL2 | FS_UPWIND1 */
  int time_scheme;         /* FS_FE | FS_RK3 */
  int precision;           /* FS_FP64 | FS_MIXED */
  const double* body_force;/* host: n[1] values of an x-momentum source per y row, or NULL */
} fs_grid_desc;

/* Solver state.  The caller owns every buffer (e.g. torch tensors).
 * u[c]  device, velocity component c with the extents of fs_field_extent:
 *       double for FS_FP64 grids, float for FS_MIXED grids.
 * p     device, double, cell-centred pressure written by fs_step (may be NULL).
 * body  device, double[4] = {w_x, w_y, wdot_x, wdot_y}: rigid-body
 *       displacement and velocity; NULL when the grid has no body. */
typedef struct {
  void*   u[3];
  double* p;
  double* body;
} fs_state;

/* Immersed body (§2.3.3): a closed polygon of Lagrangian markers, or several
 * disjoint closed contours (an array of cylinders), rigid, translating with
 * the displacement of fs_state.body, optionally elastically mounted (Eq. 12). */
typedef struct {
  int nm;                  /* number of markers (>= 3) */
  const double* X0;        /* host: rest x of each marker, ordered around the surface */
  const double* Y0;        /* host: rest y */
  const double* ds;        /* host: arc length per marker; dV_i = ds_i * h (shell of one cell) */
  double centre[2];        /* reference point (rotation centre) at rest */
  double omega;            /* prescribed surface angular velocity (geometry does not turn) */
  double mass;             /* m of Eq. (12); <= 0 holds the body fixed */
  double stiffness;        /* k */
  double damping;          /* c */
  int active[2];           /* DOF mask: x, y */
  int delta_kernel;        /* FS_PESKIN4 | FS_ROMA3 */
  int ncontour;            /* number of closed contours; 0 or 1: all markers form one contour */
  const int* contour_start;/* host: ncontour increasing first-marker indices (the first 0), each
                              contour >= 3 markers and closed on its own first marker; NULL when
                              ncontour <= 1 */
} fs_body_desc;

/* Parameter-gradient accumulators filled by fs_step_adjoint (added to, never cleared). */
typedef struct {
  double* body_force;      /* device, n[1] doubles: dJ/d f_x(y_j), or NULL */
  double* stiffness;       /* device, 1 double: dJ/dk, or NULL */
} fs_param_grad;

/* Create a grid: validates the description, builds metrics, transform plans
 * and tridiagonal tables, and allocates every workspace on the current CUDA
 * device.  stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: FS_ERR_ARG (bad sizes, BC combination, non-uniform x/z),
 * FS_ERR_UNSUPPORTED (transform length with a prime factor > 13),
 * FS_ERR_CUDA (allocation). */
int fs_create_grid(const fs_grid_desc* desc, void* stream, fs_grid** out);

/* Free every device buffer the grid owns.  Synchronises the grid's stream. */
int fs_destroy_grid(fs_grid* grid);

/* Change the stream later work is enqueued on. */
int fs_set_stream(fs_grid* grid, void* stream);

/* Extents (ex, ey, ez) of velocity component comp (0..dim-1); comp = -1 gives
 * the cell counts (pressure).  Host output. */
int fs_field_extent(const fs_grid* grid, int comp, int ext[3]);

/* Attach a rigid body (2-D grids, uniform x and y near the body).  Marker
 * arrays are host memory and are copied.  Replaces any previous body.
 * Eqs. (18)-(23): solid faces (inside the polygon: an odd number of edge
 * crossings to their right) and IB faces (non-solid faces with a solid
 * same-component neighbour) are forced; the target velocity is the body
 * velocity inside and the half-distribution-normalised marker interpolation
 * on IB faces.  Every step then classifies the faces row by row from the
 * edges crossing each row (edges sorted by their lowest point, found by
 * bisection), computes F_N (Eq. 19) per marker, and forms the interpolation
 * on each IB face by gathering the markers of the nearby cells (markers
 * binned by the cell of their rest position; the body only translates): a
 * fixed summation order per face, so results are bitwise reproducible, with
 * no atomics.  Errors: FS_ERR_ARG (bad contour list), FS_ERR_UNSUPPORTED
 * (3-D grid, RK3 grid). */
int fs_set_ib_markers(fs_grid* grid, const fs_body_desc* body);

/* Attach a static 3-D body made of axis-aligned boxes (the paper's cube
 * roughness and obstacle cases, §3.4, forced as in §2.3.3): faces strictly
 * inside a box are solid, non-solid faces with a solid same-component
 * neighbour are IB faces, and both are forced to the velocity of a body at
 * rest, u_s = u_c = 0 (Eqs. 5, 18, 23).  The markers only carry the force,
 * q_i = -sum_faces f delta_h(x - X_i) dv (Eq. 20, 3-D tensor-product delta of
 * the chosen kernel), F = rho sum_i q_i dV_i.  The classification is done once,
 * here.  Replaces any previous box body.
 *   boxes  host, nbox x 6 doubles: x0, x1, y0, y1, z0, z1 (x0 < x1 ...)
 *   X      host, nm x 3 marker positions;  dV  host, nm marker volumes
 * fs_forces then returns F[3], torque 0 and q (nm x 3).  Requirements: 3-D
 * grid, forward Euler, uniform x, y and z.  fs_step_adjoint returns
 * FS_ERR_UNSUPPORTED on such a grid.  Errors: FS_ERR_ARG, FS_ERR_UNSUPPORTED,
 * FS_ERR_CUDA. */
int fs_set_ib_boxes(fs_grid* grid, int nbox, const double* boxes, int nm, const double* X, const double* dV,
                    int delta_kernel);

/* Advance st by nsteps time steps of size dt (Eqs. 4-10, 18-23, 12).
 * dt > 0: fixed step, no host synchronisation.
 * dt <= 0: adaptive step dt = 0.5 * min(h) / max|u| from the state before
 *          each step (§2.5, CFL condition), which synchronises once per step.
 * st->u is updated in place; st->p (if not NULL) receives the pressure of the
 * last step; st->body (required when a body is attached) is advanced by RK4.
 * Errors: FS_ERR_ARG (NULL field), FS_ERR_DIVERGED (checked only for dt <= 0),
 * FS_ERR_CUDA. */
int fs_step(fs_grid* grid, fs_state* st, double dt, int nsteps);

/* Discrete adjoint of one fs_step(dt, 1) (§2.4.1): given the forward state at
 * step n (st_n, not modified) and the adjoint lam of the state after the
 * step, overwrite lam with the adjoint of the state before the step and add
 * parameter gradients to g.  dJdF: host, dim doubles, the sensitivity of the
 * loss to the hydrodynamic force of this step (may be NULL).  The forward
 * step is recomputed internally.  The epsilon mask is frozen (its derivative
 * is zero almost everywhere).
 * Strongly coupled steps (fs_set_coupling with max_subiters > 1, elastically
 * mounted body) are differentiated implicitly (§2.4.1) at the fixed point of
 * Algorithm 1: the forward sub-iteration is re-run from st_n to its converged
 * body state s* (synchronising once per sub-iteration, as fs_step does), the
 * fluid step is linearised at (u^n, s*) and the body ODE at (s^n, F(u^n, s*)),
 * and mu solves (I - B_F J_s)^T mu = lam_s + U_s^T lam_u + J_s^T dJdF (B the
 * RK4 step, U the new velocity, J_s the force's dependence on the body
 * kinematics), a 4 x 4 system solved on the device; then lam_s^n = B_s^T mu,
 * lam_u^n = U_u^T lam_u + J_u^T (dJdF + B_F^T mu) and dJ/dk += B_k^T mu.  It
 * costs the forward sub-iterations plus one fluid adjoint for the loss and one
 * per active DOF, and synchronises the stream at its end (FS_ERR_DIVERGED when
 * I - dB/ds is singular).  The body-force gradient is not provided there
 * (FS_ERR_UNSUPPORTED).
 * Errors: FS_ERR_UNSUPPORTED (rotating surface with a body, Smagorinsky model,
 * static box body), FS_ERR_ARG, FS_ERR_CUDA. */
int fs_step_adjoint(fs_grid* grid, const fs_state* st_n, fs_state* lam,
                    const double* dJdF, fs_param_grad* g, double dt);

/* fs_step_adjoint with dJdF in device memory (dim doubles, or NULL): the
 * reverse sweep of a rollout can then keep the per-step force sensitivities on
 * the device and needs no host read between adjoint steps. */
int fs_step_adjoint_dev(fs_grid* grid, const fs_state* st_n, fs_state* lam,
                        const double* dJdF, fs_param_grad* g, double dt);

/* One RK3 step (fs_step with nsteps = 1 and a fixed dt > 0) that leaves its two
 * intermediate stage states in v1[dim], v2[dim]: caller-owned device arrays
 * shaped like st->u, in the grid's precision.  st->p, if not NULL, receives the
 * pressure.  Errors: FS_ERR_ARG (NULL arrays, dt <= 0, a forward-Euler grid),
 * FS_ERR_UNSUPPORTED (body, static boxes or Smagorinsky model), FS_ERR_CUDA. */
int fs_step_record(fs_grid* grid, fs_state* st, double dt, void* const* v1, void* const* v2);

/* fs_step_adjoint of a step recorded by fs_step_record from st_n, with its
 * stage states v1, v2 (device, not modified): nothing of the forward step is
 * recomputed.  The result equals fs_step_adjoint's.  Errors as fs_step_record. */
int fs_step_adjoint_recorded(fs_grid* grid, const fs_state* st_n, void* const* v1, void* const* v2,
                             fs_state* lam, fs_param_grad* g, double dt);

/* Solve the discrete pressure Poisson equation D G p = rhs (Eq. 9) exactly
 * (FFT / DCT along x and z, FP64 tridiagonal along y) for the zero
 * volume-weighted-mean solution.  rhs, p: device doubles with the cell
 * counts' extents; may alias.  rhs must be compatible (zero volume-weighted
 * sum) when the operator is singular. */
int fs_solve_pressure(fs_grid* grid, const double* rhs, double* p);

/* Solve D G p = rhs (Eq. 9) with the paper's Krylov iteration (§2.5 and
 * Table 1: conjugate gradients): CG on A = -V D G (symmetric positive
 * semi-definite in the plain inner product, V the cell volumes), optionally
 * Jacobi-preconditioned by diag(A), from p = 0 until ||r|| <= tol ||r_0|| or
 * maxit iterations.  The right-hand side's plain mean is removed first (the
 * constant null space when no pressure is imposed) and the result has zero
 * volume-weighted mean, the gauge of fs_solve_pressure, which it matches to
 * the tolerance.  FP64 grids only; every step runs in FP64.
 *   rhs, p   device doubles with the cell counts' extents; must not alias
 *   jacobi   0: plain CG (the paper's default), 1: Jacobi preconditioning
 *   iters    host, iterations taken (may be NULL)
 *   relres   host, final ||r|| / ||r_0|| (may be NULL)
 * Synchronises the grid's stream every 8 iterations to test convergence; the
 * first call allocates a workspace of 3 cells + 16 doubles kept by the grid.
 * Errors: FS_ERR_ARG, FS_ERR_UNSUPPORTED (mixed grid), FS_ERR_DIVERGED (NaN
 * residual), FS_ERR_CUDA. */
int fs_solve_pressure_cg(fs_grid* grid, const double* rhs, double* p, double tol, int maxit, int jacobi,
                         int* iters, double* relres);

/* Replace the x-momentum source profile (n[1] values, device doubles) used by
 * later steps, e.g. to make it a differentiable parameter.  The grid must
 * have been created with a body_force profile.  Enqueued on the grid's stream. */
int fs_set_body_force(fs_grid* grid, const double* fx);

/* Strong fluid-structure coupling (§2.3.3, Algorithm 1).  With max_subiters > 1
 * every forward-Euler step of a grid with an elastically mounted body
 * sub-iterates: the fluid is advanced from u^n with the kinematics of the
 * current body iterate (iterate 0 = the body at level n), the body ODE is
 * advanced from its level-n state with the force of that fluid solve, until
 * xi = |w_k - w_{k-1}|^2 / |w_{k-1}|^2 < tol (|w_k - w_{k-1}|^2 while w_{k-1} = 0)
 * or max_subiters fluid solves.  max_subiters = 1 (the default) is the weakly
 * coupled step.  Each sub-iteration reads xi on the host (one stream
 * synchronisation).  fs_step_adjoint differentiates such a step implicitly
 * at its fixed point.  Errors: FS_ERR_ARG (max_subiters < 1, tol <= 0). */
int fs_set_coupling(fs_grid* grid, int max_subiters, double tol);

/* Constant-coefficient Smagorinsky subgrid model (§2.5; the LES of §3.4):
 * every later step adds d_j tau_ij, tau_ij = 2 nu_t S_ij, nu_t = (C_s Delta)^2
 * sqrt(2 S_ij S_ij), Delta = (h_x h_y h_z)^(1/3), to R of Eq. (4); normal
 * strains at cell centres, shear strains at cell edges, nu_t at centres and
 * averaged to edges.  cs = 0 switches the model off.  Provided for 3-D grids
 * periodic (hence uniform) in x, y and z with central convection and no body;
 * fs_step_adjoint returns FS_ERR_UNSUPPORTED while it is on.
 * Errors: FS_ERR_ARG (cs < 0), FS_ERR_UNSUPPORTED, FS_ERR_CUDA. */
int fs_set_les(fs_grid* grid, double cs);

/* Number of IB faces (both components) classified by the last step of a grid with
 * a 2-D body (host output; synchronises the grid's stream).  FS_ERR_STATE
 * without a body. */
int fs_ib_face_count(fs_grid* grid, int* count);

/* Sub-iterations and final xi of the last strongly coupled step (host outputs, may be NULL). */
int fs_coupling_stats(const fs_grid* grid, int* subiters, double* xi);

/* Replace the spring stiffness k of the attached body (Eq. 12). */
int fs_set_stiffness(fs_grid* grid, double k);

/* Copy the force of the last step, {F_x, F_y, torque}, to device memory
 * (3 doubles) on the grid's stream, without synchronising. */
int fs_forces_device(fs_grid* grid, double* F);

/* Hydrodynamic force of the last step (Eq. 20 with F = rho sum_i q_i dV_i).
 * Host outputs: F[dim], torque[1], q[nm * 2] marker forces (q may be NULL);
 * for a static 3-D box body F[3], torque 0 and q[nm * 3].
 * Synchronises the grid's stream.  FS_ERR_STATE before the first FSI step. */
int fs_forces(fs_grid* grid, double* F, double* torque, double* q);

/* Diagnostics of a state: out[0] = max |u|, out[1] = max |D u| (FP64),
 * out[2] = kinetic energy 1/2 sum u^2 dV.  Host output; synchronises. */
int fs_diagnostics(fs_grid* grid, const fs_state* st, double out[3]);

/* Number of kernels launched by this grid since creation (host counter). */
long long fs_kernel_launches(const fs_grid* grid);

/* Device status bits set by kernels since the last call, then cleared:
 * bit 0 = a bulk-copy wait of the staged predictor gave up after 2 s (the
 * outputs of that step are invalid).  Host output; synchronises the stream. */
int fs_device_status(fs_grid* grid, unsigned* bits);

/* Launch parameters chosen by an autotuner (0 restores the default):
 *   "stencil_bx"      x threads of the 256-thread stencil blocks: 32, 64, 128, 256
 *   "fft_lines"       complex lines per block of the mixed-radix transforms
 *                     (lengths other than 64, 128, 256): 1..16
 *   "predictor_cells" cells per thread of the FP32 predictor: 1 (the one-cell kernel), 2 (3-D) or
 *                    4 (default; 2-D: fully periodic grids without a body)
 *   "predictor_zmarch" z planes per thread of the four-cell predictor: 1 (no
 *                     march) .. 64; default 8
 *   "pdl"             1 (default): step kernels use programmatic dependent
 *                     launch (each starts while its predecessor drains);
 *                     0: ordinary stream-ordered launches
 *   "predictor_staged" 1 (default): on fully periodic FP32 grids with n_x =
 *                     128 or 256 the predictor stages its input planes in
 *                     shared memory with bulk asynchronous copies; 0: it reads
 *                     them from global memory (four-cell z-marching kernel)
 *   "predictor_chunk" staged predictor work split: 0 (default) equal shares of
 *                     the (row block, plane) units for grids whose three
 *                     velocity fields fit in 64 MB, else runs of planes aligned
 *                     across row blocks (about two blocks per SM); -1 equal
 *                     shares; N > 0 aligned runs of N planes
 *   "y_spectral"      periodic y only: 1 (default) DFT along y in the grid's
 *                     field precision, zero mode exact; 0: the FP64 cyclic
 *                     tridiagonal solve per x/z wavenumber (rebuilds the y
 *                     tables; synchronises).  Same discrete solution.
 *   "ysolve_twisted"  FP64 tridiagonal y solve form: 1 twisted factorisation,
 *                     two threads per column (where ny <= 586, and on periodic
 *                     y where ny is even; elsewhere the partitioned form); 0 the
 *                     partitioned form; -1 (default) twisted when the grid has
 *                     at least 148 * 64 columns (n_x n_z) and ny <= 292.
 *                     Rebuilds the y tables (synchronises the stream)
 *   "ysolve_twist_columns" columns per block of the twisted solve: 64 or 32
 *                     (0, the default: 64 while a block fits an SM, ny <= 292,
 *                     else 32); rebuilds the y tables
 *   "ysolve_tiled"    1 (default): the twisted solve loads FP32 tiles of at
 *                     least 32 rows as 16-row tensor-map boxes (not on walls
 *                     with ny odd); 0: one bulk copy per row
 *   "xz_plane"        on 3-D FP32 grids with nx = nz of 64 or 128 and periodic
 *                     x (no immersed body) the x and z transforms of the
 *                     Poisson solve run fused per y position, its x-z plane in
 *                     shared memory (one pass over the field each way instead
 *                     of two; not where "ysplit" applies): 1 (default) one
 *                     block per plane, 2 the plane split over a cluster of two
 *                     blocks (slower at 128^3: 0.288 against 0.219 ms per
 *                     step); 0: separate x and z kernels
 *   "ysplit"          1: on periodic-z grids whose twisted y solve has two or
 *                     more column blocks along x, the z transforms and the y
 *                     solve of the two halves of the x spectrum run as two
 *                     independent chains on two streams (a second, library-owned
 *                     stream; fork after the x transform, join before its
 *                     inverse); 0 (default): one chain.  Same result bit for bit
 *                     (at 128^3 no faster: each half's y solve, one block per
 *                     SM, takes nearly the whole solve's time)
 *   "ysolve_segments" segments per column of the partitioned wall-bounded y
 *                     solve: 4, 8 or 16 (default: 8 for ny >= 192 or when the
 *                     grid has fewer 32-column blocks than two per SM, else 4);
 *                     rebuilds the y tables
 *                     (synchronises the stream; set it before capturing graphs)
 * Results do not depend on them (ysolve_*, y_spectral: up to rounding).
 * FS_ERR_ARG for an unknown key or value. */
int fs_set_tuning(fs_grid* grid, const char* key, int value);

/* Kernel timing.  After fs_profile_begin, every launch whose kernel name
 * contains `filter` ("" = all) is bracketed by CUDA events on the grid's
 * stream.  fs_profile_end synchronises the stream and writes one line per
 * kernel name, "name launches total_ms", into report (host, len bytes,
 * truncated and NUL-terminated). */
int fs_profile_begin(fs_grid* grid, const char* filter);
int fs_profile_end(fs_grid* grid, char* report, int len);

/* Allocation-free statistics of one velocity component (the paper has no
 * counterpart; this is a library service).  For callers that may not call
 * cudaMalloc -- e.g. a host application whose device memory belongs to its
 * own pool allocator, or a loop where an allocation's implicit device
 * synchronisation is not allowed -- and therefore cannot create an fs_grid.
 * Computes, on `stream`, out[0] = sum over the field of 0.5 u^2 vol w_j and
 * out[1] = max |u|, where w_j = wy[j] for the row index j of each element
 * (wy: device, ext[1] doubles, or NULL for w_j = 1).
 *   u          device, dense x-fastest array of ext[0] * ext[1] * ext[2]
 *              elements, double (FS_FP64) or float (FS_MIXED)
 *   out        device, 2 doubles, written by the GPU (read it after the stream)
 * Allocates nothing: its reduction scratch is a fixed 64 KiB file-scope
 * device array present on every device that loads the library, until exit.
 * The first call in each CUDA context of a device (the primary context, a
 * driver-API context, the primary context re-created after cudaDeviceReset)
 * looks up that array's address (cudaGetSymbolAddress); make that first call
 * before any stream capture.
 * Every call shares the scratch: calls that overlap on the GPU (different
 * streams, no ordering between them) race and give wrong results.  Each call
 * overwrites every scratch slot it reads, so nothing needs clearing.
 * Errors: FS_ERR_ARG for NULL pointers, bad precision or extents, and for
 * fields of more than 33,554,432 elements (the scratch holds 4096 partials of
 * 8192 elements each); FS_ERR_CUDA for a failed launch. */
int fs_component_stats_noalloc(const void* u, int precision, const int ext[3], double vol,
                               const double* wy, double* out, void* stream);

/* Text of the calling thread's last error ("" if none). */
const char* fs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FS_H */
