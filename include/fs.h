/*
 * fs.h -- C ABI of the GB300-native Taylor-Hood P2/P1 Navier-Stokes stepper.
 *
 * One time step is the backward-Euler Oseen linearisation of the unsteady
 * incompressible Navier-Stokes equations (paper, Sec. 2.1 Eq. (3) and
 * Sec. 2.2.1, the Oseen equation with the convecting velocity lagged to
 * u_h^n): find u in V_h = [P2]^d, p in Q_h = P1 with
 *     ((u - u^n)/dt, v) + ((u^n . grad) u, v) + nu (grad u, grad v)
 *       - (p, div v) = (f^{n+1}, v),        (div u, q) = 0.
 * The library assembles this system on the GPU into a fixed sparsity
 * pattern and solves it with a right-preconditioned flexible GMRES(m)
 * (the paper's linear solver module, Sec. 3.2: GMRES).
 *
 * Conventions for every call:
 *  - Ownership: the library owns every handle and every device buffer it
 *    allocates; pointers passed in are borrowed for the duration of the call
 *    and are never freed by the library.
 *  - Device pointers are CUDA global-memory pointers on the current device;
 *    host pointers are plain malloc/numpy memory.  Each argument says which.
 *  - Streams: a problem runs every launch on the cudaStream_t given at
 *    creation (NULL = the legacy default stream).  Calls return when the
 *    work is enqueued unless they say they synchronise.
 *  - Errors: every call returns an fs_status; FS_OK is 0.  A message with
 *    details is available from fs_last_error() (thread-local, valid until
 *    the next call on the same thread).  Device-side failures (iteration
 *    caps, NaN/Inf, bounded waits that ran out) come back as status codes;
 *    no kernel traps.
 *  - Layouts: unknown vectors are component-blocked
 *    [u_x (n_p2) | u_y (n_p2) | u_z (n_p2, 3D only) | p (n_vert)], FP64.
 *    P2 node ids: vertices first (0..n_vert-1), then edge midpoints in the
 *    lexicographic order of their (min,max) vertex pairs.
 */
#ifndef FS_H
#define FS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FS_OK = 0,
  FS_ERR_INVALID_ARG = 1,
  FS_ERR_INVALID_MESH = 2,
  FS_ERR_OOM = 3,
  FS_ERR_CUDA = 4,
  FS_ERR_NOT_CONVERGED = 5,
  FS_ERR_NUMERIC = 6,
  FS_ERR_TIMEOUT = 7,
  FS_ERR_BUSY = 8,
  FS_ERR_UNSUPPORTED = 9
} fs_status;

/* Built-in manufactured problems (the paper's problem library, Sec. 3.1
 * "MathModel"; solutions of Sec. 3.3 and Sec. 4.1). */
typedef enum {
  FS_PROBLEM_UNSTEADY_BENCH = 0, /* 2D, Sec. 4.1: u1 = 2 pi sin t sin^2(pi x)
                                    sin(pi y) cos(pi y), u2 = -2 pi sin t
                                    sin(pi x) cos(pi x) sin^2(pi y),
                                    p = 20 sin t (x^2 y - 1/6)            */
  FS_PROBLEM_STEADY_POLY = 1,    /* 2D, Sec. 3.3 polynomial solution (no
                                    time derivative in f)                 */
  FS_PROBLEM_CHANNEL = 2,        /* 2D channel [0,2.2]x[0,0.41]: Poiseuille
                                    inflow U_max = 1.5, f = 0             */
  FS_PROBLEM_CUBE = 3,           /* 3D: u = sin t curl(Phi (1,1,1)),
                                    Phi = sin^2(pi x) sin^2(pi y) sin^2(pi z),
                                    p = sin t (x^2 y z - 1/12)            */
  FS_PROBLEM_POLY_OSEEN = 4,     /* u in P2 (div-free), p in P1, constant
                                    convecting field wconst (exactness)   */
  FS_PROBLEM_POLY_OSEEN_T = 5,   /* (1 + t) times the fields of problem 4:
                                    affine in time, so backward Euler
                                    reproduces it exactly at every step
                                    (checks the time level of f, of the
                                    Dirichlet data and of the pin)        */
  FS_PROBLEM_POLY3 = 6           /* 2D: u = (x^3, -3 x^2 y) (div-free, P3),
                                    p = x^2 - y^2 (P2), constant convecting
                                    field wconst: exact for P3/P2         */
} fs_problem_kind;

typedef enum {
  FS_PREC_FP64 = 0,        /* everything in FP64 (the plain FP64 path)     */
  FS_PREC_FP32_REFINE = 1  /* FP32 inner FGMRES + preconditioner, FP64
                              iterative refinement on r = b - A x          */
} fs_precision;

/* Dirichlet side bits: 1 x=lo, 2 x=hi, 4 y=lo, 8 y=hi, 16 z=lo, 32 z=hi. */
typedef struct {
  int dim;             /* 2 (triangles) or 3 (tetrahedra)                   */
  int n[3];            /* cells per axis (n[2] ignored in 2D), each >= 1    */
  double lo[3], hi[3]; /* box corners                                       */
  double jitter;       /* interior vertices move by jitter*h*(2U-1) per axis,
                          U from SplitMix64(seed ^ (3 v + axis)); < 0.25   */
  uint64_t seed;
  int dirichlet_sides; /* bit mask of sides carrying Dirichlet velocity      */
} fs_mesh_desc;

typedef struct fs_mesh fs_mesh;
typedef struct fs_problem fs_problem;

/* Builds a structured simplicial mesh (Sec. 2.2.1: a conforming mesh T_h;
 * Sec. 3.3: init_mesh['uniform_tri']): 2 triangles per square split along
 * v00-v11, or the 6 Kuhn tetrahedra per cube, the P2/P1 DOF map and the
 * block CSR patterns with their per-element slot tables.  Host memory only
 * until a problem is created on it.  Fails with FS_ERR_INVALID_MESH when a
 * simplex is degenerate (|det J| <= 1e-12 h^d).  *out receives the handle. */
int fs_mesh_create(const fs_mesh_desc* desc, fs_mesh** out);
int fs_mesh_destroy(fs_mesh* mesh);

/* A batch: `count` independent structured meshes (same dim) numbered as one
 * mesh with several disconnected pieces: all vertices instance by instance,
 * then all edge nodes, then all cells.  Every later call treats the batch
 * like one mesh; each kernel launch covers every instance.  descs is a host
 * array of count descriptions.  Errors as fs_mesh_create. */
int fs_mesh_create_batch(const fs_mesh_desc* descs, int count, fs_mesh** out);

/* Where each instance sits in the union numbering.  offsets (host, 6 int64
 * per instance, may be NULL): first vertex, vertex count, first edge node
 * (union P2 id), edge node count, first cell, cell count.  Returns the number
 * of instances, or a negative status. */
int fs_mesh_instances(const fs_mesh* mesh, int64_t* offsets);

/* Sizes of the Taylor-Hood P2/P1 discretisation (Sec. 2.2.1, V_h and Q_h
 * with k = 2).  nnz counts the monolithic saddle-point CSR
 *   [A 0 -Bx^T; 0 A -By^T; Bx By D] (3D analogous) with an explicit
 * pressure diagonal D; nnz_a, nnz_b count the scalar P2-P2 block and one
 * P1-P2 divergence block. */
typedef struct {
  int dim, nloc;
  int64_t n_vert, n_edge, n_p2, n_cell, n_dof, nnz, nnz_a, nnz_b;
} fs_dofmap_info;

/* DOF map export (Sec. 3.1 "DOF management").  Every output pointer is a
 * host pointer and may be NULL to skip it:
 *   coords   n_vert x dim   FP64 vertex coordinates
 *   cell2dof n_cell x nloc  P2 node ids per cell: vertices, then edges
 *                           (triangle (1,2),(2,0),(0,1); tetrahedron
 *                           (0,1),(0,2),(0,3),(1,2),(1,3),(2,3))
 *   rowptr   n_dof + 1      int64 monolithic CSR row pointers
 *   col      nnz            int32 columns, strictly ascending per row
 *   dirichlet n_p2          1 for Dirichlet P2 nodes
 * info (required) receives the sizes. */
int fs_dof_map(const fs_mesh* mesh, fs_dofmap_info* info, double* coords,
               int32_t* cell2dof, int64_t* rowptr, int32_t* col,
               uint8_t* dirichlet);

typedef struct {
  int problem;       /* fs_problem_kind                                     */
  double nu;         /* kinematic viscosity                                 */
  double dt;         /* time step (> 0)                                     */
  double t0;         /* initial time                                        */
  int precision;     /* fs_precision                                        */
  int pin_pressure;  /* 1: pressure row of vertex 0 -> identity holding
                        p_exact(x_0, t) (all-Dirichlet boundaries)          */
  int init;          /* 0: u^0 = I_h u(., t0); 1: zero inside, exact on
                        Dirichlet nodes                                     */
  double wconst[3];  /* constant convecting field (FS_PROBLEM_POLY_OSEEN)   */
  int deterministic; /* 1: the per-step convection assembly adds into the
                        matrix colour by colour (cells of a colour share no
                        node) without atomics, so every run of a problem
                        gives bit-identical systems and states (every other
                        part of the step always sums in a fixed order);
                        0: one launch with FP64 atomics, faster (channel
                        512x96: 0.09 vs 0.17 ms; cube 48^3: 2.3 vs 3.9 ms)
                        and equal to rounding                            */
} fs_problem_desc;

/* Creates a device-resident problem on `mesh` (which must outlive it):
 * uploads the mesh tables, assembles the step-invariant parts (P2 mass,
 * viscous and divergence blocks, the P1 pressure Laplacian and lumped mass)
 * and builds the multigrid hierarchies of the preconditioner.  `stream` is
 * a cudaStream_t (NULL = default stream).  Synchronises. */
int fs_problem_create(fs_mesh* mesh, const fs_problem_desc* desc,
                      void* stream, fs_problem** out);
int fs_problem_destroy(fs_problem* prob);

/* Problem on a batched mesh: one description per instance (host array of
 * count = number of instances).  The instances may differ in nu and
 * pin_pressure only.  Every instance runs its own Arnoldi process (own
 * Hessenberg matrix, rotations, convergence test), so its iterates do not
 * depend on the other instances; the launches are shared.  fs_problem_create
 * on a batched mesh applies one description to all instances. */
int fs_problem_create_batch(fs_mesh* mesh, const fs_problem_desc* descs,
                            int count, void* stream, fs_problem** out);

/* A Taylor-Hood P3/P2 problem on a single 2D mesh (paper Sec. 4.1, the
 * P3-P2 experiment, which the paper solves by IPCS): P3 velocity (vertices,
 * then two nodes per edge in the lexicographic order of the edges, the one
 * nearer the edge's smaller vertex first, then one interior node per cell)
 * and P2 pressure (vertices, then one node per edge).  State layout
 * [u_x (n3) | u_y (n3) | p (np)] in that numbering (fs_problem_sizes).
 * Assembles the step-invariant blocks on the GPU; stepped by fs_step_ipcs,
 * with fs_get_state / fs_set_state and fs_assemble_step (no export) also
 * available; the coupled solver calls answer FS_ERR_UNSUPPORTED.  dt must be
 * finite; FS_ERR_UNSUPPORTED for a batched or 3D mesh.  Synchronises. */
int fs_problem_create_p3(fs_mesh* mesh, const fs_problem_desc* desc, void* stream,
                         fs_problem** out);

/* Sizes of a problem's unknowns (host array of 3): velocity nodes per
 * component, pressure nodes, n_dof. */
int fs_problem_sizes(const fs_problem* prob, int64_t* sizes);

/* Assembles the Oseen system of the step t -> t_next (paper Sec. 2.2.1,
 * Oseen equation; BForm/LForm of Sec. 3.1) with the convecting velocity
 * w = u^n taken from the current state (or wconst), into the problem's
 * fixed block-CSR values, and the right-hand side
 *   b_u = M (u^n/dt + I_h f(t_next)),  b_p = 0,
 * with Dirichlet rows replaced by identity rows holding u_exact(t_next) and
 * the pinned pressure row holding p_exact(x_0, t_next).
 * val_out (device, FP64, monolithic nnz, may be NULL) receives the values in
 * the monolithic CSR order of fs_dof_map; b_out (device, FP64, n_dof, may be
 * NULL) the right-hand side. */
int fs_assemble_step(fs_problem* prob, double t_next, double* val_out,
                     double* b_out);

typedef struct {
  int restart;        /* GMRES(m) restart length m (must be 30)             */
  int max_iter;       /* cap on (inner) Krylov iterations per solve         */
  double rtol;        /* stop at ||b - A x||_2 <= rtol ||b||_2, FP64 true
                         residual; a residual that stops decreasing (a
                         restart cycle or refinement step that no longer
                         contracts) is accepted within 100 rtol, the
                         rounding floor of the system                      */
  double inner_rtol;  /* FP32 inner solve tolerance (precision mode)        */
  int max_refine;     /* cap on FP64 refinement steps (precision mode)      */
  int use_graph;      /* 1: replay restart cycles as captured CUDA graphs   */
} fs_solve_opts;

typedef struct {
  int iters;          /* Krylov iterations (inner ones in precision mode);
                         over a batch: the largest of the instances        */
  int refinements;    /* FP64 refinement steps (0 in FP64 mode)             */
  int status;         /* fs_status of the solve                             */
  int cycles;         /* GMRES restart cycles                               */
  double rel_res;     /* final FP64 ||b - A x|| / ||b||                     */
} fs_solve_stats;

/* Fills opts with the defaults: m = 30, max_iter 2000, rtol 1e-14, inner_rtol
 * 1e-5, max_refine 30, use_graph 1. */
void fs_default_solve_opts(fs_solve_opts* opts);

/* Solves the system last assembled by fs_assemble_step (paper Sec. 3.2,
 * GMRES) with right-preconditioned flexible GMRES(m); the preconditioner is
 * block upper-triangular: Cahouet-Chabard Schur approximation
 * nu Mp^-1 + dt^-1 Kp^-1 and a multigrid V-cycle on the velocity block.
 * x (device, FP64, n_dof) holds the initial guess and receives the solution;
 * NULL means the problem's state vector.  Synchronises.  stats may be NULL.
 * Returns FS_ERR_NOT_CONVERGED (with the best iterate kept) when max_iter or
 * max_refine is reached first, FS_ERR_NUMERIC on NaN/Inf. */
int fs_solve(fs_problem* prob, const fs_solve_opts* opts, double* x,
             fs_solve_stats* stats);

/* nsteps backward-Euler Oseen steps: assemble (w = u^n), solve, t += dt.
 * Each solve starts from the polynomial extrapolation in time through x^n
 * and up to four previous states (5 x^n - 10 x^(n-1) + 10 x^(n-2)
 * - 5 x^(n-3) + x^(n-4) once they are known, lower orders before, and x^n
 * after problem creation, fs_solve, or fs_set_state to a time other than
 * the current one); the converged state
 * does not depend on the starting point beyond the solver tolerance.
 * per_step (host, nsteps entries, may be NULL) receives each solve's stats.
 * Synchronises. */
int fs_step(fs_problem* prob, int nsteps, const fs_solve_opts* opts,
            fs_solve_stats* per_step);

/* Non-blocking time stepping for callers that drive several problems at
 * once (the serving loop): fs_step_begin enqueues the first step's assembly
 * and the first device part of its solve and returns; fs_step_poll advances
 * the solve's state machine by every part that has completed (wait = 0:
 * never blocks; wait = 1: blocks until the next part completes) and sets
 * *done when all nsteps are finished, returning their status then.  One step
 * sequence per problem at a time (FS_ERR_BUSY otherwise). */
int fs_step_begin(fs_problem* prob, int nsteps, const fs_solve_opts* opts);
int fs_step_poll(fs_problem* prob, int wait, int* done);

/* Picard iteration of the nonlinear step (paper Sec. 2.2.1: the convection
 * term linearised around the latest iterate, ((u^k . grad) u^{k+1}, v), one
 * Oseen solve per iterate; Sec. 3.3: model.run(maxstep, tol) iterates until
 * the change falls below tol).  Iterate k convects with u^k (u^0 = u^n) and
 * keeps u^n in the backward-Euler load; it stops when
 *   ||u^{k+1} - u^k||_2 <= nl_tol * max(1, ||u^{k+1}||_2)
 * (velocity entries, FP64) or after max_picard solves.  One iteration is
 * exactly the Oseen step of fs_step.  Each linear solve is fs_solve's
 * (options opts, NULL = defaults); the first of a time step starts from the
 * extrapolated state history, later ones from the latest iterate.
 * Single problems only (FS_ERR_UNSUPPORTED on a batch).  Synchronises. */
typedef struct {
  int picard_iters;   /* linear solves taken                               */
  int krylov_iters;   /* their Krylov iterations, summed                   */
  int status;         /* fs_status: FS_ERR_NOT_CONVERGED when max_picard
                         solves did not reach nl_tol (last iterate kept)  */
  double update;      /* last ||u^{k+1} - u^k|| / max(1, ||u^{k+1}||)      */
  double rel_res;     /* FP64 relative residual of the last linear solve   */
} fs_picard_stats;

/* nsteps time steps, each iterated to nl_tol; per_step (host, nsteps
 * entries, may be NULL).  The time advances by dt per step even when a
 * step's iteration fails (its last iterate is kept), as in fs_step.  Needs
 * a finite dt. */
int fs_step_picard(fs_problem* prob, int nsteps, const fs_solve_opts* opts, double nl_tol,
                   int max_picard, fs_picard_stats* per_step);

/* The steady problem (the Sec. 3.3 example: no time derivative): a problem
 * created with dt = inf (no mass term in the operator, the load or the
 * preconditioner's Schur part) is iterated at its fixed time t0 from its
 * current state.  stats may be NULL.  FS_ERR_INVALID_ARG for a finite dt;
 * fs_step refuses dt = inf. */
int fs_solve_steady(fs_problem* prob, const fs_solve_opts* opts, double nl_tol,
                    int max_picard, fs_picard_stats* stats);

/* Incremental pressure-correction stepping (paper Sec. 2.2.1, IPCS, with
 * density 1): each step solves, in this order,
 *   1. (u* - u^n)/dt + ((w . grad) u^n, v) + nu (grad u*, grad v)
 *        - (p^n, div v) = (f^{n+1}, v)      (w = u^n, convection explicit;
 *                                             u* = u_D(t^{n+1}) on the boundary)
 *   2. (grad dp, grad q) = -(1/dt) (div u*, q),  dp = p^{n+1} - p^n
 *        (the pinned vertex takes p_exact(x_0, t^{n+1}) - p^n(x_0); the
 *        paper prints the right-hand side with the opposite sign, which
 *        contradicts its own step 3)
 *   3. (u^{n+1} - u*, v)/dt = -(grad dp, v)  (u^{n+1} = u_D(t^{n+1}) on the
 *        boundary), p^{n+1} = p^n + dp.
 * The three systems (M/dt + nu K, the P1 Laplacian, M) are symmetric
 * positive definite once their boundary unknowns are eliminated; each is
 * solved in FP64 by Jacobi-preconditioned conjugate gradients to a relative
 * residual of rtol (checked every 8 iterations; FS_ERR_NOT_CONVERGED when
 * the true residual is above 100 rtol after max_iter iterations), whatever
 * the problem's precision.  Needs a single problem with Dirichlet velocity on
 * the whole boundary and the pressure pin (FS_ERR_UNSUPPORTED otherwise).
 * per_step (host, nsteps entries, may be NULL).  Synchronises. */
typedef struct {
  int iters[3];       /* CG iterations of the three stages                  */
  int status;         /* fs_status of the step                             */
  double rel_res[3];  /* their true relative residuals                     */
} fs_ipcs_stats;
int fs_step_ipcs(fs_problem* prob, int nsteps, double rtol, int max_iter,
                 fs_ipcs_stats* per_step);

/* Per-instance statistics of the last solve (host array, one entry per
 * instance). */
int fs_instance_stats(const fs_problem* prob, fs_solve_stats* per_instance);

/* y = A x with the assembled FP64 saddle-point operator (device FP64
 * vectors of n_dof entries). */
int fs_apply_operator(fs_problem* prob, const double* x, double* y);

/* State access: x (n_dof FP64) and the current time.  x_out/x_in are host
 * pointers when `host` is 1, device pointers otherwise.  Synchronises.
 * fs_set_state at the problem's current time continues the stepped history
 * (the initial guess of fs_step extrapolates from the previous state); at
 * another time it starts a new history. */
int fs_get_state(fs_problem* prob, double* x_out, int host, double* t_out);
int fs_set_state(fs_problem* prob, const double* x_in, int host, double t);

/* Sizes of the problem's device footprint in bytes (HBM admission). */
int64_t fs_problem_device_bytes(const fs_problem* prob);

/* ---- Continuous-batching request loop (no counterpart in the paper: its
 * workflow runs one simulation at a time, Sec. 3.1 ComputationModel). ----
 * Requests wait in a FIFO queue and are admitted while a slot is free and
 * their estimated device footprint fits in the budget left by the resident
 * requests.  Admitted requests are set up by host worker threads, then
 * stepped through fs_step_begin / fs_step_poll on their own streams, so the
 * work of all resident requests overlaps on the device.  Times are the
 * caller's clock (seconds), passed to submit and progress. */
typedef struct fs_server fs_server;
typedef struct {
  int64_t hbm_budget;   /* bytes of device memory the resident requests may use */
  int max_slots;        /* resident requests at most                          */
  int setup_threads;    /* host threads setting requests up (<= 0: 4)        */
} fs_server_desc;
typedef struct {
  int64_t id;
  int status;           /* fs_status of the request                           */
  int nsteps, iters;    /* steps run; Krylov iterations of its last step      */
  double arrival, admitted, started, finished;  /* caller clock, seconds     */
  int64_t device_bytes; /* measured footprint                                 */
} fs_request_result;
int fs_server_create(const fs_server_desc* desc, fs_server** out);
/* Destroys the server and every request still queued or resident. */
int fs_server_destroy(fs_server* server);
/* Queues one request (host descriptions, copied).  keep_state = 1 keeps the
 * final state on the host for fs_server_take_state.  *id receives its id.
 * FS_ERR_OOM when its estimate alone exceeds the budget. */
int fs_server_submit(fs_server* server, const fs_mesh_desc* mesh,
                     const fs_problem_desc* problem, int nsteps, double arrival,
                     int keep_state, int64_t* id);
/* Admits, starts and advances requests without blocking; *n_completed
 * receives the number of requests that finished in this call. */
int fs_server_progress(fs_server* server, double now, int* n_completed);
/* Moves up to max finished-request records into out (host); *n = count. */
int fs_server_pop_completed(fs_server* server, fs_request_result* out, int max,
                            int* n);
/* Copies the kept final state (n_dof FP64, host) of a finished request. */
int fs_server_take_state(fs_server* server, int64_t id, double* x, int64_t n);
int fs_server_status(const fs_server* server, int* queued, int* resident,
                     int64_t* bytes_reserved);
/* The admission estimate of a request's device footprint in bytes. */
int64_t fs_server_estimate_bytes(const fs_mesh_desc* mesh, int precision);

/* FP64 residual check of a monolithic CSR system (the format fs_dof_map and
 * fs_assemble_step export; paper Sec. 3.1, the error step after the linear
 * solver): out2[0] = ||b - A x||_2, out2[1] = ||b||_2.
 *   n       rows (>= 1); rowptr (n + 1, int64), col (int32), val (FP64),
 *           x, b (n, FP64): device pointers, borrowed;
 *   out2    host pointer to 2 doubles;
 *   stream  cudaStream_t (NULL = default stream).
 * Per-block partial sums go to stream-ordered scratch (cudaMallocAsync,
 * freed before return).  Synchronises the stream.  FS_ERR_INVALID_ARG on a
 * null pointer or n < 1, FS_ERR_OOM / FS_ERR_CUDA on runtime failures. */
int fs_csr_residual_norm(int64_t n, const int64_t* rowptr, const int32_t* col,
                         const double* val, const double* x, const double* b,
                         double* out2, void* stream);

/* The same residual check for callers that cannot allocate device memory
 * (the paper has no counterpart: it is a deployment aid).  Serving processes
 * whose device memory is already committed to resident problems under a
 * fixed budget, and host applications that forbid libraries to grow their
 * device footprint after start-up, cannot call cudaMalloc when they want to
 * check a solution; this entry point calls no allocator at all.  Its scratch is a fixed array in the library's static device memory
 * (about 128 KB, held by every GPU that loads the library until the process
 * exits), sized for systems of at most 4,194,304 rows: larger n returns
 * FS_ERR_INVALID_ARG with a message, before any device work.  Arguments,
 * results and errors are those of fs_csr_residual_norm.
 * Set-up: the first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  The address is cached per device for the
 * life of the process and does not survive a cudaDeviceReset of that
 * device.  Like fs_csr_residual_norm, the call waits for its stream to
 * finish (it copies the two norms to the host before returning).  Every
 * call shares the one array and clears
 * what must start at zero itself; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller. */
int fs_csr_residual_norm_noalloc(int64_t n, const int64_t* rowptr,
                                 const int32_t* col, const double* val,
                                 const double* x, const double* b,
                                 double* out2, void* stream);

/* Execution schedule of the multigrid preconditioner (no counterpart in
 * the paper, whose solver is a library call).  The levels of a hierarchy
 * with at most tail_rows rows (and every level below them) run as one kernel
 * on one thread-block cluster, their passes separated by cluster barriers;
 * larger levels run one kernel per pass.  0 = no fused levels.  The choice
 * changes launch counts and timing only: results are identical (the same
 * per-row arithmetic in the same order).
 * fs_set_schedule drops the problem's captured CUDA graphs (they are
 * re-captured by the next solve); FS_ERR_BUSY while a step is in progress.
 * fs_autotune times one application of the preconditioner (a CUDA graph of
 * `reps` applications, CUDA events) for every pair of candidate thresholds
 * {0, 4096, 16384, 65536} of the velocity and pressure hierarchies and both
 * smoothing group depths, and the saddle-point SpMV (`reps` launches) for
 * every SpMV group depth, then the persistent form of the preconditioner
 * (persistent_precond = 1) against the best of those; it installs the
 * fastest of each and reports them.  Leaves the state and assembled system
 * unchanged.  Synchronises. */
typedef struct {
  int64_t tail_rows_velocity;
  int64_t tail_rows_pressure;
  int32_t spmv_group;    /* SELL slots a thread issues together in the SpMV:
                            4, 6 or 8; 0 = 6 in FP32, 4 in FP64 */
  int32_t smooth_group;  /* ... in the smoothing passes: 4 or 6; 0 = 4    */
  int32_t coarse_degree; /* degree of the Chebyshev smoother on the levels
                            below the finest (pre and post): 3, 2 or 1;
                            0 = 2 (1: the first step of the restriction is
                            the pre-smoothing, one step after the
                            correction the post-smoothing; not with the
                            fused tail, which then stays off, nor with the
                            persistent form).  Unlike the other fields it
                            changes the
                            preconditioner, so iteration counts (not the
                            solution beyond rtol) depend on it; the
                            autotuner keeps the value in place          */
  int32_t serial_launches; /* 0: the solver's kernels are launched as
                            programmatic dependent launches (a kernel may
                            be scheduled while its predecessor drains and
                            waits for that predecessor's completion before
                            its first memory access); 1: plain serialised
                            launches.  Timing only: results are identical.
                            The autotuner keeps the value in place       */
  int32_t persistent_precond; /* 1: each application of the block
                            preconditioner is one persistent cooperative
                            kernel over a device work-list of (phase,
                            instance, row range) items, where an item waits
                            only for the previous phase of its own instance
                            (a batch's instances advance independently,
                            and instances that have converged are skipped);
                            0: one kernel per pass over all instances.  The
                            per-row arithmetic is the same (results agree
                            to rounding: the fused cluster tail and the
                            slot-group depth are not used in this mode, it
                            issues 4 slots at a time).  A wait that has not
                            ended after one second makes the solve return
                            FS_ERR_TIMEOUT.  fs_autotune times both forms */
  int32_t fine_degree;   /* degree of the Chebyshev smoother on the finest
                            level of both hierarchies (pre and post): 3, 2
                            or 1; 0 = 2.  Like coarse_degree it changes the
                            preconditioner (iteration counts, not the
                            solution beyond rtol); the autotuner keeps the
                            value in place                              */
  int32_t cheb_ratio;    /* the Chebyshev smoother targets the interval
                            [1.1 lmax / cheb_ratio, 1.1 lmax] of D^-1 A on
                            every level (lmax estimated at set-up): 2 to
                            64; 0 = 8.  It changes the preconditioner like
                            the degrees; fs_autotune_smoother picks it (and
                            the degrees) by timing steps                */
  int32_t schur;         /* approximation of the pressure Schur complement:
                            0 Cahouet-Chabard, S^-1 = nu Mp^-1 + dt^-1 Kp^-1;
                            1 pressure convection-diffusion,
                            S^-1 = Mp^-1 (Mp/dt + nu Kp + Np(w)) Kp^-1 with
                            Np(w) the convection by the step's w on the
                            pressure space (assembled with the system).
                            Changes the preconditioner like the degrees.
                            Not with persistent_precond (FS_ERR_UNSUPPORTED) */
} fs_schedule;
typedef struct {
  int candidates;        /* schedules timed                                  */
  double default_ms;     /* one preconditioner application, schedule before */
  double best_ms;        /* ... with the installed schedule                  */
  double spmv_default_ms;  /* one SpMV, schedule before                      */
  double spmv_best_ms;     /* ... with the installed schedule                */
  fs_schedule best;
  double persistent_ms;    /* one preconditioner application in the persistent
                              form, with the installed schedule's smoothing
                              degree (0 when it could not be timed)        */
} fs_tune_report;
int fs_get_schedule(const fs_problem* prob, fs_schedule* out);
int fs_set_schedule(fs_problem* prob, const fs_schedule* sched);
int fs_autotune(fs_problem* prob, int reps, fs_tune_report* report);
/* Picks the smoother (fs_schedule.cheb_ratio, coarse_degree, fine_degree)
 * by timing steps.  cand holds ncand triples (cheb_ratio, coarse_degree,
 * fine_degree); a 0 keeps that field of the installed schedule.  For each
 * candidate the problem's state is put back to the one at the call, one
 * untimed step captures the solver's graphs, the state is put back again
 * and nsteps steps are timed with CUDA events on the problem's stream.  The
 * fastest candidate is installed and the state at the call is restored,
 * with no step history (the next solves start as after fs_set_state at
 * another time).  ms_out / iters_out (host, ncand entries, may be NULL)
 * receive each candidate's mean time and inner iterations per step;
 * best_out (may be NULL) the installed schedule.  Callers can search the
 * fields one after the other (degrees, then the interval).  No counterpart
 * in the paper (its solver is a library call).  FS_ERR_INVALID_ARG for a
 * field out of its range (fs_set_schedule's), FS_ERR_UNSUPPORTED for P3/P2
 * problems or a degree of 1 with the persistent form, FS_ERR_BUSY while a
 * step is in progress, the first failing step's status otherwise (the state
 * is restored and the schedule left as it was).  Synchronises. */
int fs_autotune_smoother(fs_problem* prob, int nsteps, const int32_t* cand, int ncand,
                         double* ms_out, double* iters_out, fs_schedule* best_out);

/* Instrumentation (no counterpart in the paper).
 * fs_launch_count: kernels launched by this library since load, counting
 * every node of each replayed CUDA graph and every pass of a graph's
 * Arnoldi loop node (host-side counter).
 * fs_profile_kernel: times `reps` back-to-back launches of one hot kernel on
 * the problem's own data and stream with CUDA events (after 3 warm-up
 * launches) and returns the mean duration and the kernel's algorithmic bytes
 * per launch (each array it must touch counted once).  Kernel ids below;
 * kernel | FS_PROFILE_COLD_L2 times each launch alone (its own event pair)
 * after a read of twice the L2 size has filled the L2 with other data, so
 * every byte the kernel touches once comes from DRAM (its working set may
 * still be re-read from L2 within the launch); a temporary device buffer of
 * that size is allocated (stream-ordered) and freed.  Leaves the problem's
 * state and assembled system unchanged.  Synchronises. */
enum {
  FS_KERNEL_SPMV = 0,           /* saddle-point SpMV, solver arithmetic      */
  FS_KERNEL_SPMV_FP64 = 1,      /* saddle-point SpMV, FP64                   */
  FS_KERNEL_CHEB = 2,           /* fused Chebyshev step, finest P2 level     */
  FS_KERNEL_ASSEMBLE_CONV = 3,  /* per-step convection assembly (FP64)       */
  FS_KERNEL_PRECOND = 4,        /* one block-preconditioner application in
                                   the solver arithmetic, timed as a CUDA
                                   graph of `reps` applications; alg_bytes
                                   is 0 (a latency unit of many kernels)   */
  FS_KERNEL_CGS = 5,            /* one CGS2 orthogonalisation (its three
                                   passes) at Arnoldi step j = m/2 on the
                                   Krylov scratch; alg_bytes counts the
                                   3j + 8 vector sweeps the passes must make
                                   (each vector once per pass)            */
  FS_KERNEL_CGS_DOT = 6,        /* its first pass alone (h = V^T w):
                                   j + 2 sweeps                           */
  FS_KERNEL_CGS_UPD = 7,        /* its second pass alone (w -= V h, re-dot,
                                   norm): j + 3 sweeps                    */
  FS_KERNEL_CGS_FIN = 8,        /* its third pass alone (w -= V h2,
                                   normalise): j + 3 sweeps               */
  FS_PROFILE_COLD_L2 = 0x100    /* flag: L2-cold timing, see above        */
};
int64_t fs_launch_count(void);
int fs_profile_kernel(fs_problem* prob, int kernel, int reps, double* avg_ms,
                      double* alg_bytes);

const char* fs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FS_H */
