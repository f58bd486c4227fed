/*
 * sem.h -- C ABI of the GB300 (sm_103a) SEM Poisson/Helmholtz hot path.
 *
 * The library implements the data-parallel hot path of the spectral element
 * pressure/Helmholtz solve scaled in Vincent et al., "Strong Scaling of
 * OpenACC enabled Nek5000 on several GPU based HPC systems" (arXiv
 * 2109.03592):
 *
 *   - the matrix-free local operator w = A_L u of Alg. 1 (tensor-product
 *     derivative contractions with the GLL matrix D along r, s, t, the
 *     pointwise product with the geometric factors g1..g6 and h1, the D^T
 *     back-contractions) plus the h2 * B mass term of the Helmholtz problem
 *     (Sec. 2, Eq. 4);
 *   - direct stiffness summation QQ^T over shared GLL nodes, the "exchange of
 *     element face values" of Sec. 2, followed by the Dirichlet mask;
 *   - Jacobi-preconditioned conjugate gradients (Sec. 2: "iterative solvers
 *     with proper preconditioners"), in FP64 and as FP32-inner / FP64-outer
 *     iterative refinement;
 *   - a request server that solves many such problems concurrently;
 *
 * and, around that path:
 *
 *   - per-point coefficients h1(x), h2(x) for the velocity Helmholtz solves
 *     of Sec. 2, Eq. 4 (sem_mesh_set_coefficients);
 *   - projection of the initial guess onto previous solutions (sem_proj_*);
 *   - the P_N - P_{N-2} pressure operator E = D B^-1 D^T of Sec. 2, Eq. 5,
 *     and its CG (sem_pressure_*);
 *   - the overlapping Schwarz preconditioner of Sec. 2, Eq. 6, with a coarse
 *     grid solve (sem_schwarz_*).
 *
 * Conventions shared by every entry point:
 *
 *   Local vectors ("E-vectors") hold one value per element-local GLL point,
 *   duplicated on shared faces/edges/vertices, in the layout of Alg. 1's
 *   u(i,j,k,e): index l = i + n*(j + n*(k + n*e)), n = N+1, contiguous.  They
 *   are FP64 (double) unless an entry point's `prec` says SEM_FP32 (float).
 *
 *   `_dev` pointers are device pointers on the current CUDA device, owned by
 *   the caller (for example PyTorch tensors passed by data_ptr()).  `_host`
 *   pointers are host memory owned by the caller.  The library owns every
 *   array inside a sem_mesh / sem_server.
 *
 *   `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *   asynchronous on it unless stated otherwise.
 *
 *   Every call returns a sem_status and never aborts; on failure
 *   sem_last_error() gives a message for the calling thread.  No call falls
 *   back to CPU computation: without a usable GPU the calls fail with
 *   SEM_ERR_CUDA.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SEM_OK = 0,
  SEM_ERR_INVALID = 1,        /* bad argument or descriptor */
  SEM_ERR_OOM = 2,            /* device allocation failed, or a request exceeds the server's HBM budget */
  SEM_ERR_CUDA = 3,           /* a CUDA call failed (text in sem_last_error) */
  SEM_ERR_NOT_CONVERGED = 4,  /* maxit reached before the tolerance */
  SEM_ERR_BREAKDOWN = 5,      /* p^T A p <= 0 or NaN inside CG */
  SEM_ERR_BUSY = 6,           /* server queue full */
  SEM_ERR_DEVICE_TIMEOUT = 7, /* a bounded device-side wait gave up */
  SEM_ERR_BAD_MESH = 8,       /* inverted element (det J <= 0) or inconsistent topology */
  SEM_ERR_TIMEOUT = 9,        /* sem_server_poll: result not ready within timeout */
  SEM_ERR_NOT_FOUND = 10,     /* unknown request id */
  SEM_ERR_CANCELLED = 11      /* request cancelled before it finished */
} sem_status;

typedef enum { SEM_FP64 = 0, SEM_FP32 = 1, SEM_MIXED = 2 } sem_prec;

typedef enum { SEM_MESH_BOX = 0, SEM_MESH_PIPE = 1, SEM_MESH_EXPLICIT = 2 } sem_mesh_kind;

/*
 * Mesh descriptor (Sec. 2: non-overlapping, body-conforming hexahedra; Sec. 4.2:
 * straight pipe flow case).  Element faces are numbered 0: i=0, 1: i=N,
 * 2: j=0, 3: j=N, 4: k=0, 5: k=N; element corner c = a + 2b + 4d sits at
 * (i, j, k) = (a N, b N, d N).
 *
 * SEM_MESH_BOX: [0,lx]x[0,ly]x[0,lz], nx*ny*nz affine elements ordered
 *   e = ex + nx (ey + ny ez), homogeneous Dirichlet on all six faces.
 * SEM_MESH_PIPE: O-grid straight pipe of radius R and length L: a central
 *   square of half-width a with nc x nc elements and four curved blocks of
 *   nc (tangential) x nr (radial) elements; in the +x block the point with
 *   tangential s in [-1,1] and radial t in [0,1] is
 *   (1-t)(a, a s) + t R (cos(pi s/4), sin(pi s/4)), the other blocks are its
 *   rotations by 90/180/270 degrees; radial levels
 *   t_k = 1 - tanh(beta(1-k/nr))/tanh(beta); nzp uniform layers in z.
 *   Element e = layer * nc(nc+4nr) + e2d; square elements first
 *   (e2d = ey nc + ex, i along x, j along y), then blocks q = 0..3
 *   (e2d = nc^2 + q nc nr + r nc + m; i runs outward, j along s); k along z.
 *   Dirichlet on the wall (face 1 of the outermost ring); periodic in z when
 *   periodic_z != 0 (then nzp >= 3), else Dirichlet end caps too.
 * SEM_MESH_EXPLICIT: E elements with host arrays xyz [E][3][n^3] (GLL point
 *   coordinates, component-major per element), vert [E][8] (global vertex
 *   ids per corner; shared corners share ids, periodic identifications too)
 *   and dirichlet_face [E][6] (nonzero = Dirichlet face).  The arrays are
 *   read during sem_mesh_create only.
 */
typedef struct {
  int kind; /* sem_mesh_kind */
  int N;    /* polynomial order, 1 <= N <= 11 */
  int nx, ny, nz;
  double lx, ly, lz;
  int nc, nr, nzp;
  double R, L, a, beta;
  int periodic_z;
  int64_t E;
  const double* xyz;
  const int64_t* vert;
  const uint8_t* dirichlet_face;
} sem_mesh_desc;

typedef struct sem_mesh sem_mesh;

typedef struct {
  int64_t E;            /* elements */
  int N;                /* order */
  int64_t n_local;      /* E (N+1)^3 */
  int64_t n_global;     /* distinct GLL nodes */
  int64_t n_segments;   /* gather-scatter segments (shared or Dirichlet nodes) */
  int64_t n_seg_points; /* local points inside those segments */
  size_t dev_bytes;     /* device memory held by the mesh */
} sem_mesh_info_t;

/* Build a mesh on the current device: coordinates, geometric factors
 * g1..g6 and B (FP64, plus FP32 copies), the first-touch global numbering,
 * the gather-scatter plan, multiplicities, the Dirichlet mask and the
 * assembled diagonals used by the Jacobi preconditioner.  Synchronous.
 * SEM_ERR_BAD_MESH if some det J <= 0 or the topology is inconsistent;
 * SEM_ERR_INVALID for a bad descriptor (N outside 1..11, empty or
 * inconsistent sizes) or a mesh of 2^31 or more local points (the
 * gather-scatter plan holds 32-bit local indices); SEM_ERR_OOM. */
sem_status sem_mesh_create(const sem_mesh_desc* desc, void* stream, sem_mesh** out);
sem_status sem_mesh_destroy(sem_mesh* mesh);
sem_status sem_mesh_info(const sem_mesh* mesh, sem_mesh_info_t* info);

/* Global id of every local point, assigned in order of first appearance when
 * local points are scanned in ascending local index (host output, n_local
 * int64).  Two local points share an id iff they are the same GLL node. */
sem_status sem_mesh_global_ids(const sem_mesh* mesh, int64_t* host_out);

/* Copies of mesh data into caller buffers (device, FP64, local layout):
 * coordinates [E][3][n^3]; factors G [E][6][n^3] (g1..g6 = G_rr, G_ss, G_tt,
 * G_rs, G_rt, G_st of w_i w_j w_k detJ J^{-1} J^{-T}); B [E][n^3]
 * (w_i w_j w_k detJ); multiplicity and mask [n_local] (mask = 0 on Dirichlet
 * nodes, 1 elsewhere).  Any output pointer may be NULL to skip it. */
sem_status sem_mesh_coords(const sem_mesh* mesh, double* xyz_dev, void* stream);
sem_status sem_mesh_geometry(const sem_mesh* mesh, double* G_dev, double* B_dev, void* stream);
sem_status sem_mesh_weights(const sem_mesh* mesh, double* mult_dev, double* mask_dev, void* stream);

/* Per-point operator coefficients.  Alg. 1 scales the contracted gradient
 * G (ur, us, ut) at every local point by that point's h1(i,j,k,e); the
 * Helmholtz term of Sec. 2, Eq. 4 is read the same way with a per-point h2
 * (variable viscosity and mass coefficient).
 *   h1_dev, h2_dev: device FP64 arrays of n_local values in the local layout
 *   [E][n^3], read during the call and not kept; NULL means 1 at every point.
 * From then on every operator entry point on this mesh (sem_ax, sem_apply,
 * sem_jacobi, the solvers, batches, projection spaces) applies
 *   h1_eff(q) = h1 * h1_dev[q],  h2_eff(q) = h2 * h2_dev[q]
 * with the scalar h1, h2 that the call passes.  Both NULL restores the
 * constant-coefficient operator.  The factors are stored pre-multiplied
 * (h1 G, h2 B in FP64, FP32 and the FP32 pair form: 128 B per local point
 * with both), so the operator kernels read no more bytes than without.
 * sem_mesh_geometry and sem_rhs keep using the plain G and B.
 * A projection space on the mesh drops its basis at its next solve.
 * Errors: SEM_ERR_INVALID (null mesh; an h1 value <= 0 or an h2 value < 0 or
 * non-finite: the mesh keeps its previous coefficients), SEM_ERR_OOM.
 * Runs on `stream` and returns after the device finished; not to be called
 * while a solve, batch or server request on this mesh is in flight. */
sem_status sem_mesh_set_coefficients(sem_mesh* mesh, const double* h1_dev, const double* h2_dev, void* stream);

/* w = A_L u: Alg. 1 plus the Helmholtz term, element by element, with
 * h1 (scaling the stiffness after the G contraction) and h2 (scaling B u):
 * scalars, times the mesh's per-point coefficients if it has any.
 * No assembly and no mask.  u and w: local vectors of `prec` SEM_FP64 or
 * SEM_FP32 (SEM_FP32 uses the FP32 factors).  u and w must not overlap. */
sem_status sem_ax(const sem_mesh* mesh, const void* u_dev, void* w_dev, double h1, double h2,
                  sem_prec prec, void* stream);

/* v <- QQ^T v in place (sum over all copies of each node, in ascending local
 * index, written back to every copy); then, if apply_mask, v <- 0 on every
 * Dirichlet node.  Bit-reproducible.  prec SEM_FP64 or SEM_FP32. */
sem_status sem_gs(const sem_mesh* mesh, void* v_dev, sem_prec prec, int apply_mask, void* stream);

/* Right-hand side b = mask QQ^T (B f) from nodal forcing values f (FP64). */
sem_status sem_rhs(const sem_mesh* mesh, const double* f_dev, double* b_dev, void* stream);

/* Assembled operator y = mask QQ^T A_L x (FP64). */
sem_status sem_apply(const sem_mesh* mesh, const double* x_dev, double* y_dev, double h1, double h2,
                     void* stream);

/* Jacobi preconditioner M^{-1} = mask / QQ^T diag(A_L) for (h1, h2) (FP64;
 * 0 on Dirichlet nodes). */
sem_status sem_jacobi(const sem_mesh* mesh, double h1, double h2, double* minv_dev, void* stream);

typedef struct {
  double tol;       /* stop when ||r|| <= tol ||b||, ||v||^2 = sum_l v_l^2 / mult_l; default 1e-10 */
  double h1, h2;    /* operator coefficients (Poisson: 1, 0), times the mesh's per-point ones */
  double inner_tol; /* SEM_MIXED: relative tolerance of each FP32 inner solve; <= 0 picks the tuned value */
  int maxit;        /* iteration cap (per inner solve for SEM_MIXED); <= 0 means 20000 */
  int max_outer;    /* SEM_MIXED: refinement steps cap; <= 0 means 50 */
  int prec;         /* SEM_FP64 (plain PCG) or SEM_MIXED (FP32 inner / FP64 outer); SEM_FP32 = plain FP32 PCG */
  int refine;       /* SEM_MIXED: 0 = reliable updates (CG direction kept across FP64 residual
                       replacements; Sleijpen & van der Vorst 1996), 1 = restarted refinement
                       (defect correction: a fresh FP32 PCG on each FP64 residual) */
  double delta;     /* SEM_MIXED, refine = 0: replace the residual when the FP32 one has dropped by
                       this factor since the last replacement; <= 0 means 0.3 (sem_pcg_solve) or
                       0.1 (batched and served solves, where a replacement costs a host round trip) */
  int precond;      /* sem_pressure_solve: SEM_PRECOND_DEFAULT (0) or SEM_PRECOND_JACOBI = diag(E)^-1,
                       SEM_PRECOND_NONE = plain CG.  The velocity solvers are Jacobi-preconditioned
                       always and ignore it. */
} sem_solve_opts;

#define SEM_PRECOND_DEFAULT 0
#define SEM_PRECOND_NONE 1
#define SEM_PRECOND_JACOBI 2

typedef struct {
  int iters;       /* CG iterations (summed over inner solves for SEM_MIXED) */
  int outer_iters; /* refinement steps (SEM_MIXED), else 0 */
  double rel_res;  /* final ||r|| / ||b||: the true residual b - A x with the FP64 operator, except
                      when a SEM_FP64 solve stops on breakdown or maxit (then its CG recurrence
                      residual); SEM_MIXED always reports its last true residual */
  double ms;       /* device time of the solve (CUDA events on the internal stream) */
  int status;      /* sem_status of the solve */
} sem_solve_result;

/* Solve A x = b, A = mask QQ^T A_L, with Jacobi PCG (Sec. 2).  b_dev: FP64
 * right-hand side (continuous, zero on Dirichlet nodes, e.g. from sem_rhs).
 * x_dev: FP64, in: initial guess (masked), out: solution.  Synchronous with
 * respect to `stream` (it waits for prior work on it and returns when x is
 * written).  Returns the solve's status (also in result->status). */
sem_status sem_pcg_solve(const sem_mesh* mesh, const double* b_dev, double* x_dev,
                         const sem_solve_opts* opts, sem_solve_result* result, void* stream);

/* The same solve from host buffers: copies b in and x out inside the call
 * (end-to-end use by callers whose data lives in host memory). */
sem_status sem_pcg_solve_host(const sem_mesh* mesh, const double* b_host, double* x_host,
                              const sem_solve_opts* opts, sem_solve_result* result, void* stream);

/* Many solves of one odd polynomial order N at once (the serving form of the
 * hot path): ragged meshes, each with its own b_dev[k] / x_dev[k] (as for
 * sem_pcg_solve) and opts[k] (prec must be SEM_MIXED with refine = 0).  Up to
 * 32 requests are active at a time; one CUDA graph per step advances every
 * active request by 8 CG iterations with batched kernels (a persistent
 * bulk-copy pipelined FP32 local operator over the concatenated element
 * tiles, per-request alpha, batched QQ^T and update); requests beyond 32
 * join as others finish.  Each request's arithmetic depends only on its own
 * data, so its result equals that of a batch of one.  Synchronous.  A mesh
 * may appear several times (several right-hand sides on one mesh, e.g. the
 * three velocity components of a Helmholtz step); each repeat gets its own
 * work vectors (~80 B per local point), which the mesh keeps for its later
 * batches and frees with sem_mesh_destroy.  The engine of an order (its
 * buffers and captured graph) is kept for later calls of the same order.
 * Returns SEM_OK, or the first request's failing status (results[k].status
 * has each).  A failure of the batch itself (SEM_ERR_CUDA, SEM_ERR_OOM, or
 * SEM_ERR_DEVICE_TIMEOUT when it does not finish within 2^20 steps) is
 * returned at once, and the requests it had not finished get no result. */
sem_status sem_pcg_solve_batch(const sem_mesh* const* meshes, const double* const* b_dev, double* const* x_dev,
                               const sem_solve_opts* opts, sem_solve_result* results, int count, void* stream);

/* ---- solve without device allocation -------------------------------------- */

/* Largest mesh (local points) sem_pcg_solve_noalloc accepts. */
#define SEM_NOALLOC_MAX_POINTS (1 << 18)

/* The FP64 solve of sem_pcg_solve (opts->prec must be SEM_FP64) for callers
 * that cannot allocate device memory: code whose device memory is owned by a
 * fixed pool or another allocator, and real-time loops that cannot afford
 * cudaMalloc's latency or its implicit synchronisation.  The paper has no
 * counterpart; this is an interface convenience of this library.
 *
 * Its scratch (work vectors, reduction partials, the CG state; ~10.5 MB) is
 * one file-scope device array of fixed size, present on every device that
 * loads the library until the process exits; the call itself allocates
 * nothing.  The caller passes b_dev (input) and x_dev (initial guess in,
 * solution out) as for sem_pcg_solve.  Meshes with more than
 * SEM_NOALLOC_MAX_POINTS local points are rejected with SEM_ERR_INVALID.
 * b_dev and x_dev must be 16-byte aligned (SEM_ERR_INVALID otherwise).
 * Every call shares the one array and overwrites it, so calls whose work
 * overlaps on the GPU (different streams or threads) race and must not be
 * issued.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Same solve rule as sem_pcg_solve with SEM_FP64: CG on the tuned operator,
 * then the true residual ||b - A x|| / ||b|| with the native FP64 operator,
 * and restarts from x (at most 3, within maxit) while it misses opts->tol;
 * result->rel_res is that true residual and result->outer_iters the number
 * of restarts.  Runs on `stream` (on the mesh's device, which it makes
 * current) and returns when x is written; result->ms is 0. */
sem_status sem_pcg_solve_noalloc(const sem_mesh* mesh, const double* b_dev, double* x_dev,
                                 const sem_solve_opts* opts, sem_solve_result* result, void* stream);

/* ---- projection onto previous solutions --------------------------------- */
/* Sec. 2 (the velocity and pressure solves) accelerates successive solves
 * with one operator by projecting each new solution onto the space spanned by
 * earlier ones (the paper cites Fischer 1998 for it).  A space holds an
 * A-orthonormal basis x_1..x_l of earlier solutions (global inner product,
 * x_i^T A x_j = delta_ij) and A x_i, in library-owned device memory; a solve
 * starts CG from xbar = sum_i (x_i^T b) x_i, the best approximation to
 * A^{-1} b from the space in the A-norm, then A-orthogonalises the increment
 * x - xbar against the basis (two Gram-Schmidt passes), A-normalises it and
 * appends it; a full basis restarts from the newest solution alone. */
typedef struct sem_proj sem_proj;

/* Projection space for the operator (h1, h2) of one mesh: max_vectors in
 * 1..SEM_PROJ_MAX_VECTORS; allocates 2 * max_vectors + 3 local vectors of
 * doubles on the mesh's device.  The mesh must outlive the space.  Errors:
 * SEM_ERR_INVALID (null mesh/out, bad count, h1/h2 as in sem_pcg_solve),
 * SEM_ERR_OOM. */
#define SEM_PROJ_MAX_VECTORS 16
sem_status sem_proj_create(const sem_mesh* mesh, int max_vectors, double h1, double h2, sem_proj** out);
sem_status sem_proj_destroy(sem_proj* proj);

/* Solves A x = b as sem_pcg_solve does (same b/x layout, opts and result;
 * opts->h1, h2 must equal the space's, else SEM_ERR_INVALID), except that x_dev
 * is output only: the initial guess is the projection of b onto the space.
 * After a converged solve the new direction joins the space; after a failed
 * one the space is unchanged.  result->iters counts the CG iterations after
 * the projection; result->ms covers projection, solve and update.  Not thread
 * safe for one space; spaces of different meshes are independent. */
sem_status sem_proj_solve(sem_proj* proj, const double* b_dev, double* x_dev, const sem_solve_opts* opts,
                          sem_solve_result* result, void* stream);

/* Number of basis vectors held (0..max_vectors). */
sem_status sem_proj_size(const sem_proj* proj, int* nvec);

/* Empties the space (after the operator or the mesh changed). */
sem_status sem_proj_reset(sem_proj* proj);

/* ---- staggered P_N - P_{N-2} pressure space ------------------------------ */

/* Sec. 2 discretises velocity with Lagrange interpolants of order N on the
 * GLL points and pressure with interpolants of order N - 2 on the
 * Gauss-Legendre (GL) points, and solves the consistent Poisson equation for
 * the pressure update (Sec. 2, Eq. 5).  With m = N - 1 GL points per
 * direction, a pressure field is element-local (discontinuous): [E][m^3]
 * doubles, i fastest, n_pressure = E m^3 values.  A velocity is three local
 * vectors, component-major: [3][n_local] doubles (component a of local point
 * l at a * n_local + l).
 *
 * Definitions (the paper does not write them out; textbook staggered SEM):
 * at every GL point q of an element, J = dx/dr of the isoparametric map
 * evaluated there, rho_q = rho_i rho_j rho_k (GL weights) and
 *   F[b][a](q) = rho_q adj(J)_{ba} = rho_q det(J) (dr_b/dx_a);
 * the weak divergence  (D u)_q = sum_{a,b} F[b][a](q) (d u_a / d r_b)(q)
 * (the GL quadrature of the divergence against the GL Lagrange basis), the
 * weak gradient D^T (its transpose), and
 *   E p = sum_a D_a M^{-1} D_a^T p,   M^{-1} v = mask QQ^T(v) / QQ^T(B),
 * the inverse of the assembled GLL mass on the velocity nodes that are not
 * Dirichlet.  E is symmetric positive semi-definite; with Dirichlet velocity
 * on the whole boundary of an affine mesh (N >= 3) the constants span its
 * null space.
 *
 * All calls: FP64, asynchronous on `stream`, except that the first pressure
 * call on a mesh builds its GL-point data (9 m^3 doubles per element) on
 * `stream` and synchronises `stream` (so it must not be made while `stream`
 * is being captured).  Errors: SEM_ERR_INVALID (null argument, N < 2,
 * overlapping buffers), SEM_ERR_OOM, SEM_ERR_BAD_MESH (det J <= 0 at a GL
 * point), SEM_ERR_CUDA. */

/* Host only (no device use): the 1D data of the pressure space for order N
 * (2..11), m = N - 1: GL nodes zeta [m] (roots of P_m, ascending) and weights
 * rho [m]; Ig [m][n] = l_l(zeta_i) and DIg [m][n] = l_l'(zeta_i) for the GLL
 * Lagrange basis l_l of order N (n = N + 1).  Any output may be NULL. */
sem_status sem_pressure_basis(int N, double* zeta_host, double* rho_host, double* Ig_host, double* DIg_host);

/* Number of pressure values of the mesh: E (N-1)^3. */
sem_status sem_pressure_info(const sem_mesh* mesh, int64_t* n_pressure);

/* Copy of the GL-point factors F [E][9][m^3] (entry 3 b + a is F[b][a]). */
sem_status sem_pressure_factors(const sem_mesh* mesh, double* F_dev, void* stream);

/* u_a = (D_a^T p) element by element: p [E][m^3] -> u [3][n_local]; no
 * assembly, no mask.  p and u must not overlap. */
sem_status sem_pressure_grad(const sem_mesh* mesh, const double* p_dev, double* u_dev, void* stream);

/* q = sum_a D_a u_a element by element: u [3][n_local] -> q [E][m^3]. u and
 * q must not overlap. */
sem_status sem_pressure_div(const sem_mesh* mesh, const double* u_dev, double* q_dev, void* stream);

/* q = E p (Sec. 2, Eq. 5).  work_dev: caller-owned scratch of 3 n_local
 * doubles (the three velocity components), overwritten; it must not overlap
 * p or q.  q may equal p (p is read in full before q is written). */
sem_status sem_pressure_apply(const sem_mesh* mesh, const double* p_dev, double* q_dev, double* work_dev,
                              void* stream);

/* q = E p in FP32 (the factors, basis matrices and fields rounded from FP64,
 * the inverse assembled mass applied as its FP32 reciprocal): p, q [E][m^3]
 * floats, work_dev 3 n_local floats of caller-owned scratch; p, q, work
 * distinct.  The first call on a mesh builds the FP32 copies (synchronising
 * the stream). */
sem_status sem_pressure_apply_f32(const sem_mesh* mesh, const float* p_dev, float* q_dev, float* work_dev,
                                  void* stream);

/* Pressure solve for Sec. 2, Eq. 5: E p = g on the mean-free pressure space.
 * The constants are E's null space when the velocity is Dirichlet on the
 * whole boundary (exactly on affine meshes; on curved elements GL quadrature
 * leaves them a near-null mode), so the pressure is fixed up to a constant.
 * Solved: Pm E Pm p = Pm g with Pm = I - 1 1^T / n_pressure, by CG from
 * p = 0 in the Euclidean inner product over the pressure values, Jacobi
 * preconditioned (opts->precond SEM_PRECOND_DEFAULT or SEM_PRECOND_JACOBI:
 * z = Pm (r / diag(E)), the scaled residual projected back to the mean-free
 * space, so that the preconditioner is symmetric positive definite there;
 * diag(E) is built once per mesh, see sem_pressure_diag) or plain
 * (SEM_PRECOND_NONE: z = r), stopped when ||r|| <= opts->tol ||Pm g|| for the recurrence
 * residual and then for the true residual Pm (g - E p) (CG restarts from p,
 * at most 5 times, when the recurrence drifted); tol <= 0 means 1e-10,
 * maxit <= 0 means 20000.  opts->prec: SEM_FP64 (as above) or SEM_MIXED:
 * the same CG with E applied in FP32 (sem_pressure_apply_f32) and reliable
 * updates -- when the recurrence residual has dropped by opts->delta (<= 0
 * means 0.1) since the last replacement, at least 8 iterations later, or
 * below 0.2 tol, the true residual is formed with the FP64 E and replaces it
 * (result->outer_iters counts them); the solve stops when the true residual
 * meets tol.  The other fields of opts are ignored.
 * result->rel_res is the true residual once converged.
 * g_dev, p_dev: [E][m^3] FP64; p_dev is output only (mean zero).  Every
 * reduction is deterministic.  The iteration runs on the device: its scalars
 * stay in device memory and 8 iterations are one CUDA graph, launched on a
 * stream of the call's own (ordered after `stream`); the host reads the
 * state once per graph and synchronises before returning.  Allocates
 * 4 n_pressure + 3 n_local doubles of scratch for the call.  Returns the solve's status (also in result->status): SEM_OK,
 * SEM_ERR_NOT_CONVERGED or SEM_ERR_BREAKDOWN (<p, E p> <= 0), with result
 * filled in; result->outer_iters is 0 (SEM_FP64) and result->ms the device
 * time.  SEM_MIXED allocates a further 2 n_pressure + 3 n_local floats, and
 * keeps FP32 copies of the GL-point data on the mesh (36 B per pressure
 * value). */
sem_status sem_pressure_solve(const sem_mesh* mesh, const double* g_dev, double* p_dev, const sem_solve_opts* opts,
                              sem_solve_result* result, void* stream);

/* diag(E) of the pressure operator (the Jacobi preconditioner of
 * sem_pressure_solve): E_qq = sum_a sum_l D_a[q, l]^2 mask_l / (QQ^T B)_l over
 * the GLL points l of q's element (unit pressure q reaches only its own
 * element's velocity copies; no element holds two copies of one node), with
 * the rows D_a[q, l] = sum_b F[b][a](q) C_b[q, l] of the weak divergence,
 * summed by factorisation in FP64.  d_dev [E][m^3] FP64, device.  Ordered on
 * stream. */
sem_status sem_pressure_diag(const sem_mesh* mesh, double* d_dev, void* stream);

/* ---- overlapping Schwarz preconditioner: host set-up ---------------------- */

/* Sec. 2, Eq. 6 preconditions with local solves on overlapping subdomains.
 * Here a subdomain is one element with all its GLL nodes (the overlap is the
 * nodes shared with neighbours), and its local problem is replaced by the
 * separable fast-diagonalisation form built from 1D operators per reference
 * direction: with the element's mean length l along it, K = (2/l) D^T W D and
 * B = (l/2) W on the n GLL points; at an end shared with a neighbour of mean
 * length l' normal to the shared face, K[end][end] += (2/l') (D^T W D)[N][N]
 * and B[end][end] += (l'/2) w_N; an end on a Dirichlet face is decoupled (its
 * off-diagonal entries of K removed).  These calls solve K S = B S diag(lam)
 * with S^T B S = I (lam ascending); the local inverse is then
 * (S_t (x) S_s (x) S_r) (h1 (lam_t + lam_s + lam_r) + h2)^{-1} (S_t (x) S_s (x) S_r)^T.
 * Host only: no device use.  The device apply of this preconditioner is not
 * part of the library. */

/* One 1D problem.  l_lo, l_hi <= 0: no neighbour at that end; dir_lo, dir_hi:
 * that end is on a Dirichlet face.  S_host [n][n] row-major (column c is the
 * c-th eigenvector), lam_host [n].  SEM_ERR_INVALID for N outside [1, 11] or
 * l <= 0. */
sem_status sem_schwarz_fdm_1d(int N, double l, double l_lo, double l_hi, int dir_lo, int dir_hi, double* S_host,
                              double* lam_host);

/* Every element of a mesh given on the host: glo [E][n^3] global ids (as
 * sem_mesh_global_ids), xyz [E][3][n^3] GLL coordinates, dirichlet_face [E][6]
 * (faces 0: i = 0, 1: i = N, 2: j = 0, 3: j = N, 4: k = 0, 5: k = N).  Mean
 * lengths are the mean over the n^2 GLL lines of the distance between their
 * ends; two element faces are neighbours when their four corner nodes have
 * the same global ids (in any orientation).  Outputs S_host [E][3][n][n] and lam_host [E][3][n]
 * (direction r, s, t); each distinct 1D problem is solved once, and
 * *n_distinct (nullable) receives their number. */
sem_status sem_schwarz_setup_host(int64_t E, int N, const int64_t* glo, const double* xyz,
                                  const uint8_t* dirichlet_face, double* S_host, double* lam_host,
                                  int64_t* n_distinct);

/* ---- overlapping Schwarz preconditioner on the device (Sec. 2, Eq. 6) ------
 * Eq. 6 preconditions the solve with local solves on overlapping subdomains
 * plus a coarse-grid solve.  Here (the paper leaves the pieces undefined):
 *   M^{-1} r = mask QQ^T (W A~_e^{-1} (W r_e) for every element e) + R_0^T A_0^{-1} R_0 r
 * - subdomain e: the element with all its GLL nodes (overlap = shared nodes);
 *   A~_e: the separable fast-diagonalisation form of its local problem, 1D
 *   operators from the element's mean lengths and its face neighbours' (see
 *   sem_schwarz_setup_host), A~_e^{-1} = (S_t(x)S_s(x)S_r)(h1 (lam_r + lam_s +
 *   lam_t) + h2)^{-1}(S_t(x)S_s(x)S_r)^T;
 * - W = mult^{-1/2} at every local point (symmetric weighting);
 * - coarse space: the trilinear functions of the element vertices that are
 *   not Dirichlet; R_0 r = sum over global nodes of phi r, A_0 = R_0 A R_0^T
 *   (Galerkin), solved through its inverse, formed once on the device
 *   (Gauss-Jordan, SPD), when A_0 has at most SEM_SCHWARZ_DENSE_COARSE_MAX
 *   unknowns; larger A_0 are solved approximately by a fixed symmetric
 *   two-level cycle (Chebyshev smoothing in diag(A_0)^-1 A_0, and the exact
 *   correction on aggregates of about 64 vertices grouped by coordinate
 *   bisection), so M stays a fixed SPD operator. */
typedef struct sem_schwarz sem_schwarz;
#define SEM_SCHWARZ_COARSE 1             /* flags: include the coarse-grid term */
#define SEM_SCHWARZ_FP32_PRECOND 2       /* flags: SEM_FP64 solves apply the FP32 preconditioner
                                            (z = M32 float(r), back to FP64): FP64 CG at the cost of
                                            the FP32 application; M is then not exactly linear, which
                                            CG tolerates at the 1e-7 level of FP32 rounding */
#define SEM_SCHWARZ_DENSE_COARSE_MAX 8192

typedef struct {
  int64_t n_distinct; /* distinct 1D eigenproblems solved on the host */
  int64_t n_coarse;   /* coarse unknowns (free element vertices) */
  int coarse;         /* coarse term: 0 none, 1 dense inverse of A_0, 2 two-level cycle */
  size_t dev_bytes;   /* device memory held by the preconditioner (solver workspace excluded) */
  double setup_ms;    /* wall time of sem_schwarz_create */
} sem_schwarz_info_t;

/* Build the preconditioner of a mesh for the operator (h1, h2), scalars
 * (meshes with per-point coefficients: SEM_ERR_INVALID).  Synchronous; holds
 * library-owned device memory until sem_schwarz_destroy.  The mesh must
 * outlive it, and a later sem_mesh_set_coefficients makes it unusable
 * (SEM_ERR_INVALID from apply/solve).  Errors: SEM_ERR_INVALID,
 * SEM_ERR_BREAKDOWN (coarse matrix not positive definite), SEM_ERR_CUDA. */
sem_status sem_schwarz_create(const sem_mesh* mesh, double h1, double h2, int flags, sem_schwarz** out);
sem_status sem_schwarz_destroy(sem_schwarz* sw);
sem_status sem_schwarz_info(const sem_schwarz* sw, sem_schwarz_info_t* info);

/* z = M^{-1} r for a continuous, masked local vector r (as the CG residual):
 * r_dev, z_dev [E][n^3] device arrays of doubles (SEM_FP64) or floats
 * (SEM_FP32, the FP32 tables and fields), distinct; asynchronous on stream.
 * The coarse term works in scratch arrays of the preconditioner, so the
 * applies of one preconditioner must not overlap on the device: issue them
 * on one stream (or order their streams), and not while a sem_schwarz_solve
 * with it runs.  Errors: SEM_ERR_INVALID (null or equal arrays, another
 * prec, coefficients changed since create), SEM_ERR_CUDA. */
sem_status sem_schwarz_apply(const sem_schwarz* sw, const void* r_dev, void* z_dev, sem_prec prec, void* stream);

/* PCG for A x = b with z = M^{-1} r in place of Jacobi; b_dev, x_dev, opts and
 * result as sem_pcg_solve (opts->h1, h2 must be the preconditioner's).
 * SEM_FP64: FP64 CG and FP64 preconditioner, the final true residual checked
 * with the native FP64 operator (restarts as sem_pcg_solve).  SEM_MIXED: FP32
 * CG with the FP32 operator and preconditioner on the system scaled by
 * 1/||b||, FP64 reliable updates (opts->delta; <= 0 means 0.3) with the
 * native FP64 residual.  Synchronous; one solve at a time per preconditioner. */
sem_status sem_schwarz_solve(sem_schwarz* sw, const double* b_dev, double* x_dev, const sem_solve_opts* opts,
                             sem_solve_result* result, void* stream);

/* ---- serving ------------------------------------------------------------ */

typedef struct {
  size_t hbm_budget_bytes; /* device bytes the server may hold for requests; 0 = 80% of free memory */
  int max_slots;           /* requests solved concurrently (each on its own stream); <= 0 means 8 */
  int max_queue;           /* admitted-but-waiting requests; <= 0 means 4096 */
  int device;              /* CUDA device ordinal */
  int batch;               /* 0 (default): mixed-precision requests of odd order N run in per-order
                              batches (one CUDA graph of batched kernels advances them together;
                              requests join and leave between graph launches); 1: every request
                              is solved alone on its slot's stream */
} sem_server_opts;

typedef struct sem_server sem_server;

/* Start a server: worker threads take queued requests as slots and HBM
 * budget free up; each builds the request's mesh, forms b = mask QQ^T (B f)
 * and runs sem_pcg_solve on its own stream, so requests overlap on the GPU. */
sem_status sem_server_create(const sem_server_opts* opts, sem_server** out);

/* Queue a solve.  desc: as for sem_mesh_create (explicit arrays are copied
 * before return); f_host: nodal forcing [E (N+1)^3] (copied before return);
 * opts: solve options.  SEM_ERR_OOM if the request alone exceeds the HBM
 * budget, SEM_ERR_BUSY if the queue is full.  *req_id receives the id. */
sem_status sem_server_submit(sem_server* srv, const sem_mesh_desc* desc, const double* f_host,
                             const sem_solve_opts* opts, uint64_t* req_id);

/* Wait up to timeout_ms (< 0: forever) for a request.  On completion copies
 * the solution into x_host (nullable, [n_local] FP64) and the record into
 * result (nullable), forgets the request and returns its solve status;
 * SEM_ERR_TIMEOUT if not done yet (the request stays known). */
sem_status sem_server_poll(sem_server* srv, uint64_t req_id, int timeout_ms, double* x_host,
                           sem_solve_result* result);

/* Where a request's latency went, in milliseconds of host wall time:
 * queue_ms: submit until a slot takes it (slots and HBM budget); setup_ms:
 * building its mesh and b = mask QQ^T (B f); wait_ms: until its engine admits
 * it into the running batch (0 when solved alone); solve_ms: until its result
 * is copied out; total_ms: submit until the result is visible to poll
 * (completion), whenever the caller polls. */
typedef struct {
  double queue_ms, setup_ms, wait_ms, solve_ms, total_ms;
} sem_request_timing;

/* sem_server_poll that also fills timing (nullable) for the completed request. */
sem_status sem_server_poll_timed(sem_server* srv, uint64_t req_id, int timeout_ms, double* x_host,
                                 sem_solve_result* result, sem_request_timing* timing);

/* Cancel a queued request (one already running finishes). */
sem_status sem_server_cancel(sem_server* srv, uint64_t req_id);

typedef struct {
  uint64_t submitted, completed, rejected, cancelled;
  int queued, running;
  size_t hbm_in_use, hbm_budget;
} sem_server_stats;

sem_status sem_server_stats_get(sem_server* srv, sem_server_stats* out);

/* Stop accepting work, finish running requests, drop queued ones, free all. */
sem_status sem_server_destroy(sem_server* srv);

/* ---- host-only helpers (no GPU needed) ----------------------------------- */

/* First-touch global numbering from element corner vertex ids alone (the
 * topological construction sem_mesh_create uses): vert [E][8] as in
 * sem_mesh_desc; out glo [E (N+1)^3].  *n_global receives the node count. */
sem_status sem_topology_numbering(int64_t E, int N, const int64_t* vert, int64_t* glo_host,
                                  int64_t* n_global);

/* One rank's gather-scatter halo under an element partition (Sec. 3.1
 * partitions elements across ranks, one per GPU; Sec. 2 sums shared face
 * values across them).  This library runs one GPU per process, so it uses no
 * halo itself; the split is defined here for a multi-rank QQ^T.  elem_rank
 * [E] gives each element's rank (>= 0); a rank's local vector holds its
 * elements in ascending element order, (N+1)^3 points each.  For every global
 * node with copies on `rank` and on another rank, in ascending global id:
 * node_gid[k], and its copies node_ptr[k] .. node_ptr[k+1]-1 as (copy_rank,
 * copy_local = index in that rank's local vector) in ascending global local
 * index.  Summing each node's copies in that order gives QQ^T bit for bit as
 * on one rank; nodes with all copies on `rank` need no exchange.  Call with
 * node_gid = NULL for *n_nodes and *n_copies, then with arrays of those
 * sizes (node_ptr: n_nodes + 1).  Host memory only; no GPU needed. */
sem_status sem_gs_halo(int64_t E, int N, const int64_t* vert, const int32_t* elem_rank, int rank,
                       int64_t* n_nodes, int64_t* n_copies, int64_t* node_gid, int64_t* node_ptr,
                       int32_t* copy_rank, int64_t* copy_local);

/* Corner vertex ids [E][8] of the built-in box / pipe generators. */
sem_status sem_mesh_vertices(const sem_mesh_desc* desc, int64_t* vert_host, int64_t* E_out);

/* Which kernel FP64 requests on this mesh use, as chosen by the autotuner at
 * creation: 1 = double-float (FP32-pair) arithmetic, 0 = native FP64. */
int sem_mesh_fp64_kernel(const sem_mesh* mesh);

/* Local-operator kernel variant the autotuner chose for `prec` (SEM_FP64
 * or SEM_FP32): 0 / 1 register kernels with ~256 / ~128 threads per CTA,
 * 2 / 3 (FP32) persistent kernels fed by bulk copies into a shared-memory
 * ring.  -1 for a bad argument. */
int sem_mesh_ax_variant(const sem_mesh* mesh, sem_prec prec);

/* Synchronise `stream` and report whether a local-operator kernel launched
 * on this mesh gave up a bounded device-side wait (the bulk-copy pipelined
 * kernels wait on shared-memory barriers with an iteration limit):
 * SEM_ERR_DEVICE_TIMEOUT if so (the affected output is invalid; the flag is
 * cleared), else SEM_OK.  Solves report such a timeout in their status. */
sem_status sem_mesh_check(const sem_mesh* mesh, void* stream);

/* Number of CUDA kernels the library has launched in this process (a graph
 * replay counts each of its kernel nodes).  Monotone; thread-safe. */
uint64_t sem_kernel_launches(void);

const char* sem_status_str(sem_status s);
const char* sem_last_error(void);
int sem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
