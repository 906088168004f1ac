/*
 * dg.h -- C ABI of libdg, a GB300 (sm_103a) interior-penalty discontinuous
 * Galerkin solver for the steady diffusion-convection-reaction problem
 *
 *     alpha u - eps Lap u + b . grad u = f   in Omega (a polygon in R^2),
 *     u = gD on Gamma_D,   eps grad u . n = gN on Gamma_N            (Eq. (1))
 *
 * following Uzunca & Karasozen, "A Matlab Tutorial for Diffusion-Convection-
 * Reaction Equations using DGFEM" (arXiv:1502.02941): SIPG / NIPG / IIPG for
 * diffusion (Sec. 1, Eq. (ds)), upwinding for convection, discontinuous P_k
 * elements on triangles, weakly imposed boundary data.
 *
 * Conventions for every call:
 *   - Every call returns a dg_status; DG_OK (0) on success.  Arguments are
 *     checked before anything is launched; dg_status_string() names a code and
 *     dg_last_error() gives the message of the handle's last failure.
 *   - Pointers are marked "host" or "device".  Device pointers are plain CUDA
 *     global-memory addresses on the handle's device (e.g. a torch tensor's
 *     data_ptr()).  The caller owns every buffer it passes; the handle owns the
 *     mesh, the assembled blocks and its solver workspace.
 *   - Work is issued on the handle's stream.  Calls return without waiting for
 *     the GPU, except those that return values to host memory (dg_mesh_upload,
 *     dg_gmres_solve, dg_dense_solve, dg_mixed_solve, dg_l2_error,
 *     dg_precond_setup), which synchronise the stream.
 *   - Indices are 0-based (the paper's MATLAB arrays are 1-based).
 *   - Unknowns are element-major: x[K*nb + i] is the coefficient of the i-th
 *     orthonormal Dubiner basis function of element K, nb = (k+1)(k+2)/2
 *     (the DoF formula of the Sec. 4 listing).
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status codes                                                              */
/* ------------------------------------------------------------------------ */
typedef int dg_status;
#define DG_OK                  0
#define DG_ERR_INVALID_ARG     1  /* a pointer, size or enum is out of range */
#define DG_ERR_CUDA            2  /* a CUDA runtime call failed */
#define DG_NOT_CONVERGED       3  /* solver hit its iteration cap; info still filled */
#define DG_ERR_TIMEOUT         4  /* a bounded device-side wait expired (reserved: no kernel of this library spins on a flag) */
#define DG_ERR_NONFINITE       5  /* NaN/Inf met in data or in a residual */
#define DG_ERR_SINGULAR_BLOCK  6  /* a diagonal block could not be inverted */
#define DG_ERR_MESH            7  /* invalid mesh: clockwise element, edge shared by
                                     more than two elements, boundary edge without
                                     a condition, or a condition on a non-boundary edge */
#define DG_ERR_STATE           8  /* call order violated (e.g. apply before assemble) */
#define DG_ERR_NOMEM           9  /* device allocation failed */

/* ------------------------------------------------------------------------ */
/* enumerations                                                              */
/* ------------------------------------------------------------------------ */
/* DG variant, the paper's `method` numbering (Sec. 2.2, set_parameter). */
#define DG_NIPG 1   /* kappa = +1 */
#define DG_SIPG 2   /* kappa = -1 */
#define DG_IIPG 3   /* kappa =  0 */

/* Arithmetic / storage types of an operator apply. */
#define DG_F64  0   /* f64 blocks, f64 vectors, f64 accumulation */
#define DG_F32  1   /* f32 blocks, f32 vectors, f32 accumulation */
#define DG_BF16 2   /* bf16 blocks, f32 vectors, f32 accumulation */

/* Which block copies dg_assemble stores (bit mask). */
#define DG_STORE_F64  1
#define DG_STORE_F32  2
#define DG_STORE_BF16 4

/* Preconditioners. */
#define DG_PRECOND_NONE          0
#define DG_PRECOND_BLOCK_JACOBI  1
#define DG_PRECOND_MLP           2   /* block Jacobi + learned element-local correction (flexible GMRES) */
#define DG_PRECOND_SCHWARZ       3   /* one-layer-overlap restricted additive Schwarz (exact patch solves) */

/* Point sets of dg_quad_points / dg_eval. */
#define DG_POINTS_VOLUME   0  /* [ne][(k+2)^2]: Duffy-collapsed Gauss-Legendre */
#define DG_POINTS_BOUNDARY 1  /* [n_bedges][k+2]: Gauss-Legendre on boundary edges */
#define DG_POINTS_ERROR    2  /* [ne][(k+4)^2]: the L2-error rule */
#define DG_POINTS_FACE     3  /* [ne][3][k+2]: Gauss-Legendre on the three faces of every element */

/* ------------------------------------------------------------------------ */
/* parameters                                                                */
/* ------------------------------------------------------------------------ */
/*
 * Method parameters (Sec. 1 last paragraph; Sec. 4 set_parameter) and solver
 * settings.  Fill with dg_params_default() and override fields.
 */
typedef struct {
    int32_t method;            /* DG_NIPG / DG_SIPG / DG_IIPG */
    int32_t degree;            /* k, 1..3 */
    double  sigma_int;         /* interior-edge penalty sigma; <= 0 selects the
                                  paper's rule: 3k(k+1) for SIPG/IIPG, 1 for NIPG */
    double  sigma_bdry_factor; /* boundary-edge penalty = factor * sigma_int
                                  (paper: 2); <= 0 selects 2 */
    double  b0;                /* superpenalisation exponent (Sec. 4 set_parameter):
                                  the penalty terms carry sigma eps / |e|^b0;
                                  1 (the paper's default) .. 8 */
    int32_t store;             /* DG_STORE_* mask of block copies to keep */
    int32_t gmres_m;           /* GMRES restart length, 1..64 (default 50) */
    double  tol;               /* relative residual target ||F-Ax||/||F|| */
    int32_t max_it;            /* cap on Arnoldi steps (default 10000) */
    int32_t precond;           /* DG_PRECOND_* (default block Jacobi) */
} dg_params;

/*
 * Problem data (Eq. (1)).  alpha is a constant; the advection field is
 * affine, b(x,y) = (b[0] + b[1] x + b[2] y, b[3] + b[4] x + b[5] y).  The data
 * f, gD, gN are given at the library's quadrature points (dg_quad_points), the
 * way the paper's vectorised sub-functions fsource / DBCexact / NBCexact are
 * evaluated on arrays of points, or as constants when the pointer is NULL.
 *   f  : device [ne][(k+2)^2]     at DG_POINTS_VOLUME
 *   gD : device [n_bedges][k+2]   at DG_POINTS_BOUNDARY; read on Dirichlet edges
 *        and on the inflow part (b.n < 0) of EVERY boundary edge, Neumann ones
 *        included (the inflow term of Eq. (ds) runs over all of Gamma^-)
 *   gN : device [n_bedges][k+2]   at DG_POINTS_BOUNDARY; read on Neumann edges
 * The diffusion coefficient is the constant eps, or, when eps_q is given, the
 * paper's fdiff(x, y) (Sec. 2.2) evaluated at the points:
 *   eps_q : device [ne][(k+2)^2]  at DG_POINTS_VOLUME (the volume term)
 *   eps_f : device [ne][3][k+2]   at DG_POINTS_FACE (the face terms
 *           {eps grad u}, {eps grad v}, the penalty sigma eps / h_e and the
 *           Dirichlet RHS terms); on an interior edge the mean of the two
 *           elements' values at each point is used, which is eps(x) itself
 *           for a continuous eps
 * eps_q and eps_f are given together (DG_ERR_INVALID_ARG otherwise), need the
 * f64 block copy in params.store, and are not read in batch mode
 * (DG_ERR_INVALID_ARG).  All terms of Eq. (ds) are linear in eps, so the
 * library assembles the eps = 0 operator and adds the pointwise-eps terms.
 */
typedef struct {
    double eps;
    double alpha;
    double b[6];
    const double* f;   double f_const;
    const double* gD;  double gD_const;
    const double* gN;  double gN_const;
    const double* eps_q;   /* NULL: constant eps */
    const double* eps_f;
} dg_coeffs;

/* Sizes of the uploaded mesh for the current degree. */
typedef struct {
    int32_t ne;          /* elements */
    int32_t nv;          /* nodes */
    int32_t n_bedges;    /* boundary edges (Dirichlet + Neumann) */
    int32_t n_interior;  /* interior edges */
    int32_t nb;          /* unknowns per element, (k+1)(k+2)/2 */
    int64_t dofs;        /* ne * nb */
    int32_t q_volume;    /* (k+2)^2 */
    int32_t q_edge;      /* k+2 */
    int32_t q_error;     /* (k+4)^2 */
    int64_t block_bytes[3]; /* bytes of the stored f64 / f32 / bf16 block copies (0 if absent) */
} dg_info;

/* Result of an iterative solve. */
typedef struct {
    int32_t iterations;  /* inner Arnoldi steps (all cycles) */
    int32_t restarts;    /* completed restart cycles */
    int32_t outer;       /* refinement steps (dg_mixed_solve), else 0 */
    int32_t status;      /* DG_OK or DG_NOT_CONVERGED */
    double  relres;      /* final true relative residual ||F - A x|| / ||F|| in f64 */
} dg_solve_info;

/* ------------------------------------------------------------------------ */
/* handle                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct dg_handle dg_handle;

/* Create a handle on CUDA device `device`, issuing work on `stream`
   (a cudaStream_t; NULL = the legacy default stream).  *h receives the handle.
   The solvers launch the Arnoldi-step kernels of their f32 (inner) GMRES with
   programmatic dependent launch (each kernel may be scheduled while its
   predecessor finishes); the environment variable DG_PDL=0, read here, turns
   that off. */
dg_status dg_create(dg_handle** h, int device, void* stream);
/* (Test hook: with the environment variable DG_FAIL_CUDA_CALL=n set when the
   handle is created, the n-th CUDA runtime call the handle checks reports a
   failure after the real call has succeeded: the call in progress returns
   DG_ERR_CUDA with dg_last_error naming the injected failure, and later
   calls behave normally.  No GPU fault is involved.) */
/* Free the handle and all device memory it owns.  NULL is accepted. */
dg_status dg_destroy(dg_handle* h);
/* Create / destroy a CUDA stream that is ordered with the legacy default
   stream (created without cudaStreamNonBlocking), for callers whose own work
   runs on the legacy stream: unlike the legacy stream it can be captured into
   the solver's CUDA graphs. */
dg_status dg_stream_create(int device, void** stream);
dg_status dg_stream_destroy(void* stream);

/* ------------------------------------------------------------------------ */
/* device memory of a handle                                                 */
/* ------------------------------------------------------------------------ */
/*
 * (Runtime; the paper, a MATLAB code, has no counterpart.)
 * A handle keeps its mesh, assembled operator, preconditioner and solver
 * workspaces in device memory it allocates as the calls need it (arrays grow
 * when a larger mesh or degree needs more, and are kept for reuse).  By
 * default that memory comes from cudaMalloc.  A caller that owns the device's
 * memory (a framework's caching allocator, a pool sized at start-up) can
 * supply it instead, in one of two ways, right after dg_create and before any
 * other call that allocates:
 *   - dg_set_allocator: the handle calls alloc(ctx, bytes, device, stream)
 *     for every array and free(ctx, ptr, bytes, device, stream) when it
 *     releases one (stream = the handle's stream at that moment).  alloc must
 *     return memory on the handle's device, aligned to 256 bytes, or NULL
 *     (the call then fails with DG_ERR_NOMEM).
 *   - dg_set_arena: the handle carves every array out of the caller's device
 *     buffer [base, base + bytes) (base aligned to 256 bytes; first fit with
 *     256-byte granules); DG_ERR_NOMEM when the arena has no free range large
 *     enough.  The caller keeps the buffer alive until dg_destroy.
 * Either call moves the handle's 64-byte flag block to the new source and
 * fails with DG_ERR_STATE if the handle already holds any other device memory
 * (if the new source cannot give the flag block, the call returns
 * DG_ERR_NOMEM and the handle stays on cudaMalloc).
 * dg_destroy releases everything through the source in use.  Small pinned
 * HOST buffers for solver status words still come from cudaMallocHost, and
 * CUDA graph instantiation may allocate inside the driver.
 * Ownership: the handle owns the memory it obtained until it releases it.
 */
typedef void* (*dg_alloc_fn)(void* ctx, size_t bytes, int device, void* stream);
typedef void (*dg_free_fn)(void* ctx, void* ptr, size_t bytes, int device, void* stream);
dg_status dg_set_allocator(dg_handle* h, dg_alloc_fn alloc_fn, dg_free_fn free_fn, void* ctx);
dg_status dg_set_arena(dg_handle* h, void* base, size_t bytes);

/* Categories of the handle's device memory for dg_workspace_size. */
#define DG_WS_TOTAL     0  /* everything the handle holds now */
#define DG_WS_MESH      1  /* mesh arrays, geometry, adjacency, reference tables */
#define DG_WS_OPERATOR  2  /* assembled block copies (params.store) and F */
#define DG_WS_PRECOND   3  /* block-Jacobi inverses, A M^-1, Schwarz rows */
#define DG_WS_SOLVER    4  /* Krylov bases, solver states, refinement, batch and Newton buffers */
#define DG_WS_LEARNED   5  /* network weights, training rows and training workspace */
#define DG_WS_SCRATCH   6  /* shared scratch (assembly factors, reductions, dense LU) and flags */
#define DG_WS_PEAK      7  /* largest DG_WS_TOTAL since dg_create or the last dg_set_allocator / dg_set_arena */
/*
 * Bytes of device memory the handle holds in category `what` (DG_WS_*), as
 * requested from its memory source (an arena rounds each array up to 256
 * bytes on top of this).  DG_WS_PEAK sizes an arena for a later handle that
 * runs the same sequence of calls on the same sizes: with first fit,
 * arrays re-allocated as they grow can fragment the arena, so leave headroom
 * (a quarter more covers the library's own call sequences).  Returns 0 for a
 * NULL handle or an unknown category.  Host-side bookkeeping, no
 * synchronisation.
 */
size_t dg_workspace_size(const dg_handle* h, int what);

/* Change the stream later calls issue work on. */
dg_status dg_set_stream(dg_handle* h, void* stream);
/* Human-readable text of a status code (static storage). */
const char* dg_status_string(dg_status s);
/* Message of the last failed call on h (handle-owned storage). */
const char* dg_last_error(const dg_handle* h);

/* Fill p with defaults: SIPG, k = 1, paper's penalty rule, factor 2, b0 = 1,
   store f64, GMRES(50), tol 1e-10, max_it 10000, block Jacobi. */
dg_status dg_params_default(dg_params* p);

/* ------------------------------------------------------------------------ */
/* mesh and parameters  (the paper's getmesh and set_parameter)             */
/* ------------------------------------------------------------------------ */
/*
 * Upload a triangulation (Sec. 2.1 data structure; the paper's getmesh):
 *   nodes     host [nv][2]  f64 coordinates
 *   elems     host [ne][3]  i32 node ids, counter-clockwise, 0-based
 *   dirichlet host [nd][2]  i32 start/end node of each Dirichlet edge
 *   neumann   host [nn][2]  i32 start/end node of each Neumann edge
 * The arrays are copied; the element adjacency, face types, boundary-edge
 * numbering and per-element geometry are built on the device.  Every boundary
 * edge must carry exactly one condition.  Returns DG_ERR_MESH for an invalid
 * mesh.  Invalidates assembled data.  Synchronises.
 */
dg_status dg_mesh_upload(dg_handle* h, const double* nodes, int nv, const int* elems, int ne,
                         const int* dirichlet, int nd, const int* neumann, int nn);

/*
 * Uniform (red) refinement, the paper's uniformrefine (Sec. 2.1): every
 * triangle is cut into four by its edge midpoints and every boundary edge into
 * two.  Host arrays in (as dg_mesh_upload), caller-allocated host arrays out;
 * no GPU is used and no handle is needed.  With nodes_out == NULL only the
 * sizes are written: *nv_out = nv + (number of distinct edges), *ne_out = 4 ne,
 * *nd_out = 2 nd, *nn_out = 2 nn.  Otherwise nodes_out [*nv_out][2] keeps the
 * old nodes first and then the edge midpoints, numbered in the order their
 * edges are first met (elements in order, local edges (0,1), (1,2), (2,0));
 * element (a, b, c) with midpoints m_ab, m_bc, m_ca becomes (a, m_ab, m_ca),
 * (m_ab, b, m_bc), (m_ca, m_bc, c), (m_ab, m_bc, m_ca) in elems_out
 * [4 ne][3], counter-clockwise when the parent is; boundary edge (s, e)
 * becomes (s, m), (m, e).  DG_ERR_MESH for a node index out of range or a
 * boundary edge that is not an element edge.
 */
dg_status dg_mesh_refine(const double* nodes, int nv, const int* elems, int ne, const int* dirichlet, int nd,
                         const int* neumann, int nn, double* nodes_out, int* nv_out, int* elems_out, int* ne_out,
                         int* dirichlet_out, int* nd_out, int* neumann_out, int* nn_out);

/* Set method and solver parameters (the paper's set_parameter).  A change of
   degree invalidates assembled data. */
dg_status dg_set_params(dg_handle* h, const dg_params* p);

/* Sizes of the uploaded mesh under the current parameters. */
dg_status dg_get_info(dg_handle* h, dg_info* out);

/*
 * Physical coordinates of a point set (DG_POINTS_*), written to device
 * xy[...][2] in the layout given at the DG_POINTS_* constants.  Boundary edges
 * are numbered in (element, local face) order; each edge's points run
 * counter-clockwise around its element.
 */
dg_status dg_quad_points(dg_handle* h, int which, double* xy);

/* Outward unit normal (device [n_bedges][2]) and condition (device [n_bedges],
   1 Dirichlet, 2 Neumann; may be NULL) of every boundary edge. */
dg_status dg_boundary_info(dg_handle* h, double* normals, int* type);

/* ------------------------------------------------------------------------ */
/* assembly  (the paper's global_system, Sec. 2.3)                          */
/* ------------------------------------------------------------------------ */
/*
 * Assemble Stiff = D + C + R (Eq. (system)) and F_i = l_h(phi_i) of Eq. (ds)
 * on the device, element row by element row: per element K the diagonal block
 * A_KK (volume terms eps grad u.grad v + (b.grad u) v + alpha u v, and the
 * K-side parts of the face terms) and one block per neighbour L across face f,
 * A_KL (interior-penalty, symmetry/non-symmetry and upwind coupling).  Face
 * terms: -{eps grad u}.[v] + kappa {eps grad v}.[u] + (sigma eps/h_e)[u].[v]
 * on interior and Dirichlet edges (h_e = |e|, boundary sigma = factor*sigma),
 * upwind b.n(u_out - u_in) v on the inflow part of interior edges and
 * -b.n u_in v on the inflow part of every boundary edge.  RHS: f v, Dirichlet
 * terms gD (sigma eps/h_e v + kappa eps grad v.n), inflow -b.n gD v, Neumann
 * gN v.  Block copies are kept in the precisions of params.store.
 */
dg_status dg_assemble(dg_handle* h, const dg_coeffs* c);

/* Copy the assembled F (device [dofs] f64). */
dg_status dg_get_rhs(dg_handle* h, double* F);

/*
 * Copy the assembled blocks of one stored precision into device out
 * [ne][4][nb][nb] (type per dtype: f64 / f32 / bf16 as uint16), row-major:
 * slot 0 = A_KK, slot 1+f = A_{K,L(f)} for the neighbour across local face f
 * (face f joins local vertices f and f+1 mod 3); absent neighbours give zero
 * blocks.  nbr (device [ne][3], may be NULL) receives L(f), -1 on the boundary.
 */
dg_status dg_get_blocks(dg_handle* h, int dtype, void* out, int* nbr);

/* ------------------------------------------------------------------------ */
/* operator apply and preconditioner                                         */
/* ------------------------------------------------------------------------ */
/*
 * y = Stiff x (Eq. (system): D u + C u + R u) for device vectors of `dofs`
 * entries: f64 for DG_F64, f32 for DG_F32 and DG_BF16.  Requires the matching
 * block copy in params.store.  x and y must not overlap.
 */
dg_status dg_apply(dg_handle* h, int dtype, const void* x, void* y);

/* Build the preconditioner (DG_PRECOND_BLOCK_JACOBI: f64 Gauss-Jordan inverse
   with partial pivoting of every diagonal block A_KK, plus an f32 copy, and the
   right-preconditioned operator A M^-1 (blocks A_KL A_LL^-1 formed in f64,
   stored for each of the f64 / f32 block copies) that the solvers apply in one
   pass per Arnoldi step).  DG_PRECOND_SCHWARZ additionally forms, for every
   element K, the rows of K in the inverse of its patch matrix A_P (K and its
   face neighbours, f64 Gaussian elimination with partial pivoting): the
   preconditioner z_K = (A_P^-1 r_P)_K is then one block-sparse apply with the
   sparsity of A (f64 and f32 copies).  DG_ERR_SINGULAR_BLOCK if a diagonal
   block or a patch matrix is singular.  Synchronises. */
dg_status dg_precond_setup(dg_handle* h, int kind);

/* z = M^-1 r for device vectors (f64 for DG_F64, f32 otherwise). */
dg_status dg_precond_apply(dg_handle* h, int dtype, const void* r, void* z);

/* ------------------------------------------------------------------------ */
/* solvers  (replacing the paper's Stiff\F, Sec. 2.3)                       */
/* ------------------------------------------------------------------------ */
/*
 * Restarted GMRES(m) in f64 with right preconditioning (params.precond),
 * x0 = 0, classical Gram-Schmidt with the norm taken as ||w||^2 - sum h_d^2 in
 * the same reduction and one conditional re-orthogonalisation pass (when less
 * than 0.49 ||w||^2 remains), Givens rotations on the device; one CUDA graph
 * per restart cycle on a non-default stream.  Stops when the true residual
 * ||F - A x||/||F|| <= params.tol (checked at every restart) or after
 * params.max_it Arnoldi steps (DG_NOT_CONVERGED, info still filled).
 *   F    device [dofs] f64 right-hand side, or NULL for the assembled F
 *   x    device [dofs] f64 solution (output)
 *   info host, may be NULL
 * Synchronises.
 */
dg_status dg_gmres_solve(dg_handle* h, const double* F, double* x, dg_solve_info* info);

/*
 * Mixed-precision solve by iterative refinement.  The outer loop computes the
 * true residual r = F - A x with the f64 blocks (f64 arithmetic) and stops when
 * ||r||/||F|| <= params.tol.  Each correction solves A_lo d = r/||r||
 * approximately with restarted GMRES(inner_m) on f32 vectors, using the f32
 * (inner_dtype DG_F32) or bf16 (DG_BF16) block copy with f32 accumulation and
 * the params.precond preconditioner (block Jacobi: the f64 inverses applied in
 * f32; Schwarz: the f32 copy of the patch-inverse rows), to relative
 * residual inner_tol or for at most 8 restart cycles (8 inner_m steps: past
 * that the f32 iteration sits at its accuracy floor and a fresh f64 residual
 * serves better); dot products accumulate in f64 beyond per-thread
 * compensated f32 partial sums, Hessenberg/Givens in f64.  Then x += ||r|| d in
 * f64.  Needs DG_STORE_F64 and the inner copy in params.store.
 *   inner_m   1..64;  inner_tol in (0,1);  max_outer >= 1 corrections
 *   F device [dofs] f64 or NULL (assembled F); x device [dofs] f64 output
 *   info: iterations = inner Arnoldi steps in total, outer = corrections,
 *         relres = final f64 relative residual.
 * DG_NOT_CONVERGED after max_outer corrections or params.max_it inner steps.
 * Synchronises.
 */
dg_status dg_mixed_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                         const double* F, double* x, dg_solve_info* info);

/*
 * GMRES-based mixed-precision refinement: flexible GMRES(params.gmres_m) in f64
 * on the f64 blocks (f64 vectors, orthogonalisation and Givens), whose
 * preconditioner z = A_lo^-1 v is the low-precision solve of dg_mixed_solve
 * (f32 GMRES(inner_m) with block Jacobi on the f32 / bf16 copy, to inner_tol or
 * 8 restart cycles).  Where plain refinement stalls because cond(A) times the
 * unit roundoff of the inner copy is near or above 1 (bf16 on
 * convection-dominated operators), the outer Krylov method still converges.
 * Same arguments as dg_mixed_solve; max_outer caps the outer FGMRES steps
 * (one inner solve each), params.max_it the inner steps in total.
 *   info: iterations = inner Arnoldi steps in total, outer = outer FGMRES steps,
 *         restarts = outer restart cycles, relres = final f64 relative residual.
 * params.precond must be DG_PRECOND_BLOCK_JACOBI, DG_PRECOND_SCHWARZ or
 * DG_PRECOND_NONE (for the inner solve).  DG_NOT_CONVERGED when a cap is reached.  Synchronises.
 */
dg_status dg_gmres_ir_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                            const double* F, double* x, dg_solve_info* info);

/*
 * Direct solve Stiff x = F (the paper's coef = Stiff\F, Sec. 2.3) by dense LU
 * with partial pivoting on the device.  For small systems: dofs <= 4096.
 * The matrix is factored in f32 and the solution refined in f64 (residual
 * F - Stiff x with the f64 blocks, correction from the f32 factors) until
 * ||F - Stiff x||_inf <= sqrt(dofs) eps_f64 ||Stiff||_inf ||x||_inf, at most 10
 * steps; when that does not converge, or the f32 factorization meets a zero
 * pivot, the matrix is factored in f64 instead (also when the environment
 * variable DG_DENSE_F64=1 was set at dg_create).  F device or NULL (assembled
 * F; may equal x); x device output.  DG_ERR_SINGULAR_BLOCK when the f64
 * factorization meets a zero pivot.  Synchronises.
 */
dg_status dg_dense_solve(dg_handle* h, const double* F, double* x);

/* ------------------------------------------------------------------------ */
/* batches of independent instances                                          */
/* ------------------------------------------------------------------------ */
/*
 * Declare a batch.  The uploaded mesh (dg_mesh_upload) is the concatenation of
 * n_inst independent meshes: instance i owns elements [elem_start[i],
 * elem_start[i+1]) (host [n_inst+1], from 0 to ne); no edge may join two
 * instances (DG_ERR_MESH).  coeffs host [n_inst][8] = eps, alpha, b[0..5] of
 * each instance (Eq. (1)); degree, method and penalties come from the params
 * and are shared.  After this call dg_assemble assembles every instance with
 * its own coefficients in one pass (the eps/alpha/b of dg_coeffs are ignored;
 * f, gD, gN are read as usual over the whole concatenated mesh).
 */
dg_status dg_batch_setup(dg_handle* h, int n_inst, const int* elem_start, const double* coeffs);

/* Leave batch mode (dg_assemble uses dg_coeffs again). */
dg_status dg_batch_clear(dg_handle* h);

/* Choose the work-item size of the batched reductions (unknowns per item,
   from 2048 to 32768) by timing the batched multi-dot on the assembled batch;
   the choice is kept in the handle and returned in *tile.  Synchronises. */
dg_status dg_batch_autotune(dg_handle* h, int* tile);

/* Set the work-item size directly (256..2^20), or 0 for the default 4096. */
dg_status dg_batch_set_tile(dg_handle* h, int tile);

/*
 * Solve every instance of the batch.  inner_dtype DG_F64: restarted GMRES
 * (params.gmres_m) in f64 per instance, all instances advancing together with
 * per-instance reductions, Hessenberg/Givens and convergence.  DG_F32 /
 * DG_BF16: per-instance f64 iterative refinement (as dg_mixed_solve) around a
 * batched GMRES(inner_m) on f32 vectors with the f32 / bf16 block copy.
 * The preconditioner is params.precond (block Jacobi, Schwarz, the learned
 * correction or none).  Each instance stops when its own
 * ||F_i - A_i x_i|| / ||F_i|| <= params.tol.
 *   F device [dofs] f64 or NULL (assembled F); x device [dofs] f64 output;
 *   its, relres, status: host [n_inst] or NULL -- Arnoldi steps (inner steps
 *   summed over corrections), final f64 relative residual, DG_OK /
 *   DG_NOT_CONVERGED per instance.
 * Returns DG_NOT_CONVERGED if any instance missed the tolerance.  Synchronises.
 */
dg_status dg_batch_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                         const double* F, double* x, int* its, double* relres, int* status);

/*
 * GMRES-based refinement of every instance of the batch (the batched form of
 * dg_gmres_ir_solve): per instance, f64 flexible GMRES(params.gmres_m) on the
 * f64 operator whose preconditioner is the low-precision inner solve
 * z = A_lo^-1 v, a batched GMRES(inner_m) on f32 vectors with the f32 / bf16
 * block copy and params.precond (block Jacobi, Schwarz or none), stopped at
 * inner_tol or after 8 restart cycles.  All instances that take outer step j
 * run their inner solves together; each instance stops when its own
 * ||F_i - A_i x_i|| / ||F_i|| <= params.tol, after max_outer outer steps, or
 * once it has spent params.max_it inner steps.  Converges where plain
 * refinement stalls (restarted inner GMRES stagnating on diffusion-dominated
 * instances).  inner_dtype DG_F32 or DG_BF16; arguments as dg_batch_solve,
 * its = inner Arnoldi steps per instance.  DG_ERR_INVALID_ARG for
 * DG_PRECOND_MLP.  Synchronises.
 */
dg_status dg_batch_gmres_ir_solve(dg_handle* h, int inner_dtype, int inner_m, double inner_tol, int max_outer,
                                  const double* F, double* x, int* its, double* relres, int* status);

/*
 * A group of batches solved in one call: hs [nh] distinct handles, each set up
 * with dg_batch_setup (typically one batch per degree, since a handle's
 * kernels are specialised on its degree, when the instances of a workload
 * differ in degree).  Every batch is solved as by dg_batch_solve /
 * dg_batch_gmres_ir_solve with the shared arguments, each from its own host
 * thread on its handle's stream, so that the batches' launch sequences run on
 * the GPU at the same time; the call returns when all have finished.  Give
 * the handles different non-default streams to let them overlap (one stream
 * serialises them; the results are the same).
 *   F [nh] (or NULL: every batch's assembled F; an entry may be NULL), x [nh],
 *   its / relres / status [nh] (or NULL; an entry may be NULL): the per-batch
 *   arguments of the single-batch calls, all as there.
 * Returns the first error of a batch other than DG_NOT_CONVERGED, else
 * DG_NOT_CONVERGED if any instance of any batch missed the tolerance, else
 * DG_OK; each handle's dg_last_error describes its own batch.  Synchronises.
 * (Runtime; the paper has no counterpart.)
 */
dg_status dg_batch_group_solve(dg_handle* const* hs, int nh, int inner_dtype, int inner_m, double inner_tol,
                               int max_outer, const double* const* F, double* const* x, int* const* its,
                               double* const* relres, int* const* status);
dg_status dg_batch_group_gmres_ir_solve(dg_handle* const* hs, int nh, int inner_dtype, int inner_m,
                                        double inner_tol, int max_outer, const double* const* F, double* const* x,
                                        int* const* its, double* const* relres, int* const* status);

/* ------------------------------------------------------------------------ */
/* non-linear reaction (Sec. 3)                                               */
/* ------------------------------------------------------------------------ */
/*
 * The paper's nonlinear_global (Sec. 3, Eq. (nonlinsystem), (newton)) for
 * r(u) = c u^p (p = 1..4; the paper's example is u^2): at the coefficients x
 * (device [dofs] f64, the layout of dg_gmres_solve's x),
 *   H  device [dofs] f64:           H_i = int_K r(u_h) phi_i,
 *   HJ device [ne][nb][nb] f64 or NULL: HJ_K(i, j) = int_K r'(u_h) phi_j phi_i,
 * the element-diagonal blocks of dH/dx (row i test, column j trial), with
 * the volume rule of the assembly.  Needs an f64 assembly of the same
 * degree; not in batch mode.  Asynchronous on the handle's stream.
 */
dg_status dg_nonlinear_global(dg_handle* h, int p, double c, const double* x, double* H, double* HJ);

/*
 * Solve alpha u - eps Lap u + b.grad u + c u^p = f (Eq. (nonlin)), i.e.
 * A v + H(v) = F with A = D + C + R assembled by dg_assemble, by Newton's
 * method (Eq. (newton)): v^0 = 0; Res^k = A v^k + H(v^k) - F;
 * J^k = A + HJ(v^k); J^k w = -Res^k by restarted GMRES(params.gmres_m) with
 * params.precond (block Jacobi, Schwarz or none) set up on J^k, to relative
 * residual lin_tol; v^{k+1} = v^k + w.  Stops when ||Res^k|| <= params.tol
 * ||F|| (DG_OK) or after max_newton corrections (DG_NOT_CONVERGED).
 *   F device [dofs] f64 or NULL (assembled F); x device [dofs] f64 output.
 *   info: outer = Newton corrections, iterations = GMRES steps summed,
 *         relres = final ||Res|| / ||F||.
 * DG_ERR_INVALID_ARG for p outside 1..4, max_newton < 1, lin_tol outside
 * (0,1) or DG_PRECOND_MLP.  The preconditioner is left set up on the last
 * Jacobian and is rebuilt by the next solve.  Synchronises.
 */
dg_status dg_newton_solve(dg_handle* h, int p, double c, int max_newton, double lin_tol, const double* F, double* x,
                          dg_solve_info* info);

/* ------------------------------------------------------------------------ */
/* learned right preconditioner (not in the paper; layered on its method)    */
/* ------------------------------------------------------------------------ */
/*
 * An element-local MLP corrects block Jacobi towards the one-layer-overlap
 * Schwarz correction it is trained on: for element K with face
 * neighbours L0..L2 and residual r, with s = sqrt(sum of r^2 over K and its
 * neighbours / (4 nb)),
 *   x   = [r_K, r_L0, r_L1, r_L2]/s ++ [log10(eps)/6 + 1, b_x, b_y, alpha,
 *          J/sqrt(det J) (4 entries)]                               (din = 4nb+8),
 *   y   = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4   (width 128),
 *   z_K = A_KK^-1 (r_K + s sigma y_K)        (A_KK^-1: the block-Jacobi inverse),
 * b at the element centroid, J the element's affine map, sigma a fixed output
 * scale set when training starts.
 * The network is nonlinear, so params.precond = DG_PRECOND_MLP makes
 * dg_gmres_solve / dg_batch_solve run flexible GMRES; if two consecutive
 * restart cycles cut the true residual by less than 10% the correction is
 * switched off and block Jacobi finishes the solve (info.outer = -1 then).
 * Parameters: one flat f32 vector W1 [128][din], b1, W2 [128][128], b2, W3,
 * b3, W4 [nb][128], b4 (row-major), sigma; inference uses them rounded to bf16 on the
 * tensor cores (tcgen05, f32 accumulation in tensor memory; the features, the
 * output scaling and A_KK^-1 in f32), training uses the same bf16-rounded
 * values in f32 GEMMs and updates f32 master weights with Adam.
 */
dg_status dg_mlp_num_params(int degree, int64_t* n);
/* Initialise the weights for params.degree (uniform He-style, counter-based hash of seed). */
dg_status dg_mlp_init(dg_handle* h, uint64_t seed);
/* Host copies of the f32 master weights (n = dg_mlp_num_params). */
dg_status dg_mlp_set_weights(dg_handle* h, const float* theta, int64_t n);
dg_status dg_mlp_get_weights(dg_handle* h, float* theta, int64_t n);
/* Append one training row per element from an iterate xk of a solve:
   r = F - A xk (device [dofs] f64; F NULL = the assembled F); the correction
   paired with r is the one-layer-overlap patch solve w (w_K from A_P w = r_P on
   K and its face neighbours), target (A_KK w_K - r_K)/s. */
dg_status dg_mlp_collect(dg_handle* h, const double* F, const double* xk);
/* The same for the first nvec Krylov basis vectors of the last f64 solve
   (dg_gmres_solve, or dg_batch_solve with DG_F64): the vectors the
   preconditioner is applied to inside GMRES.  nvec <= params.gmres_m + 1.
   DG_ERR_STATE when no f64 solve ran since the last solver call of another
   kind (the basis is then gone). */
dg_status dg_mlp_collect_basis(dg_handle* h, int nvec);
dg_status dg_mlp_num_rows(dg_handle* h, int64_t* rows);
dg_status dg_mlp_get_rows(dg_handle* h, float* X, float* T, int64_t max_rows);   /* host outputs */
dg_status dg_mlp_clear_data(dg_handle* h);
/* Adam on random mini-batches of the collected rows: `steps` updates of
   batch_rows rows each, learning rate lr; loss host [steps] or NULL.  The
   forward and backward GEMMs of each step run on the tcgen05 tensor cores
   (bf16 operands, f32 accumulation in tensor memory; the weight gradients'
   sums over the rows split over CTAs and reduced in a fixed order).
   DG_ERR_TIMEOUT when a tensor-core kernel gave up waiting for its MMAs.
   Synchronises. */
dg_status dg_mlp_train(dg_handle* h, int steps, int batch_rows, float lr, uint64_t seed, float* loss);
/* Loss (mean 0.5|y-t|^2) and gradient at the current weights on caller rows
   X device [rows][din], T device [rows][nb] (f32); loss, grad host.  The GEMMs
   run in f32 on the CUDA cores; with the environment variable DG_MLP_GRAD_TC=1
   set at dg_create they run on the tensor cores as in dg_mlp_train (then
   DG_ERR_TIMEOUT as there).  Synchronises. */
dg_status dg_mlp_loss_grad(dg_handle* h, const float* X, const float* T, int rows, double* loss, float* grad);
/* Tensor-core forward pass y on caller feature rows: X device [rows][din], Y device [rows][nb] (f32).
   The inference kernel (tcgen05 MMAs with accumulators in tensor memory)
   bounds its waits on the MMAs: DG_ERR_TIMEOUT if one ran out, here and in the
   flexible solves that apply the network.  Synchronises. */
dg_status dg_mlp_forward(dg_handle* h, const float* X, int rows, float* Y);

/* ------------------------------------------------------------------------ */
/* post-processing  (the paper's dg_error, Sec. 2.4)                        */
/* ------------------------------------------------------------------------ */
/*
 * L2 error ||u_h - u||_{L2(Omega)} with u given at DG_POINTS_ERROR (device
 * [ne][(k+4)^2] f64), and h_max = the longest mesh edge.  l2 and hmax are
 * host outputs (either may be NULL).  Synchronises.
 */
dg_status dg_l2_error(dg_handle* h, const double* x, const double* uex_q, double* l2, double* hmax);

/*
 * u_h at np points given in reference coordinates (host rs[np][2], inside the
 * reference triangle (0,0),(1,0),(0,1)), in every element: device out[ne][np].
 */
dg_status dg_eval(dg_handle* h, const double* x, int np, const double* rs, double* out);

/*
 * dg_l2_error without any device allocation.  Same inputs, outputs and result
 * as dg_l2_error (the paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory, e.g. when another allocator owns
 * all of it or a timing-critical loop must not call cudaMalloc).
 * Its reduction scratch is a fixed array inside the library (16385 doubles per
 * GPU, kept until the process exits), which limits the mesh to 4,194,304
 * elements (DG_ERR_INVALID_ARG beyond).  The handle's reference tables must
 * already exist: call dg_quad_points, dg_boundary_info or dg_assemble once
 * for the current degree first (DG_ERR_STATE otherwise).  dg_create looks up
 * the array's device address (cudaGetSymbolAddress, with the handle's device
 * current); that lookup makes the CUDA runtime load the module holding the
 * array, so the array's device memory is allocated when the first handle is
 * created on a device, not in a dg_l2_error_noalloc call.  If the current
 * CUDA context has changed since (device reset, primary context released and
 * created again), the call looks the address up anew before launching,
 * which loads the module into the new context; make calls after such a
 * change, like the first handle creation, outside any stream capture.  All calls
 * share the array: calls whose GPU work overlaps (other streams or handles on
 * the same device) race on it and must be serialised by the caller.
 * Synchronises the handle's stream.
 */
dg_status dg_l2_error_noalloc(dg_handle* h, const double* x, const double* uex_q, double* l2, double* hmax);

/* ------------------------------------------------------------------------ */
/* instrumentation                                                           */
/* ------------------------------------------------------------------------ */
/*
 * Average device time (CUDA events on the handle's stream) of one solver
 * kernel run in isolation on the handle's GMRES workspace, for roofline
 * accounting: which = DG_PROF_DOTS (the multi-dot of an Arnoldi step) or
 * DG_PROF_UPDATE (its Gram-Schmidt update), at step `param` = j (0 <= j <
 * gmres_m), for dtype DG_F64 (f64 vectors) or DG_F32 (f32 vectors); or
 * which = DG_PROF_APPLY, the operator apply of Sec. 2.3 (dg_apply) with the
 * block copy dtype = DG_F64, DG_F32 or DG_BF16 (param ignored; f32 vectors
 * for the low-precision copies), the rest of the workspace read before each
 * launch so that the operator is not left in L2 when the basis is larger
 * than L2.
 * Averaged over reps launches.  Overwrites the workspace.  Synchronises.
 * Errors: DG_ERR_STATE (not assembled, or the requested block copy not
 * stored), DG_ERR_INVALID_ARG (which, dtype, param).
 */
#define DG_PROF_DOTS   1
#define DG_PROF_UPDATE 2
#define DG_PROF_APPLY  3
dg_status dg_profile_kernel(dg_handle* h, int which, int dtype, int param, int reps, double* avg_ms);

/* Number of CUDA kernels this handle has launched so far (a graph launch
   counts each kernel node of the graph).  Host counter, no synchronisation. */
dg_status dg_get_launch_count(dg_handle* h, int64_t* count);

/* ------------------------------------------------------------------------ */
/* host-only helpers (no GPU needed)                                         */
/* ------------------------------------------------------------------------ */
/* Orthonormal Dubiner basis of degree k on the reference triangle and its
   reference gradients at np host points rs[np][2]: phi, dr, ds host
   [np][nb] (dr, ds may be NULL). */
dg_status dg_reference_basis(int degree, int np, const double* rs, double* phi, double* dr, double* ds);

/* The library's quadrature rule `which` (DG_POINTS_*) on the reference
   triangle (VOLUME, ERROR: rs[n][2], w[n], weights sum to 1/2) or on [0,1]
   (BOUNDARY: rs[n][0] = t, rs[n][1] = 0, w[n] sums to 1); n given by dg_info
   sizes for degree k.  Returns the number of points through *n. */
dg_status dg_reference_rule(int which, int degree, double* rs, double* w, int* n);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
