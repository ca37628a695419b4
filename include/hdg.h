/*
 * hdg.h — C ABI of the GB300 library for the hp-multigrid preconditioned
 * flexible GMRES solver of the statically condensed H(div)-HDG discretisation
 * of the generalized Stokes equation and of the Oseen equation (the Picard
 * linearisation of the Navier-Stokes equations, Section 4) with an
 * augmented-Lagrangian term (G. Fu & W. Kuang, "hp-multigrid preconditioner for a divergence-conforming
 * HDG scheme for the incompressible flow problems").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Meshes: conforming triangulations (dim = 2) given level by level, level 0
 * the coarsest, each finer level a uniform (red) refinement of the previous
 * one (Section 3.4.2).  Local facet f of a cell is the facet opposite local
 * vertex f.  Facets are numbered in lexicographic order of their sorted
 * global vertex pair; a facet is oriented from its lower to its higher
 * global vertex id (unit tangent t_F, unit normal n_F = (t_y, -t_x), facet
 * parameter s in [0,1] from the lower vertex).  Boundary facets carry the
 * homogeneous Dirichlet condition (Section 3.1) and own no unknowns.
 *
 * Skeleton vectors (order k): for every interior facet, in facet order,
 * dpf = 2(k+1) doubles: the normal moments  int_F (u.n_F) l_m ds, m = 0..k,
 * then the tangential coefficients of the facet unknown in the same basis,
 * where l_m = sqrt(2m+1) P_m(2s-1) / sqrt|F| is L2-orthonormal on F.
 * n_dof = n_interior_facets * dpf.  Vectors are dual (load/residual) or
 * primal (solution) in this one layout; the condensed operator is the
 * matrix of the bilinear form in this basis.
 *
 * Element matrices: per cell, n_loc x n_loc with n_loc = 3 dpf, row-major,
 * local unknown order facet 0,1,2 and within a facet the dpf unknowns above
 * (boundary facets included: the matrix is the cell's own Schur complement).
 *
 * Forcing: per cell, the values of f_h in [P^{k+1}(K)]^2 at the degree-(k+1)
 * lattice, points x = v0 + (a1/q)(v1-v0) + (a2/q)(v2-v0) with q = k+1,
 * ordered a2 = 0..q outer, a1 = 0..q-a2 inner, each point 2 doubles (x, y
 * components).  Layout [n_cells][n_lat][2], n_lat = (q+1)(q+2)/2.
 *
 * Pressure: one double per cell (the cell-constant pressure p^∂ of the
 * condensed saddle point, eq. stOptForm).
 *
 * Tetrahedra (dim = 3; the generalized Stokes operator; Section 3.4.2 edge
 * patches): local face f is opposite local vertex f; faces are numbered in
 * lexicographic order of their sorted global vertex triple a < b < c, with
 * the frame t1 = (x_b - x_a)/|.|, n_F = (x_b - x_a) x (x_c - x_a)/|.|,
 * t2 = n_F x t1 and the scalar basis l_m: the L2(F)-orthonormal Gram-Schmidt
 * basis of lambda_b^i lambda_c^j (i + j <= k, by degree then j) in the
 * barycentrics of x_b, x_c.  An interior face owns dpf = 3 nf doubles,
 * nf = (k+1)(k+2)/2: the normal moments int_F (u.n_F) l_m dS, then the t1 and
 * the t2 coefficients of the tangential unknown.  Element matrices have
 * n_loc = 4 dpf.  Forcing: [n_cells][n_lat][3] at the points
 * v0 + (a1/q)(v1-v0) + (a2/q)(v2-v0) + (a3/q)(v3-v0), a3 outer, then a2, a1
 * inner, n_lat = (q+1)(q+2)(q+3)/6.  The lowest-order levels carry 3 unknowns
 * per face.  Calls available on tetrahedra: hdg_setup_mesh_hierarchy,
 * hdg_check_hierarchy, hdg_condense (FP64 or FP32 preconditioner, block GS,
 * scalar nu, no convection, k <= 3; Dirichlet data as faces' normal moments
 * and t1, t2 coefficients), hdg_load, hdg_apply,
 * hdg_level_apply, hdg_smooth, hdg_prolong_add, hdg_restrict,
 * hdg_coarse_solve, hdg_mg_h, hdg_precond_apply, hdg_get_element_matrices,
 * hdg_solve, hdg_recover, hdg_postprocess (u* in [P^{k+1}]^3 at the lattice,
 * [n_cells][n_lat][3]), hdg_boundary_facets (sorted vertex triples),
 * hdg_get_sizes; the others return
 * HDG_ERR_UNSUPPORTED.
 *
 * Memory: pointers documented "device" must be device memory on the
 * context's device; "host" pointers are host memory.  The caller owns every
 * buffer it passes; the context owns the mesh data, element and patch
 * matrices and all workspaces and frees them in hdg_destroy.
 *
 * Streams: every call that takes a stream enqueues its work on that stream
 * (NULL = legacy default stream).  hdg_condense and hdg_solve synchronise
 * the stream before returning so that their status is final.
 *
 * Errors: no exception crosses the ABI.  Each call returns an hdg_status;
 * hdg_last_error(ctx) gives a message for the last failure on the context.
 * After HDG_ERR_CUDA the context must be destroyed.  One context per host
 * thread at a time.
 */
#ifndef HDG_H
#define HDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;
typedef struct CUstream_st *hdg_stream_t;   /* the cudaStream_t type */

typedef enum {
    HDG_OK = 0,
    HDG_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range          */
    HDG_ERR_OOM = 2,           /* device or host allocation failed                  */
    HDG_ERR_CUDA = 3,          /* a CUDA runtime call or kernel failed              */
    HDG_ERR_SINGULAR = 4,      /* a local, patch or coarse matrix has a pivot <= 0  */
    HDG_ERR_NOT_CONVERGED = 5, /* iteration limit reached before the tolerance      */
    HDG_ERR_BREAKDOWN = 6,     /* Krylov breakdown with a nonzero residual          */
    HDG_ERR_NONFINITE = 7,     /* NaN or Inf in a residual                          */
    HDG_ERR_UNSUPPORTED = 8,   /* valid request this build does not implement       */
    HDG_ERR_STATE = 9,         /* call order violated (e.g. solve before condense)  */
    HDG_ERR_TIMEOUT = 10       /* a bounded device wait gave up (a kernel skipped   */
                               /* its update; the result of the call is invalid);   */
                               /* checked at the end of hdg_solve, hdg_picard,      */
                               /* hdg_newton, hdg_adjoint, hdg_precond_apply and    */
                               /* hdg_smooth (see hdg_set_wait_limit)               */
} hdg_status;

typedef enum {
    HDG_FP64 = 0,        /* preconditioner in FP64                                 */
    HDG_MIXED_FP32 = 1,  /* preconditioner (smoothers, transfers, V-cycle) in FP32; */
                         /* outer operator, Krylov, coarse solve stay FP64          */
    HDG_MIXED_BF16 = 2,  /* as HDG_MIXED_FP32, but the order-k element matrices and */
                         /* patch inverses read by the order-k smoother and its     */
                         /* residual are stored in bfloat16, each row scaled by its */
                         /* own power of two (largest entry in [1/2, 1)); products  */
                         /* accumulate in FP32.  Single-load calls only: batched    */
                         /* (_multi) calls read the FP32 copies                     */
    HDG_MIXED_FP16 = 3   /* the same with IEEE binary16 storage                     */
} hdg_precision;

typedef struct {
    int dim;                              /* 2 (triangles) or 3 (tetrahedra, a red- */
                                          /* refined hierarchy; edge patches)       */
    int n_levels;                         /* >= 1, level 0 = coarsest               */
    const int64_t *n_vertices;            /* host [n_levels]                        */
    const int64_t *n_cells;               /* host [n_levels]                        */
    const double *const *coords;          /* host [n_levels] -> [n_vertices*dim]    */
    const int32_t *const *cells;          /* host [n_levels] -> [n_cells*(dim+1)]   */
    const int32_t *const *parent;         /* host [n_levels] -> [n_cells]: cell of  */
                                          /* level l-1 containing each cell of l;   */
                                          /* entry 0 is ignored                      */
    const int32_t *const *vertex_colour;  /* host [n_levels] -> [n_vertices] proper */
                                          /* colouring, or NULL / NULL entries for  */
                                          /* greedy colouring in vertex-id order    */
} hdg_mesh_desc;

typedef struct {
    int k;                   /* polynomial order of the finest space, 0..4         */
    double nu;               /* viscosity nu > 0                                   */
    double beta;             /* lower-order coefficient beta >= 0                  */
    double gamma;            /* augmented-Lagrangian weight: eps^{-1} = gamma*nu   */
    int m_p;                 /* high-order relaxation steps (Algorithm 2), >= 1    */
    int m_h;                 /* smoothing steps on the finest CR level, >= 1       */
    int cycle;               /* q of Algorithm 1: 1 = variable V, 2 = W            */
    int vcycle_growth;       /* m(l-1) = growth * m(l) for q = 1 (2 = doubling)    */
    hdg_precision precision; /* precision of the preconditioner                    */
    int fused_coarse_cells;  /* run MG_h on the coarsest levels with at most this  */
                             /* many cells in one thread block (0 = off; <= 2048)  */
    const double *nu_elem;   /* device [n_cells finest] per-cell viscosity, or     */
                             /* NULL for the scalar nu; coarser levels use the     */
                             /* mean over each cell's children                     */
    const double *conv;      /* Oseen problem (Section 4.1, Picard form of eq.     */
                             /* nsWeak with a fixed convecting field w_h): device  */
                             /* [n_cells finest][n_lat][2], physical components of */
                             /* w_h at each cell's degree-(k+1) lattice (the       */
                             /* forcing layout); copied by hdg_condense.  w_h      */
                             /* should be divergence free, normal-continuous and   */
                             /* tangential on the boundary (e.g. the curl of a     */
                             /* continuous stream function).  Lowest-order levels  */
                             /* use the RT_0 field with the facet fluxes of w_h    */
                             /* (mean of the two sides), summed over the fine      */
                             /* halves of each coarse facet.  NULL = generalized   */
                             /* Stokes.                                            */
    const double *newton_u;  /* Newton step of Algorithm 3 (Section 4.2): device   */
                             /* [n_dof], the previous skeleton iterate u_old, with */
                             /* conv = u_old at the lattice.  Adds the derivative  */
                             /* of the upwind form in its convecting argument (the */
                             /* switch frozen at u_old·n) to the order-k operator  */
                             /* and C_h(u_old; u_old, v) to the load, so that the  */
                             /* solution is the new iterate.  Lowest-order levels  */
                             /* keep the Picard form.  NULL = no Newton term.      */
    int smoother;            /* block smoother of every level (eq. bjac): 0 = block */
                             /* Gauss-Seidel in colour order (Section 5), 1 =      */
                             /* damped block Jacobi (all patches against one       */
                             /* residual, corrections summed, times the damping)   */
    double jacobi_damping;   /* the damping of smoother 1; <= 0 selects 0.5        */
    int hp_additive;         /* 0 = Algorithm 2 (multiplicative); 1 = its additive  */
                             /* form (Remark 3.4): z = R_sym r + Pi_0^k MG_h(Pi_k^0 */
                             /* r), R_sym = m_p forward then m_p backward sweeps    */
                             /* from zero; single-load calls only                   */
    const double *dirichlet; /* inhomogeneous Dirichlet data (Section 3.1 with      */
                             /* u = g on the boundary, e.g. a driven lid): device   */
                             /* [n_boundary_facets][dpf], for every boundary facet  */
                             /* of the finest level in hdg_boundary_facets order,   */
                             /* the skeleton values of g in the unknowns' layout:   */
                             /* normal moments int_F (g.n_F) l_m, then tangential   */
                             /* coefficients int_F (g.t_F) l_m.  Copied by          */
                             /* hdg_condense.  The loads of hdg_condense / hdg_load */
                             /* then carry -A_IB g, the pressure update of hdg_solve */
                             /* the data's boundary fluxes (which must sum to zero),*/
                             /* and hdg_recover / hdg_postprocess use g on the      */
                             /* boundary.  Preconditioners act on homogeneous       */
                             /* corrections and are unchanged.  NULL = homogeneous. */
                             /* hdg_solve only: batched solves, hdg_picard,         */
                             /* hdg_newton and hdg_adjoint return                   */
                             /* HDG_ERR_UNSUPPORTED with data set.                  */
    double pseudo_dt_inv;    /* hdg_picard only: pseudo-time continuation (Section  */
                             /* 5.2.2), 1/dt* >= 0.  Each Oseen step n >= 1 then    */
                             /* solves the backward-Euler step (u^n - u^{n-1})/dt*  */
                             /* + (Oseen operator) u^n = f, i.e. beta + 1/dt* and   */
                             /* the load f + u^{n-1}/dt* (u^{n-1} at the lattice,   */
                             /* exact since RT_k lies in [P^{k+1}]^2); a fixed      */
                             /* point is the steady solution.  0 = plain Picard.    */
} hdg_params;

typedef struct {
    double rtol;        /* inner relative tolerance (Section 5: 1e-8)               */
    double atol;        /* inner absolute tolerance (Section 5: 1e-10)              */
    double floor_rel;   /* inner solves stop at <= floor_rel*|F| at the latest      */
    double uzawa_tol;   /* stop when the pressure error estimate <= uzawa_tol |p|   */
    int restart;        /* FGMRES restart length, 1..64 (batched solves: 1..32)     */
    int max_it;         /* FGMRES iterations per inner solve                        */
    int max_uzawa;      /* Uzawa steps, 1..64                                       */
    int krylov;         /* inner Krylov method: 0 = flexible GMRES (restart);       */
                        /* 1 = preconditioned CG (the paper's method for the        */
                        /* generalized Stokes problem, Section 5; needs a symmetric */
                        /* operator and preconditioner: no convection, FP64 or the  */
                        /* FP32 preconditioner).  Same stopping norm and targets.   */
                        /* Single-load solves only.                                 */
} hdg_solve_opts;

typedef struct {
    int uzawa_its;              /* Uzawa steps taken                                */
    int krylov_its_total;       /* FGMRES iterations summed over the Uzawa steps   */
    int krylov_its[64];         /* per Uzawa step                                   */
    double res_mom;             /* final |g - A^eps u| of the last inner solve      */
    double dp_rel;              /* last |p^n - p^{n-1}|_L2 / |p^n|_L2               */
    double normF;               /* |F|_2                                            */
    double div_l2;              /* |div u_h|_L2(Omega) of the returned velocity     */
                                /* (div u_h is constant on each cell: its facet     */
                                /* fluxes over |K|); -1 from the batched solves     */
    double res_floor;           /* the inner solves' final absolute floor: the      */
                                /* larger of floor_rel |F|, atol and twice the      */
                                /* residual at which an inner FGMRES stagnated on   */
                                /* round-off (a restart cycle whose Givens estimate */
                                /* met the tolerance but whose true residual fell   */
                                /* by less than half; Remark 3.1)                   */
} hdg_solve_info;

typedef struct {
    int k;
    int n_levels;
    int64_t n_cells;            /* finest level                                     */
    int64_t n_interior_facets;  /* finest level                                     */
    int64_t n_dof;              /* order-k skeleton unknowns, finest level          */
    int64_t n_dof_level[16];    /* lowest-order unknowns per level (2 per facet)    */
    int n_colours_level[16];    /* vertex colours per level                         */
    int n_lat;                  /* forcing lattice points per cell                  */
    int64_t n_boundary_facets;  /* finest level; the order of hdg_boundary_facets   */
} hdg_sizes;

/* Fill the defaults of Section 5: rtol 1e-8, atol 1e-10, floor_rel 1e-10,
 * uzawa_tol 1e-8, restart 30, max_it 1000, max_uzawa 64, krylov 0 (FGMRES). */
void hdg_default_solve_opts(hdg_solve_opts *opts);

/* Sizes of a checked hierarchy (finest level). */
typedef struct {
    int n_levels;
    int64_t n_interior_facets;
    int64_t n_dof;            /* n_interior_facets * 2(k+1)                           */
    int n_patches;            /* vertex patches (vertices with an interior facet)     */
    int n_colours;            /* colours of the vertex colouring (colour phases)      */
    int max_patch_facets;     /* interior facets of the largest patch                 */
    int max_patch_cells;      /* cells of the largest star                            */
} hdg_hierarchy_info;

/* Validates a mesh hierarchy on the host, with no device call: every check of
 * hdg_setup_mesh_hierarchy (cell indices, manifold facets, a proper vertex
 * colouring, red-refinement parent maps) and the construction of its vertex
 * patches and transfer tables.  info (nullable) receives the finest level's
 * sizes for polynomial order k; on failure msg (nullable, msg_len bytes)
 * receives the reason.  Returns HDG_OK or HDG_ERR_INVALID_ARG. */
hdg_status hdg_check_hierarchy(const hdg_mesh_desc *desc, int k, hdg_hierarchy_info *info, char *msg,
                               int msg_len);

/* Build the topology of every level: facets, orientations, interior-facet
 * numbering, vertex patches and their colouring, parent/child maps and the
 * coarse-facet/fine-facet relations needed by the averaging transfer of
 * eq. avgOpt (Sections 2, 3.4.2).  Host arrays are copied; the caller may
 * free them on return.  device: CUDA ordinal.  Returns HDG_ERR_INVALID_ARG
 * for dim != 2, n_levels outside 1..16, inconsistent parents or a colouring
 * that is not proper. */
hdg_status hdg_setup_mesh_hierarchy(const hdg_mesh_desc *desc, int device, hdg_ctx **out);

/* Static condensation (Section 3.2, eq. stWeak; AL term eq. stALform) of the
 * order-k operator on the finest level and of the lowest-order operator on
 * every level, in FP64 on the device; then the patch inverses of the block
 * smoothers (eq. bjac, Sections 3.4.2, 3.5), the harmonic-extension blocks of
 * the transfer (eqs. div-transfer, harmonic-ex) and the dense inverse of the
 * coarsest operator (at most 16384 coarsest unknowns, else
 * HDG_ERR_INVALID_ARG).  With params->conv the local systems carry the upwind
 * convection of Section 4.1 and are eliminated by LU; the patch, transfer and
 * coarse factorisations are the same (Section 4.2).  forcing: device [n_cells][n_lat][2] (layout above) or
 * NULL; rhs_out: device [n_dof] condensed load F, or NULL.  May be called
 * again with new parameters or forcing.  Returns HDG_ERR_SINGULAR if a
 * factorisation meets a non-positive pivot. */
hdg_status hdg_condense(hdg_ctx *ctx, const hdg_params *params, const double *forcing,
                        double *rhs_out, hdg_stream_t stream);

/* Condensed load only (forcing -> F, device in/out), reusing the condensed
 * cells of the last hdg_condense.  Same layouts as hdg_condense. */
hdg_status hdg_load(hdg_ctx *ctx, const double *forcing, double *rhs_out, hdg_stream_t stream);

/* y = A^eps_{k,h} x (eqs. stOptForm, stALform): element-by-element Schur
 * complements gathered and summed per facet.  x, y: device [n_dof] FP64,
 * must not overlap. */
hdg_status hdg_apply(hdg_ctx *ctx, const double *x, double *y, hdg_stream_t stream);

/* y = (A^eps)^T x on a level (level = -1: the order-k operator, >= 0: the
 * lowest-order operator of that level): the transposed condensed operator,
 * which differs from A^eps for the Oseen and Newton operators (the upwind
 * convection is not symmetric) and equals it for the generalized Stokes
 * problem.  x, y: device FP64 of the level's size, must not overlap. */
hdg_status hdg_apply_transpose(hdg_ctx *ctx, int level, const double *x, double *y, hdg_stream_t stream);

/* z = MG_hp(r, 0, m_p, m_h, q) of Algorithm 2 (Algorithm 1 inside), in the
 * precision chosen at hdg_condense.  r, z: device [n_dof] FP64, must not
 * overlap. */
hdg_status hdg_precond_apply(hdg_ctx *ctx, const double *r, double *z, hdg_stream_t stream);

/* Augmented-Lagrangian Uzawa iteration (eq. stOpEq-ALU, with the convergent
 * sign p <- p - eps^{-1} div u) with FGMRES inner solves right-preconditioned
 * by MG_hp.  F: device [n_dof] condensed load; u: device [n_dof], in: initial
 * guess, out: skeleton velocity; p: device [n_cells], in: initial pressure,
 * out: cell pressures.  opts NULL = defaults.  info may be NULL.  Returns
 * HDG_ERR_NOT_CONVERGED when max_uzawa or max_it is reached. */
hdg_status hdg_solve(hdg_ctx *ctx, const double *F, double *u, double *p,
                     const hdg_solve_opts *opts, hdg_solve_info *info, hdg_stream_t stream);

/* Local fields of a skeleton solution (Section 3.2: "we recover the local
 * variables in an element-by-element manner"): the cell unknowns eliminated
 * by hdg_condense are recomputed from u (device [n_dof]) and the forcing
 * (device lattice layout, or NULL for zero forcing) with the current
 * parameters.  Outputs (device, each may be NULL):
 *   L_out    [n_cells][4][npk]: coefficients of L_h = -nu grad u in the
 *            orthonormal P^k basis of each cell, components (xx, xy, yx, yy),
 *            npk = (k+1)(k+2)/2 (basis: csrc/reference.cpp);
 *   ulat_out [n_cells][n_lat][2]: u_h at the degree-(k+1) lattice points, which
 *            determine u_h exactly (RT_k is contained in [P^{k+1}]^2).
 * On tetrahedra: L_out [n_cells][9][npk] (components xx, xy, xz, yx, ..., zz over
 * the orthonormal P^k basis of the reference tetrahedron composed with the cell's
 * affine map, csrc/reference3d.cpp; npk = (k+1)(k+2)(k+3)/6) and ulat_out
 * [n_cells][n_lat][3] (n_lat = (k+2)(k+3)(k+4)/6). */
hdg_status hdg_recover(hdg_ctx *ctx, const double *u, const double *forcing, double *L_out,
                       double *ulat_out, hdg_stream_t stream);

/* Local post-processing of eq. stPost (Section 5.1): per cell, u* in
 * [P^{k+1}(K)]^2 with (grad u*, grad v)_K = (-nu^{-1} L_h, grad v)_K for all v
 * in P^{k+1}(K) and (u*, 1)_K = (u_h, 1)_K (the equation read with L = -nu grad u,
 * so that grad u* approximates grad u; u* converges at order k+2 for k >= 1).
 * L_h and u_h are recovered from the skeleton solution u (device [n_dof]) and
 * the forcing (device lattice layout, or NULL for zero forcing) as in
 * hdg_recover.  ustar_out: device [n_cells][n_lat][2], the values of u* at the
 * degree-(k+1) lattice of each cell (the forcing layout; they determine u*). */
hdg_status hdg_postprocess(hdg_ctx *ctx, const double *u, const double *forcing, double *ustar_out,
                           hdg_stream_t stream);

/* Adjoint gradients of J = 1/2 ||u_h - u_target||^2_{L2(Omega)} with respect
 * to the forcing lattice values and the per-cell viscosity (Section 3.2 scheme,
 * differentiated through the discrete solution).  For the generalized Stokes
 * system the transposed local system equals the primal one with the signs of
 * the flux and pressure blocks flipped, so the adjoint is solved with the same
 * condensed operator and hp-multigrid preconditioner (hdg_solve with opts) for
 * the load (u_h - u_target, v); then dJ/dnu_K = -nu_K^{-2} (L_h, L^a)_K and
 * dJ/df_h = (u^a, lambda_n e_c)_K.  The discrete solution, hence J, does not
 * depend on the augmented-Lagrangian weight.
 * Oseen: the transposed local system is the primal one with the convection
 * block transposed (the other blocks as above), so hdg_adjoint rebuilds every
 * level's operators from the transposed convection, solves, and rebuilds the
 * primal operators before returning (two extra condensations per call).
 *   forcing:  device lattice layout, the forcing of the primal solve;
 *   u:        device [n_dof], the primal skeleton solution (from hdg_solve);
 *   u_target: device [n_cells][n_lat][2], lattice samples of the target;
 *   grad_forcing: device out, lattice layout, or NULL;
 *   grad_nu:  device out [n_cells], or NULL;
 *   J:        host out (the objective), or NULL;
 *   opts/info as hdg_solve (info describes the adjoint solve). */
hdg_status hdg_adjoint(hdg_ctx *ctx, const double *forcing, const double *u, const double *u_target,
                       double *grad_forcing, double *grad_nu, double *J, const hdg_solve_opts *opts,
                       hdg_solve_info *info, hdg_stream_t stream);

/* Multi-right-hand-side (batched) forms: nrhs systems with the one condensed
 * operator of the last hdg_condense (several loads on one mesh).  Vectors are
 * right-hand-side major, x[r * n + i] for r < nrhs (1 <= nrhs <= 64), device
 * FP64, n = n_dof (pressures: n = n_cells).  Internally the columns are
 * interleaved row by row, with nrhs padded to a power of two by zero columns,
 * so that every element-matrix and patch-inverse entry read from memory serves
 * all columns; each column keeps its own FGMRES least-squares problem,
 * tolerances and Uzawa stopping decisions, exactly as hdg_solve applies them
 * to one load.  Results match nrhs calls of the single forms up to rounding. */
#define HDG_MAX_NRHS 64

/* Y = A^eps X. */
hdg_status hdg_apply_multi(hdg_ctx *ctx, int nrhs, const double *x, double *y, hdg_stream_t stream);

/* Z = MG_hp(R) column by column, in the precision chosen at hdg_condense.  With
 * HDG_MIXED_FP16 / HDG_MIXED_BF16, k = 3 and 9..64 columns the order-k sweeps
 * run on tensor cores (mma.sync, 16-bit operands, FP32 accumulation, eq. bjac
 * with GS as in hdg_smooth): the element rows and patch inverses come from the
 * 16-bit row-scaled copies, and per patch the gathered unknowns and the patch
 * residual of each column are rounded to the 16-bit format after a power-of-
 * two scale that brings the column's largest magnitude into [1/2, 1). */
hdg_status hdg_precond_apply_multi(hdg_ctx *ctx, int nrhs, const double *r, double *z, hdg_stream_t stream);

/* hdg_smooth for nrhs columns: n_sweeps block-GS sweeps of level `level`
 * (-1 = the order-k level) on U[r] with right-hand side G[r], in the sweep
 * kernels hdg_precond_apply_multi uses. */
hdg_status hdg_smooth_multi(hdg_ctx *ctx, int level, int nrhs, const double *g, double *u, int n_sweeps,
                            int reverse, hdg_stream_t stream);

/* Tile of the batched order-k sweep on CUDA cores (the FP64 and FP32 forms):
 * rows of one column per thread (1, 2 or 4, dividing 2(k+1)) and threads per
 * block (128 or 256).  By default an autotuner picks it at the first batched
 * preconditioner application for each precision and padded width: it times one
 * colour phase of the finest level for every pair on scratch vectors and keeps
 * the fastest.  All pairs give bitwise-identical results.
 * The tensor-core sweep (16-bit precisions, k = 3) is tuned the same way over
 * its block size (128 or 256 threads; bitwise-identical results).
 * hdg_set_batched_tile forces a pair for this context (0, 0 = back to the
 * autotuner; the tensor-core sweep takes the forced thread count).
 * hdg_tune_batched runs the autotuner now for width nrhs and returns its choice
 * and the time of one colour phase in ms (rows_per_thread = 0 and the block
 * size when the sweep of that width runs on tensor cores; 0, 0, 0 for k = 0);
 * outputs may be NULL. */
hdg_status hdg_set_batched_tile(hdg_ctx *ctx, int rows_per_thread, int threads);
hdg_status hdg_tune_batched(hdg_ctx *ctx, int nrhs, int *rows_per_thread, int *threads, double *ms,
                            hdg_stream_t stream);

/* hdg_solve for nrhs loads F[r] at once; u, p are initial guesses in and
 * solutions out; info: host array [nrhs] or NULL.  Returns
 * HDG_ERR_NOT_CONVERGED when some column reaches max_uzawa or max_it. */
hdg_status hdg_solve_multi(hdg_ctx *ctx, int nrhs, const double *F, double *u, double *p,
                           const hdg_solve_opts *opts, hdg_solve_info *info, hdg_stream_t stream);

/* One load on each of n independent contexts (several meshes, for instance of
 * different sizes) solved concurrently: one host thread and one private
 * non-blocking CUDA stream per context, so that the kernels of the meshes
 * overlap on the GPU.  ctxs[i]: distinct condensed contexts on one device;
 * F[i], u[i], p[i]: as for hdg_solve on ctxs[i]; opts: shared, NULL =
 * defaults; info, status: host arrays [n] or NULL.  Synchronises before
 * returning; returns the first non-OK per-context status. */
hdg_status hdg_solve_batched(hdg_ctx *const *ctxs, int n, const double *const *F, double *const *u,
                             double *const *p, const hdg_solve_opts *opts, hdg_solve_info *info,
                             hdg_status *status);

/* Steady Navier-Stokes by Picard iteration (Section 4.2, Algorithm 3 part (i)):
 * u^(0) solves the generalized Stokes problem with the data of params (its conv
 * is ignored); step n condenses and solves the Oseen problem of eq. nsWeak
 * whose convecting field is u_h^(n-1) (its values at the degree-(k+1) lattice,
 * recovered on the device), warm-started from the previous step, until
 * ||u_h^(n) - u_h^(n-1)||_{L2} < tol or max_steps steps.
 *   forcing: device lattice layout; u: device out [n_dof]; p: device out [n_cells];
 *   opts: inner solves (NULL = defaults); steps_out, dist_out: host out or NULL.
 * On return the context holds the condensed operator of the last Oseen step.
 * Returns HDG_ERR_NOT_CONVERGED when max_steps or an inner limit is reached. */
hdg_status hdg_picard(hdg_ctx *ctx, const hdg_params *params, const double *forcing, double tol, int max_steps,
                      double *u, double *p, const hdg_solve_opts *opts, int *steps_out, double *dist_out,
                      hdg_stream_t stream);

/* Newton iteration for steady Navier-Stokes (Section 4.2, Algorithm 3 part (ii)),
 * starting from the iterate (u, p) that the context's current operator produced
 * (for instance after hdg_picard): each step condenses with newton_u = u_old and
 * conv = u_old at the lattice, solves warm-started, and stops when
 * ||u_h^(n) - u_h^(n-1)||_{L2} < tol or after max_steps.  u, p: device in/out.
 * params: the data (its conv and newton_u are replaced).  Other arguments as
 * hdg_picard.  hdg_adjoint is not available for a Newton-step operator. */
hdg_status hdg_newton(hdg_ctx *ctx, const hdg_params *params, const double *forcing, double tol, int max_steps,
                      double *u, double *p, const hdg_solve_opts *opts, int *steps_out, double *dist_out,
                      hdg_stream_t stream);

/* The finest level's boundary facets in facet order (lexicographic in the
 * sorted global vertex pair), the order of hdg_params.dirichlet: pairs (host,
 * [n_boundary_facets][2]) receives each facet's sorted global vertex ids; on
 * tetrahedra [n_boundary_facets][3], the sorted vertex triples of the faces. */
hdg_status hdg_boundary_facets(const hdg_ctx *ctx, int32_t *pairs);

/* Sizes after hdg_setup_mesh_hierarchy (k-dependent fields after hdg_condense). */
hdg_status hdg_get_sizes(const hdg_ctx *ctx, hdg_sizes *out);

/* Copy the condensed element matrices (with the AL term) to out (device):
 * level = -1: order-k finest operator [n_cells][n_loc][n_loc];
 * level = l >= 0: lowest-order operator of level l [n_cells_l][6][6]. */
hdg_status hdg_get_element_matrices(hdg_ctx *ctx, int level, double *out, hdg_stream_t stream);

/* Step-level entry points of the hot path (parity testing and composition).
 * All vectors FP64 device; lowest-order vectors have 2 unknowns per interior
 * facet of their level.  level = -1 selects the order-k operator on the
 * finest mesh, level >= 0 the lowest-order operator of that level.        */

/* y = A x on a level (level = -1: same as hdg_apply). */
hdg_status hdg_level_apply(hdg_ctx *ctx, int level, const double *x, double *y, hdg_stream_t stream);

/* n_sweeps block Gauss-Seidel sweeps on u for A u = g over the vertex
 * patches, colours in increasing order (reverse = 0) or decreasing order
 * (reverse = 1, the transpose R^T).  u updated in place.  The 2D order-k
 * sweeps (FP64 and FP32) and the FP64 sweeps of every 3D level take each patch
 * step in the closed form u_P = A_PP^-1 (g_P - A_PE u_E), E the star cells'
 * facets outside the patch, equal to u_P + A_PP^-1 (g - A u)_P up to rounding;
 * the 2D FP32 sweeps split the augmented-Lagrangian term off that coupling, so
 * their rounding does not grow with gamma.  The other sweeps (2D lowest order,
 * 3D FP32, the 16-bit precisions) keep the correction form. */
hdg_status hdg_smooth(hdg_ctx *ctx, int level, const double *g, double *u, int n_sweeps,
                      int reverse, hdg_stream_t stream);

/* uf += I_{l-1}^l uc (harmonic-extension-corrected averaging, level l >= 1). */
hdg_status hdg_prolong_add(hdg_ctx *ctx, int level, const double *uc, double *uf, hdg_stream_t stream);

/* rc = (I_{l-1}^l)^T rf (level l >= 1). */
hdg_status hdg_restrict(hdg_ctx *ctx, int level, const double *rf, double *rc, hdg_stream_t stream);

/* u = (A^eps_{0,0})^{-1} g on the coarsest level. */
hdg_status hdg_coarse_solve(hdg_ctx *ctx, const double *g, double *u, hdg_stream_t stream);

/* u = MG_h(L, g, 0, m_h, q) of Algorithm 1 on the lowest-order operator of
 * the finest level L. */
hdg_status hdg_mg_h(hdg_ctx *ctx, const double *g, double *u, hdg_stream_t stream);

/* Failure-detection hook.  The order-k FP32 sweep (HDG_MIXED_FP32) stages its
 * matrices in shared memory by bulk copies and waits for them on an mbarrier
 * with a time limit (default 1 s of global time).  When the limit passes, the
 * thread block skips its patch update, records the timeout in a device flag
 * and then waits, in bounded steps of at most 4 s in total, until its copies
 * have landed before it exits; hdg_solve, hdg_picard, hdg_newton, hdg_adjoint,
 * hdg_precond_apply and hdg_smooth (order-k level) read and clear the flag and
 * return HDG_ERR_TIMEOUT, and the context stays usable.  hdg_set_wait_limit
 * sets that first limit in nanoseconds for this context; 0 makes every first
 * wait expire at once, so that a test can drive the timeout path without
 * stalling the GPU.  Returns HDG_ERR_INVALID_ARG for a negative limit. */
hdg_status hdg_set_wait_limit(hdg_ctx *ctx, int64_t first_wait_ns);

/* Capacity, in coarse cells, of the fixed scratch array of hdg_restrict_noalloc. */
#define HDG_NOALLOC_MAX_COARSE_CELLS 32768

/* rc = (I_{l-1}^l)^T rf, exactly like hdg_restrict, for callers that cannot
 * allocate device memory when they call (for example code whose device memory
 * is owned by another allocator, or that must not grow its footprint after
 * set-up): the call allocates nothing and uses none of the context's work
 * buffers.  Its temporaries live in one array of HDG_NOALLOC_MAX_COARSE_CELLS
 * x 18 doubles (4.7 MB) compiled into the library, which every GPU that loads
 * the library holds until the process exits.  The paper has no counterpart.
 *   - The first call on a device (made with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *   - Levels whose coarse mesh has more than HDG_NOALLOC_MAX_COARSE_CELLS cells
 *     are rejected with HDG_ERR_INVALID_ARG.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads, other contexts) race and must be ordered
 *     by the caller.  The array keeps the last call's contents; every call
 *     overwrites what it reads, so nothing needs clearing.
 * Arguments as hdg_restrict (rf, rc device FP64, level >= 1). */
hdg_status hdg_restrict_noalloc(hdg_ctx *ctx, int level, const double *rf, double *rc, hdg_stream_t stream);

/* Host-side reference-element integrals that hdg_condense contracts with each
 * cell's Jacobian to form the local system of eq. stWeak (Section 3.2) for
 * order k, and to evaluate recovered fields: the blocks R1..R16 packed in that
 * order (R9..R16: point values for the upwind convection; layouts in the
 * library source, csrc/reference.cpp).  Returns the number of doubles; writes them to
 * out (host memory) when out is not NULL; returns -1 for k outside 0..4.
 * Needs no GPU. */
int64_t hdg_reference_tables(int k, double *out);

/* Measurement utility (no counterpart in the paper): enqueues on `stream` one
 * kernel of FP64 fused multiply-adds on the current device, blocks_per_sm
 * (1..64) blocks of 256 threads per SM, each thread running 8 independent FMA
 * chains for iters iterations, and writes one double to out (device, >= 1
 * double).  Returns the kernel's floating-point operations (2 per FMA), so a
 * caller that times the launch with CUDA events on `stream` obtains the FP64
 * arithmetic rate of the GPU; returns -1 for bad arguments or a launch error. */
int64_t hdg_fp64_fma_probe(int blocks_per_sm, int64_t iters, double *out, hdg_stream_t stream);

/* Number of CUDA kernels this library has enqueued in the calling process
 * (all contexts, all streams), for launch accounting in benchmarks. */
uint64_t hdg_kernel_launches(void);

void hdg_destroy(hdg_ctx *ctx);
const char *hdg_status_string(hdg_status s);
const char *hdg_last_error(const hdg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HDG_H */
