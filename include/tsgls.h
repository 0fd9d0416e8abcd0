/*
 * tsgls.h -- C ABI of the GB300 time-spectral Galerkin/least-squares (GLS)
 * Navier-Stokes operator and solver.
 *
 * Method: Esmaily & Jia, "A new stabilized time-spectral finite element
 * solver for fast simulation of blood flow", arXiv 2311.09465.  The
 * time-periodic incompressible Navier-Stokes equations are expanded in N
 * Fourier modes (section 2.4, eq. upgh_def), discretised with equal-order
 * linear tetrahedra and stabilised by a least-squares term weighted by the
 * mode-coupling matrix tau (eq. 3D-tau).  The discrete residual is eq. (Rmc);
 * its tangent is eq. (K_mat); the nonlinear solve is pseudo-time Newton with
 * restarted GMRES (sections 2.4-2.5).
 *
 * Data layout of every modal field (y, r, v, Hv): node-major, contiguous,
 *   field[V][4][N][2]   with field index 0..2 = velocity u1,u2,u3, 3 = pressure,
 *                       mode n = 0..N-1, last index = real, imaginary part.
 * This is the real-valued unknown vector of section 2.5.1 (8N reals per node).
 * The imaginary part of mode 0 is carried but is always zero on output and
 * ignored on input.  Element type is float (precision 32) or double (64).
 *
 * Ownership: pointers named "host" are read during the call and copied;
 * pointers to modal fields are caller-owned DEVICE memory (e.g. PyTorch CUDA
 * tensors) on the current CUDA device.  Handles (ts_mesh, ts_problem) are
 * library-owned and released only by the matching *_free call.  Streams are
 * cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Errors: every int-returning call returns 0 on success and a negative
 * TS_ERR_* code otherwise; ts_last_error() gives a message for the calling
 * thread.  Calls never abort the process and never leave a kernel waiting.
 */
#ifndef TSGLS_H
#define TSGLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TS_OK            0
#define TS_ERR_ARG      -1   /* invalid argument, size or state            */
#define TS_ERR_CUDA     -2   /* a CUDA runtime call failed                 */
#define TS_ERR_OOM      -3   /* device allocation failed                   */
#define TS_ERR_NOCONV   -4   /* solver hit its step or matvec cap          */
#define TS_ERR_NAN      -5   /* non-finite residual norm                   */
#define TS_ERR_UNSUPPORTED -6 /* mode count without a compiled kernel      */

/* boundary-condition kinds for ts_set_bc */
#define TS_BC_DIRICHLET  1   /* velocity prescribed (values carried in y)  */
#define TS_BC_TRACTION   2   /* -p n + mu du/dn = h n with h = 0           */
#define TS_BC_RESISTANCE 3   /* h_n = -R Q_n, Q_n = int u_n . n (per mode) */
#define TS_BC_BACKFLOW   4   /* backflow stabilisation with coefficient beta in [0,1] */

/* inflow profiles for ts_set_inlet */
#define TS_PROFILE_PARABOLIC 1 /* 2 U_n (1 - r^2/R^2), U_n = Q_n / (pi R^2)                   */
#define TS_PROFILE_WOMERSLEY 2 /* fully developed pulsatile pipe flow per mode (mean U_n)    */

/* tangent variants for ts_jvp / ts_solve (eq. K_mat) */
#define TS_JVP_PAPER   0   /* A, tau frozen; LS parts of G_i, D_j dropped (section 2.5.2) */
#define TS_JVP_FROZEN  1   /* A, tau frozen; all blocks of eq. (K_mat)                    */
#define TS_JVP_LIN_A   2   /* FROZEN + derivative of A_j (tau frozen): exact up to d tau   */
#define TS_JVP_EXACT   3   /* LIN_A + the derivative of tau (Daleckii-Krein, from the      */
                           /* eigenpairs of M): the exact Jacobian of eq. (Rmc); FP32     */
                           /* tangent products with N <= 7 only (TS_ERR_UNSUPPORTED else) */

/* ts_problem_option keys and values (implementation choices, not physics) */
#define TS_OPT_TAU64        1  /* how the FP64 residual computes tau (eq. 3D-tau):          */
#define TS_TAU64_REFINE     0  /*   FP32 Jacobi eigenvectors + FP64 refinement             */
#define TS_TAU64_DOUBLEFLOAT 1 /*   the same refinement in double-float (FP32 pair)         */
                               /*   arithmetic (default): meets the FP64 bar, 2.4x faster  */
                               /*   where FP64 runs at 1/64 of the FP32 rate               */
#define TS_TAU64_JACOBI     2  /*   FP64 Jacobi eigenpairs                                 */
#define TS_OPT_FP32_TANGENT 2  /* FP32 tangent products: 0 single launch with vector       */
                               /* atomics (default), 1 colour-ordered launches            */
#define TS_OPT_ELEMENT64    3  /* arithmetic of the FP64 element operator (the FP64         */
                               /* residual's element pass and FP64 tangent products):     */
#define TS_ELEMENT64_NATIVE 0  /*   FP64 instructions                                     */
#define TS_ELEMENT64_DOUBLEFLOAT 1 /* double-float pairs on the FP32 pipe (FP64 storage;  */
                                   /* default): meets the FP64 bar, 1.5x faster           */
#define TS_OPT_TAU_WARM     4  /* 0 (default): every FP64 residual with TS_TAU64_DOUBLEFLOAT */
                               /* computes tau from scratch; 1: its FP32 Jacobi sweeps     */
                               /* start from each quadrature point's eigenvectors of the   */
                               /* previous evaluation on this problem (cached, (2N-1)^2    */
                               /* floats per point, allocated on first use), so they stop  */
                               /* early when the state moved little.  The refinement makes */
                               /* tau independent of the start up to rounding (about 1e-15 */
                               /* relative), not bitwise.  Setting the key drops the cache; */
                               /* ts_solve uses 1 for its own residuals and restores the   */
                               /* caller's value on return.                                */

typedef struct ts_mesh ts_mesh;
typedef struct ts_problem ts_problem;

typedef struct {
  int    N;          /* independent Fourier modes (mean + N-1 harmonics), section 2.1 */
  double rho;        /* density                                                       */
  double mu;         /* dynamic viscosity; kappa in tau is mu/rho                     */
  double omega;      /* base angular frequency, Omega_mm = i m omega (eq. phi-def)    */
  double C_I;        /* tau constant, 3 for linear tetrahedra (section 2.2)           */
  double c1;         /* pseudo-time mass coefficient, 1.5 (section 2.5.3)             */
  double dt_pseudo;  /* pseudo-time step; <= 0 or inf means plain Newton              */
  int    jvp_variant;/* TS_JVP_*                                                      */
} ts_params;

typedef struct {
  int    precision;    /* 64: FP64 operator everywhere; 32: FP32 tangent products inside
                          FP64 GMRES with an FP64 outer residual (iterative refinement) */
  double tol;          /* stop when ||r||_2 <= tol * r_ref (default 1e-8)              */
  double r_ref;        /* reference norm; <= 0 means ||r(y_in)||_2                     */
  int    max_steps;    /* pseudo-time / Newton steps                                   */
  int    krylov;       /* GMRES restart length (100 in section 3.2)                    */
  double eps_ls;       /* GMRES relative tolerance (0.05 in section 2.4, remark 6)     */
  int    max_matvec;   /* per linear solve (10000 in section 3.2)                      */
  int    verbose;      /* print one line per step to stderr                            */
  int    precond;      /* right preconditioner of GMRES (changes the GMRES path only,
                          never the converged field): 0 none; 1 diagonal scaling by an
                          approximate diag(H) (viscous + mass + scalar-tau LS terms per
                          node); 2 nodal block Jacobi: the inverted 8N x 8N diagonal
                          blocks of the tangent at the current state (ts_block_diagonal),
                          rebuilt every pseudo-time step; 3 symmetric block Gauss-Seidel:
                          a forward and a backward sweep over a colouring of the node
                          graph with the assembled paper-variant blocks (ts_assemble)
                          off the diagonal and the inverted blocks of 2 on it          */
  double ser;          /* > 0: pseudo-time step grows as dt_k = dt_0 (|r_0|/|r_k|)^ser,
                          |r_0| = r_ref when given, else the first residual norm
                          (switched evolution relaxation; dt_0 = the problem's
                          dt_pseudo, which must be finite); 0: fixed dt (section 2.5.3) */
  double dt_max;       /* > 0: upper bound of the grown pseudo-time step (keeps the mass
                          term in the tangent, so GMRES stays effective); 0: no bound */
  double reject;       /* > 1 (ts_solve only, finite dt_pseudo): a step whose residual
                          norm exceeds reject x the last accepted norm is undone and
                          retried from the same state with a quarter of the pseudo-time
                          step (at most 8 times in a row; the factor recovers x2 per
                          accepted step); a step whose GMRES solve stalled above half
                          its initial residual makes the next step 8x smaller.
                          Changes the path only, never the converged field.
                          <= 1: every step is accepted.  Not in the paper.           */
} ts_solve_opts;

typedef struct {
  int    steps;         /* pseudo-time steps taken                              */
  int    matvecs;       /* total tangent products                               */
  double r_ref;         /* reference norm used                                  */
  double r_final;       /* final ||r||_2 / r_ref                                */
  double seconds;       /* wall time of the solve                               */
  double t_residual;    /* seconds in residual evaluations (incl. tau)          */
  double t_jvp;         /* seconds in tangent products                          */
  double t_krylov;      /* seconds in Gram-Schmidt, norms and updates           */
  int    hist_len;      /* entries written to hist                              */
  double hist[512];     /* ||r||/r_ref after each step (rejected ones included) */
  int    rejected;      /* steps undone by the reject test                      */
  double t_precond;     /* seconds building the preconditioner (precond 1, 2, 3) */
  double t_tau;         /* seconds in the tau launches of the residuals (CUDA   */
                        /* events around each launch on the solve's stream)     */
  int    n_residual;    /* residual evaluations (each one tau launch)           */
} ts_solve_report;

/* Copies a tetrahedral mesh to the device and precomputes per-element shape
 * function gradients, volume and the metric G_ij = dxi_k/dx_i dxi_k/dx_j
 * (eq. metric; unit reference tetrahedron), and an element colouring (no two
 * elements of one colour share a node) used for the scatter-add.
 *   xyz_host   [n_nodes][3] coordinates
 *   tets_host  [n_tets][4]  node ids, any orientation, 0-based
 *   bfaces_host[n_bfaces][3] boundary triangles (outward or not: the library
 *                            orients them with the owning tetrahedron)
 *   btag_host  [n_bfaces]   integer tag per boundary triangle
 * Fails with TS_ERR_ARG on out-of-range ids or a degenerate tetrahedron. */
int  ts_mesh_load(const double* xyz_host, int64_t n_nodes, const int32_t* tets_host,
                  int64_t n_tets, const int32_t* bfaces_host, const int32_t* btag_host,
                  int64_t n_bfaces, ts_mesh** out);
void ts_mesh_free(ts_mesh* mesh);
/* number of element colours of a loaded mesh (or negative error) */
int  ts_mesh_colors(const ts_mesh* mesh);
/* Colouring of the node graph of a loaded mesh: two nodes of one colour never
 * share an element.  Returns the number of colours (or a negative error) and,
 * when colour_host (host, n_nodes int32) is not NULL, writes each node's
 * colour there.  The block Gauss-Seidel preconditioner (ts_precond_apply kind
 * 3) sweeps the colours in this numbering. */
int  ts_mesh_node_colours(const ts_mesh* mesh, int32_t* colour_host);

/* Creates a problem (physics + boundary conditions) on a mesh.  The mesh must
 * outlive the problem.  TS_ERR_UNSUPPORTED if no kernel is compiled for N. */
int  ts_problem_create(const ts_mesh* mesh, const ts_params* params, ts_problem** out);
void ts_problem_free(ts_problem* prob);
/* Changes pseudo-time step and tangent variant of an existing problem. */
int  ts_problem_set(ts_problem* prob, double dt_pseudo, int jvp_variant);
/* Sets an implementation option (TS_OPT_*); TS_ERR_ARG for an unknown key or
 * value.  Takes effect at the next residual evaluation. */
int  ts_problem_option(ts_problem* prob, int key, int value);

/* Assigns a boundary condition to all boundary triangles with this tag.
 * TS_BC_DIRICHLET: nodes of those triangles become Dirichlet velocity nodes;
 *   their momentum rows are excluded and their values are taken from y
 *   (section 2.4 keeps Dirichlet data inside the unknown vector and holds it
 *   fixed during the iterations).  Dirichlet wins over any other tag at
 *   shared nodes.
 * TS_BC_TRACTION: zero traction, nothing to add (the default).
 * TS_BC_BACKFLOW: adds the backflow stabilisation of section 2.6 on these
 *   Neumann faces, beta = value in [0, 1]: the residual gains
 *   -int N_A (rho/2) beta |A_n|_- u_i with |A_n|_- = (A_n - |A_n|)/2,
 *   A_n = A(u . n), taken by eigenpairs at the 3 points of every face; it is
 *   zero where A_n is positive semi-definite (no backflow).  The tangent
 *   products use |A_n|_- frozen at the last residual (like tau).  Not
 *   available in ts_residual_noalloc.
 * TS_BC_RESISTANCE: outlet with h_n = -value * Q_n; the residual gains
 *   value * Q_n * int N_A n_i on that outlet (a rank-one coupling per mode). */
int  ts_set_bc(ts_problem* prob, int tag, int kind, double value);

/* Inflow boundary data (section 2.4: the Dirichlet data g are expanded in the
 * same Fourier modes as the unknowns, eq. upgh_def, g_n = (1/T) int g e^{-i n w t};
 * section 3.1 prescribes a parabolic inlet profile scaled by the flow waveform).
 * The boundary triangles with this tag form a circular inlet.  Its geometry
 * is the caller's (geometry_host: centre xyz, inflow direction xyz pointing
 * into the domain, radius R; copied) or, with geometry_host NULL, derived
 * from the triangles: the inflow direction from their area-weighted normal,
 * the centre from their area-weighted centroid, and R as the largest
 * distance from the axis of a rim node (a node of the tag that also lies on
 * triangles of other tags; right when the rim lies on the circle, as on a
 * pipe meshed to its wall).  For each mode n = 0..N-1 the velocity at an
 * inlet node at distance r from the axis is w_n(min(r, R)) times the inflow
 * direction, with w_n the profile of mean velocity U_n = Q_n / (pi R^2):
 *   TS_PROFILE_PARABOLIC  w_n = 2 U_n (1 - r^2/R^2)
 *   TS_PROFILE_WOMERSLEY  w_0 parabolic; w_n = U_n [1 - J0(L r/R)/J0(L)] /
 *                         [1 - 2 J1(L)/(L J0(L))], L = i^{3/2} alpha_n,
 *                         alpha_n = R sqrt(n omega rho/mu) (Womersley 1955; J0, J1
 *                         from their power series, adequate for alpha_n <= 15)
 * Rim nodes keep zero velocity (they belong to the wall).  All nodes of the
 * tag become Dirichlet velocity nodes (as ts_set_bc with TS_BC_DIRICHLET).
 *   Qn_host  [N][2] flow-rate coefficients (re, im) of modes 0..N-1, copied;
 *            Im(Q_0) is ignored (the mean flow is real, section 3.3)
 * A second call for the same tag replaces the first.  TS_ERR_ARG for an
 * unknown profile, a tag without triangles, a rim of fewer than 3 nodes, or
 * a zero direction or radius. */
int  ts_set_inlet(ts_problem* prob, int tag, const double* Qn_host, int profile,
                  const double* geometry_host);
/* Geometry ts_set_inlet derived for a tag: out_host[0..2] centre, [3..5] unit
 * inflow direction, [6] radius.  TS_ERR_ARG if the tag has no inlet data. */
int  ts_inlet_info(const ts_problem* prob, int tag, double* out_host);
/* The paper's initial guess (section 2.4): zero velocity and pressure
 * everywhere except the inlet Dirichlet data of every ts_set_inlet tag.
 * y: caller-owned device field, precision 32 (float) or 64 (double). */
int  ts_initial_guess(ts_problem* prob, void* y, int precision, void* stream);

/* Discrete residual r(y) of eq. (Rmc), section 2.4, for the caller's state y
 * (device, layout above, precision 32 or 64).  Momentum rows of Dirichlet
 * nodes and Im(mode 0) are zero.  Also freezes the linearisation used by
 * ts_jvp: the convolution matrices A_j of y, tau at every quadrature point
 * (eq. 3D-tau, computed by a Jacobi eigensolver), and tau L_i(y).
 * y and r may not alias. */
int  ts_residual(ts_problem* prob, const void* y, void* r, int precision, void* stream);

/* Allocation-free FP32 residual.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they call
 * in, e.g. a solver loop running under a memory pool or allocator policy that
 * forbids new device allocations after set-up, or a host that has handed all
 * free device memory to another runtime.  It computes the same r(y) as
 * ts_residual(..., 32, ...) but keeps its intermediate data (tau per
 * quadrature point and tau L) in one fixed 32 MiB device array compiled into
 * this library, and reads its DFT tables from a second, 19 KB one.
 * ts_problem_create sets these up on the current device (it resolves both
 * arrays, which loads them also under CUDA's lazy module loading, writes the
 * tables once per device and loads the two kernels this call launches), so a
 * call only launches kernels and clears r; every GPU on which a problem was
 * created holds the arrays until the process exits.  y and r are caller-owned
 * FP32 device fields; r is overwritten.  Limits: (E*4*ntau rounded up to a
 * multiple of 64) + E*12*2N floats must fit in 32 MiB (ntau = (2N-1)N rounded
 * up to a multiple of 4): about 15k tetrahedra at N = 7, 61k at N = 3; larger
 * meshes return TS_ERR_ARG with the sizes in the message.  It does not refresh
 * the linearisation state used by ts_jvp, and problems with backflow faces
 * return TS_ERR_ARG.  Every call reuses the same array, so calls whose GPU
 * work overlaps (other streams, other host threads on the same device) race
 * on it and must be serialised by the caller.  Nothing in the array needs
 * clearing between calls: each call writes every part it reads.  Calls no
 * cudaMalloc or cudaFree. */
int  ts_residual_noalloc(ts_problem* prob, const float* y, float* r, void* stream);

/* Assembled tangent of the paper's variant (section 2.5.2, eq. tangent and
 * eq. K_mat with A and tau frozen at the state of the last ts_residual call,
 * least-squares parts dropped from G_i and D_j, plus the pseudo-time mass of
 * section 2.5.3 when dt_pseudo is finite), stored block by block as the paper
 * describes: per connection of the node graph (nodes sharing an element, a
 * node with itself included) the mode matrix K_AB, used for all three velocity
 * fields, the mode matrix L_AB, and the six scalars of the mode-diagonal
 * G_AB,i and D_AB,j: 2 (2N)^2 + 8 FP32 numbers, ts_assembled_bytes() in all.
 * The blocks are those of TS_JVP_PAPER whatever the problem's variant.
 * ts_assemble builds them on the device (library-owned memory, allocated at
 * the first call); TS_ERR_ARG if no residual was computed yet,
 * TS_ERR_UNSUPPORTED for a problem with backflow faces.  A later ts_residual
 * invalidates them. */
int  ts_assemble(ts_problem* prob, void* stream);
/* Hv = H v with the assembled blocks, plus the resistance-outlet coupling
 * (evaluated matrix-free, as in ts_jvp); FP32 fields in the layout above,
 * caller-owned device memory.  Dirichlet velocity entries and Im(mode 0) of
 * v are ignored and the same rows of Hv are zero.  Equals ts_jvp of a
 * TS_JVP_PAPER problem at the same state.  TS_ERR_ARG before ts_assemble or
 * when v and Hv alias. */
int  ts_spmv(ts_problem* prob, const float* v, float* Hv, void* stream);
/* bytes of the assembled blocks (or a negative error) */
int64_t ts_assembled_bytes(const ts_problem* prob);
/* connections of the node graph of a mesh (or a negative error) */
int64_t ts_mesh_connections(const ts_mesh* mesh);

/* Nodal diagonal blocks H_AA of the tangent (eq. tangent, eq. K_mat, with A and
 * tau frozen at the state of the last ts_residual call, plus the pseudo-time
 * mass of section 2.5.3 when dt_pseudo is finite and the resistance-outlet
 * coupling of the node with itself): for every node A the 8N x 8N matrix that
 * maps the node's own unknowns (field, mode, re/im in the layout above) to its
 * own rows, summed over the elements around A.  K is shared by the three
 * velocity fields; TS_JVP_PAPER drops the least-squares parts of G_i and D_j
 * (section 2.5.2); a TS_JVP_LIN_A problem gets the blocks of TS_JVP_FROZEN
 * (the derivative of A_j is left out).  These blocks are the preconditioner of
 * ts_solve with precond = 2.
 *   blocks  caller-owned FP32 device array [V][8N][8N]
 *   invert  0: H_AA row-major (row = field * 2N + 2 mode + re/im), with the
 *           rows and columns of fixed unknowns (Im(mode 0), Dirichlet
 *           velocity) zero; 1: the inverse of H_AA with those rows and columns
 *           replaced by the identity, stored COLUMN-major (the layout the
 *           preconditioner reads).  Computed in FP32.
 * TS_ERR_ARG if no residual was computed yet.  A block that cannot be inverted
 * is stored as the identity. */
int  ts_block_diagonal(ts_problem* prob, float* blocks, int invert, void* stream);

/* The block preconditioners of ts_solve on their own (precond 2 and 3 of
 * ts_solve_opts), for use in another solver or to time them.
 * ts_precond_setup builds, at the state of the last ts_residual call,
 *   kind 2, nodal block Jacobi: B_A^{-1}, the inverted diagonal blocks of
 *           ts_block_diagonal (fixed unknowns: identity rows and columns);
 *   kind 3, symmetric block Gauss-Seidel: the same inverted blocks on the
 *           diagonal and the assembled paper-variant blocks H_AB of ts_assemble
 *           (section 2.5.2) off it (the resistance outlets' coupling between
 *           different nodes is left out; a node's own coupling is in B_A).
 * ts_precond_apply computes z = P^{-1} x (x, z: device, double, the field
 * layout, distinct):
 *   kind 2: z_A = B_A^{-1} x_A for every node A;
 *   kind 3: from z = 0, a forward sweep over the node colours of
 *           ts_mesh_node_colours in increasing order, then a backward sweep in
 *           decreasing order, each updating every node A of a colour (no two
 *           of which are coupled) as z_A = B_A^{-1} (x_A - sum_{B != A} H_AB z_B)
 *           with the z of the colours already visited; Dirichlet velocity
 *           entries and Im(mode 0) of x are ignored and the same entries of z
 *           are zero.  Computed in FP32 (x rounded), returned in FP64.
 * TS_ERR_ARG: no residual yet, kind not 2 or 3, apply before the setup of that
 * kind at the current state (a new ts_residual invalidates both), x == z.
 * TS_ERR_UNSUPPORTED (kind 3) with backflow faces. */
int  ts_precond_setup(ts_problem* prob, int kind, void* stream);
int  ts_precond_apply(ts_problem* prob, int kind, const double* x, double* z, void* stream);

/* Tangent product Hv (eq. K_mat, variant from the problem) at the state of
 * the last ts_residual call, plus c1 rho / dt_pseudo M v on the momentum rows
 * (section 2.5.3) when dt_pseudo is finite.  Dirichlet velocity entries and
 * Im(mode 0) of v are ignored; the same rows of Hv are zero.  If the last
 * residual was computed in the other precision its state is converted.
 * TS_ERR_ARG if no residual was computed yet.  v and Hv may not alias. */
int  ts_jvp(ts_problem* prob, const void* v, void* Hv, int precision, void* stream);

/* Pseudo-time Newton-GMRES solve (sections 2.4-2.5) in place on y_inout
 * (device, double, layout above, Dirichlet values already set).  Each step:
 * r = r(y); stop if ||r|| <= tol r_ref; solve (H + c1 rho/dt M) d = -r with
 * restarted GMRES (FP64 Gram-Schmidt and Hessenberg); y += d on free
 * unknowns.  Runs on the given stream; synchronises with the host once per
 * GMRES iteration.  Returns TS_ERR_NOCONV when max_steps is reached (y holds
 * the last iterate, report filled), TS_ERR_NAN on a non-finite norm. */
int  ts_solve(ts_problem* prob, void* y_inout, const ts_solve_opts* opts,
              ts_solve_report* report, void* stream);

/* ---------------------------------------------------------------------------
 * Batched lockstep solve of many instances (no counterpart in the paper,
 * which solves one problem at a time, section 2.5).  Instances may live on
 * different meshes and use different N <= 7; each keeps its own boundary
 * conditions, physics and pseudo-time schedule.  Every GMRES iteration
 * applies the FP32 LIN_A tangent (eq. K_mat) of all instances in one fused
 * launch and runs FP64 classical Gram-Schmidt as segmented reductions; the
 * device work of an iteration is one CUDA graph per Krylov index.  The
 * problems must outlive the batch; the batch works on its own stream and
 * orders itself after / before the caller's stream.
 * ------------------------------------------------------------------------- */
typedef struct ts_batch ts_batch;
/* TS_ERR_UNSUPPORTED if an instance has N > 7 (no single-launch kernel). */
int  ts_batch_create(ts_problem* const* probs, int n, ts_batch** out);
void ts_batch_free(ts_batch* batch);
/* hv[b] = H_b v[b] (FP32, LIN_A, eq. K_mat + pseudo-time mass) for every
 * instance, one fused launch plus the boundary terms; each instance needs a
 * residual evaluation first (its linearisation state). */
int  ts_batch_jvp(ts_batch* batch, const float* const* v, float* const* hv, void* stream);
/* Mixed-precision pseudo-time Newton-GMRES (as ts_solve, precision 32) on
 * every instance in lockstep; y[b] is instance b's FP64 field, reports[b]
 * its report (seconds and times are of the whole batch).  TS_ERR_NOCONV if
 * any instance hit the step cap (its report says which). */
int  ts_batch_solve(ts_batch* batch, double* const* y, const ts_solve_opts* opts,
                    ts_solve_report* reports, void* stream);
/* launch shape chosen by the autotuner (1 once tuned, else 0) */
int  ts_batch_launch_shape(const ts_batch* batch, int* warps_per_block, int* blocks);

/* ---------------------------------------------------------------------------
 * Learned initial guess (no counterpart in the paper, whose Newton iteration
 * starts from zero interior velocity with the Dirichlet data in place,
 * section 2.4): y0 = ybar + Phi diag(sigma) f(x), with Phi a POD basis of
 * solution snapshots and f a fully connected network
 *   n_in -> hidden (tanh) x n_hidden_layers -> n_out (linear)
 * from inflow coefficients, Re and Wo to the POD coefficients divided by
 * their singular values.  Solves started from it iterate to the same
 * tolerance as from the plain guess.  All buffers are row-major FP32 unless
 * stated; X [B][n_in], targets and outputs [B][n_out]; parameters are one
 * flat vector: for each layer W [n_out][n_in] then b [n_out].  Device
 * pointers unless named *_host.  TS_ERR_ARG on sizes that do not match.
 * ------------------------------------------------------------------------- */
typedef struct ts_surrogate ts_surrogate;
/* n_dof = length of one modal field (V * 8N).  Weights ~ U(+-1/sqrt(n_in))
 * from seed, biases zero. */
int  ts_surrogate_create(int n_in, int hidden, int n_hidden_layers, int n_out, int64_t n_dof,
                         uint64_t seed, ts_surrogate** out);
void ts_surrogate_free(ts_surrogate* sur);
int64_t ts_surrogate_num_params(const ts_surrogate* sur);
int  ts_surrogate_get_params(const ts_surrogate* sur, float* params_host, int64_t n);
/* also resets the Adam state */
int  ts_surrogate_set_params(ts_surrogate* sur, const float* params_host, int64_t n);
/* out = f(X) for a batch of B inputs */
int  ts_surrogate_forward(ts_surrogate* sur, const float* X, int B, float* out, void* stream);
/* gradient of (1/2B) sum_b ||f(x_b) - t_b||^2 into grad (flat, may be NULL),
 * the loss into *loss (may be NULL) */
int  ts_surrogate_gradient(ts_surrogate* sur, const float* X, const float* T, int B, float* grad,
                           double* loss, void* stream);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with this gradient */
int  ts_surrogate_adam(ts_surrogate* sur, const float* grad, double lr, void* stream);
/* POD of S snapshots Y [S][n_dof] (FP64): mean, basis of rank <= n_out
 * (eigenvalues below 1e-10 of the largest are dropped) */
int  ts_surrogate_fit_basis(ts_surrogate* sur, const double* Y, int S, void* stream);
/* fitted rank; singular values into sigma_host (may be NULL, else n_out long) */
int  ts_surrogate_basis_rank(const ts_surrogate* sur, double* sigma_host);
/* A [S][n_out] = Phi^T (y_s - ybar) / sigma (zero beyond the rank) */
int  ts_surrogate_coefficients(ts_surrogate* sur, const double* Y, int S, float* A, void* stream);
/* epochs of shuffled mini-batches (size batch, remainder dropped) of Adam on
 * the POD coefficients of Y; mean batch loss per epoch into loss_hist */
int  ts_surrogate_train(ts_surrogate* sur, const float* X_host, const double* Y, int S, int epochs,
                        int batch, double lr, uint64_t seed, double* loss_hist, void* stream);
/* y_inout (FP64 field of prob) <- ybar + Phi diag(sigma) f(x) on the free
 * entries; Dirichlet velocity values and Im(mode 0) keep their input */
int  ts_surrogate_guess(ts_surrogate* sur, ts_problem* prob, const float* x_host, double* y_inout,
                        void* stream);

/* ---------------------------------------------------------------------------
 * Time-spectral GLS convection-diffusion of a scalar (a passive tracer),
 * eq. (3D-weak) with eq. (3D-weak-def), section 2.2: for a given advecting
 * velocity a (modes at the nodes) and diffusivity kappa the residual
 *   r_A = int N_A (Omega phi + A_i dphi/dx_i) + kappa dN_A/dx_i dphi/dx_i
 *       + int (-Omega N_A + A_i dN_A/dx_i) tau (Omega phi + A_i dphi/dx_i)
 * with A_i = A(a_i) (eq. phi-def) and tau of eq. (3D-tau) with kappa, at every
 * quadrature point.  It is linear in phi (its own tangent).  Rows of
 * Dirichlet nodes and Im(mode 0) are zero; zero Neumann data elsewhere.
 * ------------------------------------------------------------------------- */
typedef struct ts_tracer ts_tracer;
/* TS_ERR_UNSUPPORTED if no kernel is compiled for N.  The mesh must outlive it. */
int  ts_tracer_create(const ts_mesh* mesh, int N, double kappa, double omega, double C_I,
                      ts_tracer** out);
void ts_tracer_free(ts_tracer* tracer);
/* nodes of the boundary triangles with this tag carry Dirichlet data (no equation) */
int  ts_tracer_set_dirichlet(ts_tracer* tracer, int tag);
/* r(phi) for the advecting velocity a: caller-owned device arrays of the
 * given precision, a [V][3][N][2] (the velocity part of a modal field), phi and
 * r [V][N][2] (one field of the modal layout).  Computes tau at every point
 * (FP64: the double-float refinement; FP32: FP32 Jacobi) into library-owned
 * buffers allocated at the first call.  r may not alias a or phi. */
int  ts_tracer_residual(ts_tracer* tracer, const void* a, const void* phi, void* r, int precision,
                        void* stream);

/* 1 (default): the GLS residual above; 0: its Galerkin terms only (tau = 0),
 * the unstabilised method the paper compares against (section 3.3). */
int  ts_tracer_set_stabilised(ts_tracer* tracer, int gls);
/* Solves r(phi) = 0 for phi_inout (FP64 device [V][N][2]; the Dirichlet values
 * already in place, the other entries the start) on the advecting velocity a
 * (FP64 device [V][3][N][2]): restarted GMRES(krylov <= 128) with two-pass
 * classical Gram-Schmidt in FP64 on the linear operator, to ||r|| <= tol
 * ||r(phi_in)||.  *matvecs_out, *rel_out: operator applications and final
 * relative residual.  TS_ERR_NOCONV at max_matvec. */
int  ts_tracer_solve(ts_tracer* tracer, const double* a, double* phi_inout, double tol, int krylov,
                     int max_matvec, int* matvecs_out, double* rel_out, void* stream);

/* Thread-local message describing the last error. */
const char* ts_last_error(void);

/* Library version string. */
const char* ts_version(void);

/* Number of kernels this library has launched in this process (all devices,
 * all streams); a diagnostic for counting launches inside a timed region. */
int64_t ts_launch_count(void);

/* Device time in milliseconds, from CUDA events on the call's stream, of
 * out[0] the tau kernel (eq. 3D-tau) of the problem's last ts_residual,
 * out[1] that residual's element pass (eq. Rmc, with the outlet terms) and
 * out[2] the element kernel of its last single-launch FP32 tangent product
 * (eq. K_mat; node pre-pass and boundary terms excluded); -1 where no such
 * call has run.  Waits for those events.  A measurement aid with no
 * counterpart in the paper.  out: caller-owned host array of 3 doubles.
 * Returns 0, TS_ERR_ARG or TS_ERR_CUDA. */
int ts_stage_times(ts_problem* pr, double* out);

#ifdef __cplusplus
}
#endif
#endif /* TSGLS_H */
