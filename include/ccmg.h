/* ccmg.h -- C ABI of the GB300 cell-centred multigrid electrostatics library (libccmg.so).
 *
 * Solves the finite-volume Poisson problem of Bartuschat & Ruede (arXiv 1410.6609),
 *     -lap(phi) = rho / eps            (Sec. 2.4, Eq. Poisson)
 * on a uniform grid of nx*ny*nz cubic cells of size h, with Dirichlet or Neumann conditions on
 * each of the six walls folded into stencil and right-hand side (Sec. 2.4, "Boundary
 * conditions"), by the cell-centred geometric multigrid of Sec. 3 / Sec. 5.3 (red-black
 * Gauss-Seidel, averaging restriction, constant prolongation with a x2 magnified correction,
 * Galerkin coarse operators, CG on the coarsest grid), iterated until the L2 norm of the
 * residual drops below a tolerance (Algorithm 1). It then evaluates the E-field by central
 * differences and the Coulomb force on charged spheres (Eq. ElectrostatForce) with subsampled
 * volume overlap (Sec. 2.4, "Subsampling").
 *
 * Conventions shared by every entry point
 *   - Fields are dense arrays of nx*ny*nz doubles, x fastest: index i + nx*(j + ny*k); cell
 *     (i,j,k) has its centre at ((i+1/2)h, (j+1/2)h, (k+1/2)h).
 *   - Faces are numbered 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z. A Dirichlet value is the potential on
 *     the face; a Neumann value is the outward normal derivative of phi on the face.
 *   - Pointers named d_* are DEVICE memory, h_* are HOST memory. All are borrowed for the
 *     duration of the call only; the context copies what it keeps.
 *   - Work is enqueued on the stream given to mg_create (NULL = the legacy default stream) in
 *     call order. Only calls that return host scalars (mg_solve, mg_residual, the *_host
 *     calls) synchronise with that stream.
 *   - Every call returns a status; none aborts. mg_last_error() gives a message for the last
 *     failing call on a context. A NULL context gives MG_ERR_INVALID.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef CCMG_H
#define CCMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,       /* bad argument or state */
  MG_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  MG_ERR_OOM = 3,           /* device allocation failed */
  MG_ERR_NOT_CONVERGED = 4, /* max_cycles reached, or NaN/Inf residual */
  MG_ERR_DIVERGED = 5,      /* residual grew by more than 1e3 over its starting value */
  MG_ERR_TIMEOUT = 6        /* a bounded device-side wait ran out */
} mg_status;

/* Wall conditions (Sec. 2.4): Dirichlet (value = the potential on the face), Neumann (value =
 * the outward normal derivative), periodic (both faces of an axis; the domain is extended
 * cyclically and the neighbour across the face is the cell at the opposite side; the value is
 * unused). */
typedef enum { MG_BC_DIRICHLET = 0, MG_BC_NEUMANN = 1, MG_BC_PERIODIC = 2 } mg_bc;

/* MG_FP64: every operation in double precision.
 * MG_MIXED: FP64 defect correction around single-precision V-cycles. The outer residual, the
 *   solution update and the coarsest-grid CG are double; smoothing, restriction and
 *   prolongation are float. (Not in the paper; the cycle itself is the paper's.) */
typedef enum { MG_FP64 = 0, MG_MIXED = 1 } mg_prec;

typedef struct {
  int nx, ny, nz;        /* cells per axis; each >= 4 and even */
  double h;              /* cell size (> 0) */
  int bc_type[6];        /* mg_bc per face; periodic in opposite pairs; at least one Dirichlet
                            face (otherwise singular) */
  double bc_value[6];    /* Dirichlet potential / Neumann outward derivative per face */
  int nu1, nu2;          /* pre- and post-smoothing sweeps (V(nu1,nu2)); 0..16, nu2 >= 1 */
  double cgc_weight;     /* magnification of the coarse-grid correction (Sec. 3: about 2) */
  int prec;              /* mg_prec */
  double eps;            /* permittivity (> 0) */
  int mixed_inner;       /* MG_MIXED: single-precision V-cycles per outer defect-correction step, 1..16 */
} mg_params;

/* Fills p with the defaults: V(2,2), cgc_weight 2, MG_FP64, eps 1, all walls Dirichlet 0,
 * mixed_inner 4. */
void mg_default_params(mg_params* p, int nx, int ny, int nz, double h);

/* Create a solver context: validates p, builds the level hierarchy (halve every dimension
 * while all are even and their halves are >= 3, Sec. 3), allocates every level on the current
 * device and captures nothing yet. The coarsest grid must have at most 4096 cells.
 * stream is a cudaStream_t (NULL = legacy default stream). */
mg_status mg_create(const mg_params* p, void* stream, mg_ctx** out);
mg_status mg_destroy(mg_ctx* ctx);
const char* mg_last_error(const mg_ctx* ctx);

/* Hierarchy introspection: number of levels and the dimensions of level l (0 = finest). */
int mg_num_levels(const mg_ctx* ctx);
mg_status mg_level_dims(const mg_ctx* ctx, int level, int* h_dims3);

/* Replace the six wall values (host array of 6 doubles). Takes effect at the next
 * mg_set_rhs, mg_efield, mg_force_gather and mg_force_gather_adjoint call. */
mg_status mg_set_bc_values(mg_ctx* ctx, const double* h_bc_value6);

/* Wall values per face cell for face `face` (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z), as the validation
 * runs of Sec. 6.3 set the boundary to the analytic potential: d_values (device) holds one
 * double per boundary cell of the face, faces 0 and 1 ny*nz values indexed j + ny*k, faces 2 and
 * 3 nx*nz indexed i + nx*k, faces 4 and 5 nx*ny indexed i + nx*j; each is the Dirichlet value or
 * the outward normal derivative (Neumann) of that cell's face, entering the right-hand side
 * (2 g / h^2 or g / h, Sec. 2.4) and the ghost values of mg_efield, mg_force_gather and their
 * adjoint. The array is copied (the call returns after the copy); NULL returns the face to its
 * uniform value. Takes effect like mg_set_bc_values. Errors: MG_ERR_INVALID for a bad face or a
 * periodic one, MG_ERR_OOM / MG_ERR_CUDA if the copy cannot be made. Batched solves have no
 * per-cell values. */
mg_status mg_set_bc_field(mg_ctx* ctx, int face, const double* d_values);

/* Variable permittivity (Sec. 3: the solver extends to discontinuous dielectricity by Galerkin
 * coarsening with the averaging restriction and the nearest-neighbour prolongation). d_eps
 * (device, nx*ny*nz doubles, natural order, positive and finite; not checked) gives the cell
 * permittivities; the equation becomes -div(eps grad phi) = rho, the flux between two cells
 * weighted by the harmonic mean of their permittivities and a wall face by its cell's (Dirichlet
 * ghost 2 g - phi, Neumann phi + h g, as in the constant case), and every coarse level carries the
 * Galerkin operator R A P of the finer one. The array is copied and the level coefficients are
 * built before the call returns; mg_set_rhs then takes f = rho with the wall terms 2 eps g / h^2
 * and eps g / h, and the cycle, the solve and the residual use the weighted operators (in
 * MG_MIXED mode the inner cycle uses single-precision copies of the coefficients, the outer
 * residual and update stay FP64). NULL returns to the constant permittivity of mg_params.
 * Errors: MG_ERR_OOM if the coefficients (7 doubles, and 5 floats in MG_MIXED mode, per cell and
 * level) cannot be allocated. */
mg_status mg_set_permittivity(mg_ctx* ctx, const double* d_eps);
/* 1 if the weighted operator is active (a variable permittivity or a reaction term is set), 0
 * otherwise (and for a NULL context). */
int mg_has_permittivity(const mg_ctx* ctx);

/* Reaction term (the Poisson-Boltzmann equation, which the paper names as the next application
 * of the solver module, Sec. 9): d_k2 (device, nx*ny*nz doubles, natural order, >= 0; not checked) gives
 * per cell k2 (the permittivity over the squared Debye length in the electrolyte, 0 where ions
 * are excluded). The operator becomes -div(eps grad phi) + k2 phi (screened, linearised
 * Poisson-Boltzmann / Debye-Hueckel), with the permittivities of mg_set_permittivity or the
 * constant eps; the reaction term adds k2 h^2 to the level-0 diagonal and is carried to the coarse
 * levels by its Galerkin product, while the diffusion part of every coarse operator carries the
 * coarse-grid correction factor (1/cgc_weight times its Galerkin product, the correction itself
 * unmagnified: the same iterates for the Poisson operator, no overshoot of the reaction part).
 * The array is copied and the coefficients built before the call returns. NULL removes the term.
 * MG_ERR_OOM if the buffers cannot be allocated. */
mg_status mg_set_reaction(mg_ctx* ctx, const double* d_k2);
int mg_has_reaction(const mg_ctx* ctx);

/* Nonlinear Poisson-Boltzmann equation -div(eps grad phi) + k2 sinh(phi) = f for a symmetric 1:1
 * electrolyte (phi in units of the thermal voltage), k2 from mg_set_reaction, f from mg_set_rhs
 * (rho with the wall terms), by Newton's method from the current solution: F = f - A_eps phi -
 * k2 sinh(phi); stop when ||F||_2 / ||f||_2 < rel_tol or after max_newton steps; else solve
 * (A_eps + k2 cosh(phi)) delta = F with homogeneous walls by V-cycles to inner_tol (at most
 * max_cycles; an inexact step is kept), phi += delta. Writes the step count and the final
 * ||F|| / ||f|| (either pointer may be NULL); the potential is the context's solution afterwards,
 * and the weighted operator holds the last linearisation (mg_set_reaction restores the linear
 * one). Returns MG_ERR_NOT_CONVERGED if the tolerance is not reached, MG_ERR_INVALID without a
 * reaction term or with negative arguments. Synchronises. */
mg_status mg_solve_pb(mg_ctx* ctx, double rel_tol, int max_newton, double inner_tol, int max_cycles, int* h_newton,
                      double* h_rel_res);

/* Right-hand side from a charge density: f = rho/eps, then adapted to the wall values once
 * on the finest grid (Sec. 2.4 and Sec. 5.3: Dirichlet face cells += 2 g / h^2, Neumann face
 * cells += g / h; periodic faces add nothing). d_rho: nx*ny*nz doubles. */
mg_status mg_set_rhs(mg_ctx* ctx, const double* d_rho);
/* Right-hand side f of A phi = f taken as is (no 1/eps, no wall terms): used for adjoint
 * solves, whose wall conditions are homogeneous. d_f: nx*ny*nz doubles. */
mg_status mg_set_rhs_f(mg_ctx* ctx, const double* d_f);

/* Start value of the iteration (warm start, Sec. 8.1: later time steps reuse the previous
 * potential). d_phi NULL sets zero. */
mg_status mg_set_solution(mg_ctx* ctx, const double* d_phi);
mg_status mg_get_solution(mg_ctx* ctx, double* d_phi);

/* ncycles V(nu1,nu2)-cycles (Sec. 3, Sec. 5.3) on the current right-hand side and solution.
 * In MG_MIXED mode one cycle is one outer defect-correction step. Stream-ordered; no sync. */
mg_status mg_vcycle(mg_ctx* ctx, int ncycles);

/* Algorithm 1: while ||f - A phi||_2 / ||f||_2 >= rel_tol and fewer than max_cycles cycles:
 * one cycle. Writes the cycle count and the final relative residual (host pointers, either
 * may be NULL). Returns MG_ERR_NOT_CONVERGED if max_cycles is reached first or the residual
 * is not finite, MG_ERR_DIVERGED if it grows above 1e3 times its starting value.
 * MG_MIXED with the constant operator, from the zero iterate of mg_set_solution(NULL) (not in
 * the paper): an outer step may carry the residual by recurrence, r <- r - s A e (see
 * mg_op_defect_update), instead of evaluating it from phi; it does so from the zero start and
 * after another such step, unless the last contraction predicts that the step reaches rel_tol.
 * The residual is evaluated directly before every decision that ends the solve (below rel_tol,
 * not finite, diverged, max_cycles), and the relative residual written to h_rel_res is always
 * that direct evaluation. Environment CCMG_DEFECT=walk (read at mg_create) evaluates it
 * directly after every step. */
mg_status mg_solve(mg_ctx* ctx, double rel_tol, int max_cycles, int* h_cycles, double* h_rel_res);
/* Counts since mg_create (host array of 3): [0] outer cycles run by mg_solve, [1] those of them
 * that carried the residual by recurrence, [2] direct evaluations of the finest-level residual
 * (mg_solve's checks, mg_residual, mg_op_residual_norm; not the stencil-free residual of a zero
 * iterate). */
mg_status mg_outer_counts(const mg_ctx* ctx, long long* h_counts3);

/* Relative residual ||f - A phi||_2 / ||f||_2 of the current solution (host scalar), and, if
 * d_r is not NULL, the residual field f - A phi itself (nx*ny*nz doubles). */
mg_status mg_residual(mg_ctx* ctx, double* h_rel_res, double* d_r);

/* E = -grad(phi) by central differences (D3Q7), with the wall ghost values
 * (Dirichlet 2 g - phi, Neumann phi + h g; across a periodic axis the cell at the opposite
 * side), or by the stencil mg_set_gradient_stencil chose.
 * d_E: 3 arrays of nx*ny*nz doubles (Ex, Ey, Ez). */
mg_status mg_efield(mg_ctx* ctx, double* d_E);

/* Gradient stencil of mg_efield, mg_force_gather and mg_step_host (Sec. 2.4, "Coulomb force"):
 *   7  (default) D3Q7 central differences everywhere, with the wall ghost values;
 *   19 the isotropy-preserving D3Q19 stencil, grad phi ~ (1/w_1) sum_q w_q phi(x + e_q) e_q / h^2
 *      (weights 1/3 rest, 1/18 faces, 1/36 edges), at every cell whose 18 neighbours lie in the
 *      domain or across periodic axes, and D3Q7 with ghosts at the others.
 * Other values return MG_ERR_INVALID and leave the setting unchanged. mg_force_gather_adjoint
 * is implemented for the D3Q7 gradient only and returns MG_ERR_INVALID while 19 is set.
 * mg_gradient_stencil returns the setting (-1 for a NULL context). */
mg_status mg_set_gradient_stencil(mg_ctx* ctx, int stencil);
int mg_gradient_stencil(const mg_ctx* ctx);

/* Charge density of P spheres with subsampling factor sf (1..8): each cell is split into sf^3
 * sub-cells and rho(cell) = sum_s density_s * (sub-cells whose centre lies in sphere s) / sf^3
 * (Sec. 2.4, "Subsampling"). Along a periodic axis a sphere that reaches across the wall puts
 * its charge in the cells at the opposite side (its periodic image); elsewhere the part outside
 * the domain is dropped. d_centers: P*3 doubles (x,y,z); d_radius, d_density: P doubles.
 * d_rho (nx*ny*nz doubles) is overwritten. */
mg_status mg_sphere_density(mg_ctx* ctx, int P, const double* d_centers, const double* d_radius,
                            const double* d_density, int sf, double* d_rho);

/* Coulomb force on each sphere, F_s = h^3 sum_b w_{s,b} density_s E(x_b) (Eq. ElectrostatForce,
 * E by the gradient of mg_efield, w the subsampled overlap; the cells b of mg_sphere_density,
 * periodic images included). d_forces: P*3 doubles. */
mg_status mg_force_gather(mg_ctx* ctx, int P, const double* d_centers, const double* d_radius,
                          const double* d_density, int sf, double* d_forces);

/* Adjoints for J = sum_{s,a} wF[s][a] F_s[a] (not in the paper). All outputs are overwritten.
 *   mg_force_gather_adjoint: d_gphi (N) = dJ/dphi, d_gdensity (P) = dJ/ddensity through the
 *     explicit density factor, d_gbc (6, device) = dJ/dbc_value through the ghost values.
 *   mg_sphere_density_adjoint: d_gdensity[s] = sum_b w_{s,b} d_gfield[b].
 *   mg_rhs_adjoint: given lambda = dJ/df, d_grho = lambda / eps and d_gbc (6, device) =
 *     sum over each face's cells of lambda * (2/h^2 Dirichlet, 1/h Neumann, 0 periodic); with the
 *     weighted operator (mg_set_permittivity / mg_set_reaction), f = rho plus eps-weighted wall
 *     terms, so d_grho = lambda and the face sums take lambda * (2 eps/h^2 or eps/h). */
mg_status mg_force_gather_adjoint(mg_ctx* ctx, int P, const double* d_centers, const double* d_radius,
                                  const double* d_density, int sf, const double* d_wF, double* d_gphi,
                                  double* d_gdensity, double* d_gbc);
mg_status mg_sphere_density_adjoint(mg_ctx* ctx, int P, const double* d_centers, const double* d_radius,
                                    int sf, const double* d_gfield, double* d_gdensity);
mg_status mg_rhs_adjoint(mg_ctx* ctx, const double* d_lambda, double* d_grho, double* d_gbc);

/* Adjoint solve (not in the paper; derived from Eq. ElectrostatForce and the wall terms of
 * Sec. 2.4): for J depending on phi = A^-1 f, dJ/df = lambda with A^T lambda = dJ/dphi. The
 * operator is symmetric (the folded 7-point stencil, its Galerkin coarse operators, and the
 * weighted operator of mg_set_permittivity / mg_set_reaction alike), so lambda solves
 * A lambda = g with homogeneous walls by the same multigrid: d_g (device, nx*ny*nz doubles,
 * natural order) is taken as the right-hand side as it is (no 1/eps, no wall terms), the
 * iteration starts from zero and runs Algorithm 1 to rel_tol (at most max_cycles cycles), and
 * lambda is written to d_lambda (device, nx*ny*nz doubles). The wall values of the forward
 * problem are neither read nor changed; the context's right-hand side and solution are replaced
 * (they hold g and lambda afterwards). Feed lambda to mg_rhs_adjoint for dJ/drho and dJ/dwall.
 * h_cycles / h_rel_res (host, may be NULL) receive the cycle count and final relative residual.
 * Returns the status of the solve (MG_ERR_NOT_CONVERGED with lambda written if the tolerance was
 * missed), MG_ERR_INVALID for null pointers, a negative tolerance or max_cycles. Synchronises. */
mg_status mg_adjoint_solve(mg_ctx* ctx, const double* d_g, double* d_lambda, double rel_tol, int max_cycles,
                           int* h_cycles, double* h_rel_res);

/* One electrostatics step with HOST buffers (Algorithm 1, the potential part): copy the
 * spheres in, set the right-hand side from their subsampled charge, solve to rel_tol from the
 * current solution (warm start), compute the force on every sphere and copy it out.
 * rel_tol < 0 selects the time-loop mode of Sec. 8.1: exactly max_cycles cycles from the current
 * solution (five at the first step, one at every later step there), h_rel_res then reporting the
 * relative residual after them. h_forces: P*3 doubles; h_cycles / h_rel_res may be NULL.
 * Synchronises. */
mg_status mg_step_host(mg_ctx* ctx, int P, const double* h_centers, const double* h_radius,
                       const double* h_density, int sf, double rel_tol, int max_cycles, double* h_forces,
                       int* h_cycles, double* h_rel_res);

/* ----------------------------------------------------------------------------------------- */
/* Level-wise operations, for verifying each kernel on its own. level 0 is the finest.
 * Level fields are exchanged in natural (x-fastest) order, in double, whatever the internal
 * layout and precision. which: 0 = solution/correction phi_l, 1 = right-hand side f_l; for
 * mg_level_get with a variable permittivity set also 2 = the diagonal D_l, 3, 4, 5 = the weights
 * of the cells' -x, -y, -z faces (scaled: A_l = (D_l phi - sum w phi_neighbour) / (2^l h^2)).
 * In MG_MIXED mode these address the single-precision hierarchy (values rounded to float). The
 * operations below use the weighted operators while a variable permittivity is set. */
mg_status mg_level_set(mg_ctx* ctx, int level, int which, const double* d_in);
mg_status mg_level_get(mg_ctx* ctx, int level, int which, double* d_out);
/* One red (colour 0, i+j+k even) or black (colour 1) Gauss-Seidel half-sweep on level l. */
mg_status mg_op_smooth(mg_ctx* ctx, int level, int colour);
/* f_{l+1} = averaging restriction of (f_l - A_l phi_l). */
mg_status mg_op_residual_restrict(mg_ctx* ctx, int level);
/* The same restriction over the red children only (their residuals times 1/4, summed in the
 * same order), the variant the single-precision cycle runs right after a black half-sweep, when
 * the black residuals are zero up to rounding. Not in the paper. */
mg_status mg_op_residual_restrict_red(mg_ctx* ctx, int level);
/* phi_l += cgc_weight * constant prolongation of phi_{l+1}. */
mg_status mg_op_prolong_correct(mg_ctx* ctx, int level);
/* The first black post-smoothing half-sweep of the single-precision cycle, fused with the
 * prolongation of the coarse correction (Sec. 3): every black cell of level l becomes the
 * half-sweep value computed from the red neighbours corrected by cgc_weight * phi_{l+1}(parent),
 * i.e. the black cells of mg_op_prolong_correct followed by mg_op_smooth(level, 1). The red cells
 * are left as they were, uncorrected (the cycle's next red half-sweep recomputes every one of
 * them). Available where the cycle runs it: MG_MIXED, constant permittivity, levels with rows of
 * whole 4-float vectors (nx a multiple of 8); MG_ERR_INVALID elsewhere.
 * mg_level_prolong_sweep_kind tells which kernel runs it: 1 the TMA-staged one, 0 the
 * direct-load one, -1 where the operation is not available. */
mg_status mg_op_prolong_smooth(mg_ctx* ctx, int level);
int mg_level_prolong_sweep_kind(const mg_ctx* ctx, int level);
/* CG on the coarsest level: phi_L = A_L^-1 f_L (rtol 1e-14, at most 2 N_L iterations);
 * h_iters (may be NULL) receives the iteration count. Synchronises. */
mg_status mg_op_coarse_solve(mg_ctx* ctx, int* h_iters);

/* Enqueue the termination residual of Algorithm 1 on its own (scaled residual and the fixed-order
 * reduction of its squared norm; in MG_MIXED mode also the scaled single-precision residual that
 * the next inner cycle solves for), without reading anything back. For timing that kernel. */
mg_status mg_op_residual_norm(mg_ctx* ctx);

/* One outer step of the MG_MIXED defect correction with the residual carried by recurrence
 * (not in the paper), for verifying it: from the iterate phi_k (d_phi; ignored with zero_start,
 * where phi_k = 0), a correction e (d_e, each value rounded to float) and the scaled residual
 * r~_k = g + sum of the six neighbours - (6 + d) phi_k (d_r; the level's units, g = f / c_0),
 * it forms phi_{k+1} = phi_k + sc e (one rounded FP64 addition; sc e exact) and
 * r~_{k+1} = r~_k - sc A e, where A e = (6 + d) e - sum of e's six neighbours is the constant
 * operator with the context's walls. The residual is carried in units of the scales as a pair of
 * floats: r~_k / sc is split into hi + lo (hi rounded to nearest, lo the rounded remainder) and
 * r~_{k+1} / sc_next is returned the same way (d_hi_out, d_lo_out: hi is the single-precision
 * right-hand side of the next inner cycles); their sum lies within 2^-44 (|r~_k| / sc +
 * |r~_{k+1}| / sc) + 2^-58 sum(|terms of A e|) of the exact value (A e is summed by three
 * cascades of error-free additions). h_sumsq receives sum(hi^2) sc_next^2, the squared norm
 * the solver takes for the next scale. All fields natural order, nx*ny*nz doubles of device
 * memory, borrowed. sc, sc_next: powers of two in [2^-800, 2^800]. Overwrites the context's
 * finest iterate, single-precision finest level and scalars (and with zero_start its finest
 * right-hand side, which then holds r~_0). MG_ERR_INVALID unless MG_MIXED with finest rows of
 * whole 4-float vectors (nx a multiple of 8), for bad scales or null pointers. Synchronises. */
mg_status mg_op_defect_update(mg_ctx* ctx, int zero_start, double sc, double sc_next, const double* d_phi,
                              const double* d_e, const double* d_r, double* d_phi_out, double* d_hi_out,
                              double* d_lo_out, double* h_sumsq);

/* Enqueue the recurrence step alone on the context's current state (the next scale from the
 * last residual norm, then the update of the iterate and of the residual pair by the current
 * single-precision finest correction, and the pair's norm), without reading anything back. For
 * timing that kernel; the state it leaves is not a residual of the iterate. MG_ERR_INVALID where
 * mg_op_defect_update is. */
mg_status mg_op_defect_step(mg_ctx* ctx);

/* The power-of-two products and precision conversions on caller data, for verifying them (not in
 * the paper): d_xf[i] = float(d_x[i] * (1/sc)) as MG_MIXED hands the outer residual to the inner
 * cycles, d_yo[i] = fma(sc, double(d_e[i]), d_y[i]) as it adds the correction, d_xs[i] =
 * d_x[i] * sc as the right-hand side and E-field kernels apply 1/eps, h^2 and 1/(2h). For a
 * power-of-two sc these run as integer exponent arithmetic with one round-to-nearest-even (the
 * solver's scales are powers of two in [2^-800, 2^800]); any other sc > 0 takes the plain
 * floating-point formula. n elements of device memory each, borrowed; enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default); no context. MG_ERR_INVALID for n < 0, null pointers
 * with n > 0, or sc not positive and finite with a finite 1/sc; MG_ERR_CUDA on a failed launch. */
mg_status mg_op_scale_convert(const double* d_x, const float* d_e, const double* d_y, long long n, double sc,
                              float* d_xf, double* d_yo, double* d_xs, void* stream);

/* Number of kernels this context has enqueued since creation (graph nodes included). */
long long mg_kernel_launches(const mg_ctx* ctx);
/* Which kernel performs the half-sweeps of a non-coarsest level: 1 = the TMA-staged z-slab
 * kernel, 0 = the vectorised direct-load kernel; -1 for an invalid context or level. Both give
 * bit-identical results. MG_MIXED takes the TMA kernel on single-precision levels with rows of
 * whole 4-float vectors, at least 8 planes and 2^24 cells per colour (where it measured faster);
 * MG_FP64 takes its FP64 counterpart on levels without a periodic axis, with rows of whole
 * 2-double vectors, at least 8 planes and 2^22 cells per colour. The environment variable
 * CCMG_SWEEP, read by mg_create, overrides this: "vec" never uses them, "tma" uses them on every
 * level they can run on (2^16 cells per colour and up). */
int mg_level_sweep_kind(const mg_ctx* ctx, int level);
/* Self-test of the device-side failure path (not in the paper): runs one TMA-staged red
 * half-sweep of `level` (single precision in MG_MIXED, FP64 in MG_FP64) in which every CTA leaves
 * one of its plane copies unissued, with a wait
 * budget of 2e7 clock cycles (about 10 ms). Each CTA's wait for that copy runs out; it sets the
 * context's error flag, waits for the copies it did issue and returns without writing the level.
 * Returns MG_ERR_TIMEOUT when the flag came back as expected (and clears it; later calls work
 * normally), MG_OK if it did not, MG_ERR_INVALID if the level has no TMA-staged sweep (see
 * mg_level_sweep_kind). Synchronises. Solves report the same flag as MG_ERR_TIMEOUT. */
mg_status mg_selftest_wait_timeout(mg_ctx* ctx, int level);

/* ----------------------------------------------------------------------------------------- */
/* Batches: B independent problems (own dimensions, cell size, walls, right-hand side; not in the
 * paper, which solves one domain) solved together. Every multigrid operation is one kernel launch
 * over all systems that take part in it; systems with different numbers of levels are scheduled
 * by depth below their finest level, all coarsest-grid CG solves share one launch, and the cycle
 * and the residual test are each one CUDA graph. Each system's iterates are bit-identical to a
 * single context solving it alone with the same parameters. All systems share prec, nu1, nu2
 * (both >= 1), cgc_weight and mixed_inner. Field pointers follow the single-context conventions
 * with the system's own dimensions. */
typedef struct mg_batch mg_batch;
mg_status mg_batch_create(int B, const mg_params* params /* B entries */, void* stream, mg_batch** out);
mg_status mg_batch_destroy(mg_batch* b);
const char* mg_batch_last_error(const mg_batch* b);
int mg_batch_size(const mg_batch* b);
mg_status mg_batch_set_rhs(mg_batch* b, int sys, const double* d_rho);        /* as mg_set_rhs */
/* Every system's right-hand side at once: h_rho is a host array of B device pointers (system s's
 * charge density, natural order, its own dimensions; none NULL). The same values, norms and
 * first defect-correction scales as B calls of mg_batch_set_rhs, in three launches instead of
 * 4 B. Stream-ordered; returns without waiting for the GPU (it may wait for the staging copy of
 * the call before the previous one). MG_ERR_INVALID for a NULL array or entry. */
mg_status mg_batch_set_rhs_all(mg_batch* b, const double* const* h_rho);
mg_status mg_batch_set_solution(mg_batch* b, int sys, const double* d_phi);   /* NULL = zero */
mg_status mg_batch_get_solution(mg_batch* b, int sys, double* d_phi);
/* ncycles cycles of every system (MG_MIXED: outer defect-correction steps). No sync. */
mg_status mg_batch_vcycle(mg_batch* b, int ncycles);
/* Algorithm 1 for every system at once: a system stops cycling as soon as its own relative
 * residual is below rel_tol (or after max_cycles); h_cycles and h_rel_res (B entries each, may
 * be NULL) receive its cycle count and final relative residual. MG_ERR_NOT_CONVERGED if any
 * system missed the tolerance. Synchronises once per cycle. */
mg_status mg_batch_solve(mg_batch* b, double rel_tol, int max_cycles, int* h_cycles, double* h_rel_res);
/* Thread-block shapes of the batched launches: h_tiles4 = {smoother bx, by, transfer bx, by},
 * bx*by a multiple of 32 and at most 256 (the smoother's bx counts 16-byte vectors of a row). */
mg_status mg_batch_set_tiles(mg_batch* b, const int* h_tiles4);
mg_status mg_batch_get_tiles(const mg_batch* b, int* h_tiles4);
/* Autotuner: times `reps` whole batched cycles for each built-in tile candidate (h_ms, at least
 * 16 entries, receives ms per cycle; *h_ncand the number of candidates), keeps the fastest and
 * returns it in h_best4. It runs cycles on the current state, so call it before setting the
 * problem, or reset the solutions afterwards. */
mg_status mg_batch_autotune(mg_batch* b, int reps, int* h_best4, double* h_ms, int* h_ncand);
long long mg_batch_kernel_launches(const mg_batch* b);

/* ----------------------------------------------------------------------------------------- */
/* Residual norm without any device allocation. The paper has no counterpart to this call.
 *
 * For callers that must not have a library call cudaMalloc or cudaFree: code whose device
 * memory is already claimed and budgeted by another allocator or a fixed pool, and
 * latency-critical loops where an allocation call (which can synchronise the whole device) is
 * not acceptable. No context is needed and nothing is allocated.
 *
 * Computes, for caller-owned fields in natural order (nx*ny*nz doubles, x fastest), the
 * residual r = f - A phi of the operator of mg_create (cell size h, wall types h_bc_type6 folded
 * into the stencil, periodic ones, in opposite pairs, wrapping around; f must already contain the
 * wall terms, as from mg_level_get(ctx, 0, 1, ...))
 * and writes d_out2[0] = ||r||_2 / ||f||_2 (||r||_2 if f is zero) and d_out2[1] = ||r||_2 to
 * device memory, enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).
 *
 * Scratch: a file-scope static device array of 2 x 4096 doubles (64 KiB), one pair of partial
 * sums per z-plane. Every GPU that loads the library holds it until the process exits. Limits:
 * nz <= 4096 (larger nz returns MG_ERR_INVALID before anything is enqueued), nx, ny >= 1, h > 0.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it with the current CUDA context; a later call under another
 * context of the device (after cudaDeviceReset, or a driver-API context) looks it up again. Make
 * the first call under each context before any stream capture. Every
 * call shares the one array: each call overwrites the partials of its own planes before
 * reading them (nothing needs to start at zero), but calls whose kernels overlap on the GPU
 * (different streams, or different host threads on one device) race on it and give wrong
 * results. Returns MG_ERR_INVALID for bad arguments, MG_ERR_CUDA if the lookup or the launch
 * fails. */
mg_status mg_residual_norm_static(int nx, int ny, int nz, double h, const int* h_bc_type6, const double* d_phi,
                                  const double* d_f, double* d_out2, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CCMG_H */
