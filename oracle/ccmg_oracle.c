/* ccmg_oracle.c -- plain, slow, obviously-correct CPU oracle for the electrostatics step of
 * Bartuschat & Ruede, "Parallel Multiphysics Simulations of Charged Particles in Microfluidic
 * Flows" (arXiv 1410.6609).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load this library. It shares no code with the CUDA path.
 *
 * Scalar FP64 loops (FP32 for the inner cycle of the mixed-precision variant), compiled with
 * -ffp-contract=off so that every product and sum is rounded on its own. No blocking, no
 * fusion: each step of the method is one loop nest, taken in the order the paper gives.
 *
 * What it computes (paper section / equation named at each function):
 *   - RHS of the Poisson equation -lap(phi) = rho/eps with Dirichlet / Neumann BCs folded into
 *     the RHS (Sec. 2.4, Eq. Poisson and the 1D derivation of the BC treatment);
 *   - the cell-centred multigrid V(nu1,nu2)-cycle: red-black Gauss-Seidel, averaging
 *     restriction, constant prolongation with a x2 magnified correction, Galerkin coarse
 *     operators in closed form, CG on the coarsest grid (Sec. 3 and Sec. 5.3);
 *   - termination on the L2 norm of the residual (Algorithm 1);
 *   - the E-field by central differences and the Coulomb force on each particle
 *     (Sec. 2.4, Eq. ElectrostatForce, D3Q7 central differences);
 *   - the charge-density subsampling of spheres (Sec. 2.4, "Subsampling");
 *   - adjoints of the force, the RHS and the subsampling (not in the paper; used to check
 *     gradients of J = sum of weighted forces).
 *
 * Boundary convention: faces 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z; bc_type 0 = Dirichlet (value = the
 * potential on the face), 1 = Neumann (value = the outward normal derivative on the face),
 * 2 = periodic (both faces of an axis; the value is unused).
 * Ghost values: Dirichlet 2 g - phi_1, Neumann phi_1 + h g (the paper derives both for
 * spacing 1; they are scaled by h here); across a periodic axis the neighbour is the cell at the
 * opposite side (Sec. 2.4). Spheres reaching across a periodic axis map their charge to the
 * cells at the opposite side, and take the field there.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Threads: with OpenMP the loops over the z-planes of a field are shared among threads (within
 * one colour for the Gauss-Seidel half-sweeps, whose cells of one colour do not depend on each
 * other); every cell is computed by the same operations as in a serial run, and every sum over
 * a field is taken in a fixed order (blocks of 2^16 values), so the results do not depend on the
 * number of threads. Without OpenMP the pragmas are ignored. */
#ifdef _OPENMP
#include <omp.h>
#endif
#define OR_PRAGMA(x) _Pragma(#x)
#define OR_PAR_FOR OR_PRAGMA(omp parallel for schedule(static))
#define OR_PAR_FOR_IF(cond) OR_PRAGMA(omp parallel for schedule(static) if(cond))

/* Number of threads of the loops above (1 without OpenMP); n < 1 leaves the setting. */
int ccmg_or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define BC_DIRICHLET 0
#define BC_NEUMANN 1
#define BC_PERIODIC 2

static size_t idx3(int i, int j, int k, int nx, int ny) {
  return (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * (size_t)k);
}

/* Diagonal shift of the folded stencil at cell (i,j,k): the neighbour entry on a boundary
 * face moves to the centre with sign +1 for Dirichlet (centre beta - alpha, alpha = -1) and
 * -1 for Neumann (centre beta + alpha). Sec. 2.4, "Boundary conditions". A periodic face keeps
 * its neighbour (the cell at the opposite side): no shift. */
static int face_shift(int type) { return type == BC_DIRICHLET ? 1 : (type == BC_NEUMANN ? -1 : 0); }

/* v modulo n in [0, n): the cell a coordinate along a periodic axis stands for. */
static int wrap_index(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}
static int diag_shift(int i, int j, int k, int nx, int ny, int nz, const int* bc) {
  int d = 0;
  if (i == 0) d += face_shift(bc[0]);
  if (i == nx - 1) d += face_shift(bc[1]);
  if (j == 0) d += face_shift(bc[2]);
  if (j == ny - 1) d += face_shift(bc[3]);
  if (k == 0) d += face_shift(bc[4]);
  if (k == nz - 1) d += face_shift(bc[5]);
  return d;
}

#define REAL double
#define FN(name) name##_d
#include "oracle_level_ops.inc"
#undef REAL
#undef FN
#define REAL float
#define FN(name) name##_f
#include "oracle_level_ops.inc"
#undef REAL
#undef FN

/* ------------------------------------------------------------------------------------------ */
/* Level hierarchy (Sec. 3): coarsen while every dimension is even and its half is >= 3.       */

#define OR_MAX_LEVELS 32

int ccmg_or_levels(int nx, int ny, int nz, int* dims_out) {
  int n = 0;
  int d[3] = {nx, ny, nz};
  for (;;) {
    if (dims_out) {
      dims_out[3 * n + 0] = d[0];
      dims_out[3 * n + 1] = d[1];
      dims_out[3 * n + 2] = d[2];
    }
    ++n;
    if (n >= OR_MAX_LEVELS) break;
    int ok = 1;
    for (int a = 0; a < 3; ++a)
      if ((d[a] % 2) != 0 || d[a] / 2 < 3) ok = 0;
    if (!ok) break;
    for (int a = 0; a < 3; ++a) d[a] /= 2;
  }
  return n;
}

/* Coefficient of level l: c_l = 1 / (2^l h^2). The Galerkin product R A_l P of the averaging
 * restriction and the constant prolongation halves the coefficient and keeps the pattern and
 * the boundary shifts (checked against the literal triple product by the tests). */
static double level_coeff(double h, int l) { return 1.0 / (ldexp(1.0, l) * h * h); }

/* ------------------------------------------------------------------------------------------ */
/* Exported single-level operations (used by per-kernel parity tests).                          */

void ccmg_or_apply(const double* phi, double* out, int nx, int ny, int nz, double c, const int* bc) {
  apply_d(phi, out, nx, ny, nz, c, bc);
}
void ccmg_or_residual(const double* phi, const double* f, double* r, int nx, int ny, int nz, double c,
                      const int* bc) {
  residual_d(phi, f, r, nx, ny, nz, c, bc);
}
void ccmg_or_rbgs_half(double* phi, const double* f, int nx, int ny, int nz, double c, const int* bc,
                       int colour) {
  rbgs_half_d(phi, f, nx, ny, nz, c, bc, colour);
}
void ccmg_or_restrict(const double* r, double* fc, int nx, int ny, int nz) {
  restrict_avg_d(r, fc, nx, ny, nz);
}
void ccmg_or_prolong_correct(double* phi, const double* ec, int nx, int ny, int nz, double omega) {
  prolong_correct_d(phi, ec, nx, ny, nz, omega);
}
void ccmg_or_apply_f(const float* phi, float* out, int nx, int ny, int nz, float c, const int* bc) {
  apply_f(phi, out, nx, ny, nz, c, bc);
}
/* Single-precision level operations (the inner cycle of the mixed-precision solve). */
void ccmg_or_rbgs_half_f(float* phi, const float* f, int nx, int ny, int nz, float c, const int* bc, int colour) {
  rbgs_half_f(phi, f, nx, ny, nz, c, bc, colour);
}
void ccmg_or_residual_f(const float* phi, const float* f, float* r, int nx, int ny, int nz, float c, const int* bc) {
  residual_f(phi, f, r, nx, ny, nz, c, bc);
}
void ccmg_or_restrict_f(const float* r, float* fc, int nx, int ny, int nz) { restrict_avg_f(r, fc, nx, ny, nz); }
void ccmg_or_prolong_correct_f(float* phi, const float* ec, int nx, int ny, int nz, float omega) {
  prolong_correct_f(phi, ec, nx, ny, nz, omega);
}

/* RHS with BCs folded in (Sec. 2.4 and Sec. 5.3 "BC Handling for Scalar Potentials": the RHS
 * is adapted once, on the finest grid only):
 *   f = rho / eps;  Dirichlet face cells f += 2 g / h^2;  Neumann face cells f += g / h.
 * Edge and corner cells receive the term of every face they touch. */
void ccmg_or_rhs(const double* rho, double* f, int nx, int ny, int nz, double h, double eps,
                 const int* bc, const double* bcv) {
  OR_PAR_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        double v = rho[p] / eps;
        const int on_face[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, k == 0, k == nz - 1};
        for (int q = 0; q < 6; ++q) {
          if (!on_face[q] || bc[q] == BC_PERIODIC) continue;
          if (bc[q] == BC_DIRICHLET)
            v = v + 2.0 * bcv[q] / (h * h);
          else
            v = v + bcv[q] / h;
        }
        f[p] = v;
      }
}

/* Boundary values given per face cell (the validation runs of Sec. 6.3 prescribe the analytic
 * potential on the boundary). bcf holds one slot per face, in face order: faces 0 and 1 (x)
 * ny*nz values indexed j + ny k, faces 2 and 3 (y) nx*nz values indexed i + nx k, faces 4 and 5
 * (z) nx*ny values indexed i + nx j; bcf_on[q] selects face q's slot over the uniform bcv[q]. The
 * value belongs to the face of the boundary cell (i,j,k). */
static double bc_at(int q, int i, int j, int k, int nx, int ny, int nz, const double* bcv, const double* bcf,
                    const int* bcf_on) {
  if (!bcf || !bcf_on || !bcf_on[q]) return bcv[q];
  const size_t sx = (size_t)ny * nz, sy = (size_t)nx * nz, sz = (size_t)nx * ny;
  const size_t off[6] = {0, sx, 2 * sx, 2 * sx + sy, 2 * sx + 2 * sy, 2 * sx + 2 * sy + sz};
  size_t t;
  if (q < 2) t = (size_t)j + (size_t)ny * k;
  else if (q < 4) t = (size_t)i + (size_t)nx * k;
  else t = (size_t)i + (size_t)nx * j;
  return bcf[off[q] + t];
}

/* ccmg_or_rhs with per-cell boundary values (bc_at): the same terms in the same order. */
void ccmg_or_rhs_field(const double* rho, double* f, int nx, int ny, int nz, double h, double eps, const int* bc,
                       const double* bcv, const double* bcf, const int* bcf_on) {
  OR_PAR_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        double v = rho[p] / eps;
        const int on_face[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, k == 0, k == nz - 1};
        for (int q = 0; q < 6; ++q) {
          if (!on_face[q] || bc[q] == BC_PERIODIC) continue;
          const double g = bc_at(q, i, j, k, nx, ny, nz, bcv, bcf, bcf_on);
          if (bc[q] == BC_DIRICHLET)
            v = v + 2.0 * g / (h * h);
          else
            v = v + g / h;
        }
        f[p] = v;
      }
}

/* Adjoint of ccmg_or_rhs: given lambda = dJ/df, returns dJ/drho = lambda / eps and
 * dJ/dbc_value[q] = sum over the face-q cells of lambda * (2/h^2 Dirichlet, 1/h Neumann). */
void ccmg_or_rhs_adjoint(const double* lam, double* grho, double* gbc, int nx, int ny, int nz,
                         double h, double eps, const int* bc) {
  for (int q = 0; q < 6; ++q) gbc[q] = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        grho[p] = lam[p] / eps;
        const int on_face[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, k == 0, k == nz - 1};
        for (int q = 0; q < 6; ++q) {
          if (!on_face[q] || bc[q] == BC_PERIODIC) continue;
          gbc[q] = gbc[q] + lam[p] * (bc[q] == BC_DIRICHLET ? 2.0 / (h * h) : 1.0 / h);
        }
      }
}

static double dot_d(const double* a, const double* b, size_t n) {
  double s = 0.0;
  for (size_t p = 0; p < n; ++p) s = s + a[p] * b[p];
  return s;
}

/* Unpreconditioned conjugate gradients (Hestenes-Stiefel) on the coarsest grid (Sec. 5.3),
 * started from x = 0 and stopped when ||r||_2 <= rtol ||b||_2 or after maxit iterations.
 * Returns the iteration count. */
int ccmg_or_cg(double* x, const double* b, int nx, int ny, int nz, double c, const int* bc, double rtol,
               int maxit) {
  const size_t n = (size_t)nx * ny * nz;
  double* r = (double*)malloc(n * sizeof(double));
  double* p = (double*)malloc(n * sizeof(double));
  double* ap = (double*)malloc(n * sizeof(double));
  for (size_t q = 0; q < n; ++q) {
    x[q] = 0.0;
    r[q] = b[q];
    p[q] = b[q];
  }
  const double bnorm = sqrt(dot_d(b, b, n));
  double rr = dot_d(r, r, n);
  int it = 0;
  if (bnorm > 0.0) {
    while (it < maxit) {
      apply_d(p, ap, nx, ny, nz, c, bc);
      const double alpha = rr / dot_d(p, ap, n);
      for (size_t q = 0; q < n; ++q) {
        x[q] = x[q] + alpha * p[q];
        r[q] = r[q] - alpha * ap[q];
      }
      ++it;
      const double rr_new = dot_d(r, r, n);
      if (sqrt(rr_new) <= rtol * bnorm) break;
      const double beta = rr_new / rr;
      for (size_t q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
      rr = rr_new;
    }
  }
  free(r);
  free(p);
  free(ap);
  return it;
}

static float dot_f(const float* a, const float* b, size_t n) {
  float s = 0.0f;
  for (size_t p = 0; p < n; ++p) s = s + a[p] * b[p];
  return s;
}

/* The same iteration in single precision, for the coarsest grid of the single-precision inner
 * cycles of the mixed-precision solver (not in the paper); rtol there is CG_RTOL_F32. */
int ccmg_or_cg_f(float* x, const float* b, int nx, int ny, int nz, float c, const int* bc, double rtol,
                 int maxit) {
  const size_t n = (size_t)nx * ny * nz;
  float* r = (float*)malloc(n * sizeof(float));
  float* p = (float*)malloc(n * sizeof(float));
  float* ap = (float*)malloc(n * sizeof(float));
  for (size_t q = 0; q < n; ++q) {
    x[q] = 0.0f;
    r[q] = b[q];
    p[q] = b[q];
  }
  const float bnorm = sqrtf(dot_f(b, b, n));
  float rr = dot_f(r, r, n);
  int it = 0;
  if (bnorm > 0.0f) {
    while (it < maxit) {
      apply_f(p, ap, nx, ny, nz, c, bc);
      const float alpha = rr / dot_f(p, ap, n);
      for (size_t q = 0; q < n; ++q) {
        x[q] = x[q] + alpha * p[q];
        r[q] = r[q] - alpha * ap[q];
      }
      ++it;
      const float rr_new = dot_f(r, r, n);
      if (sqrtf(rr_new) <= (float)rtol * bnorm) break;
      const float beta = rr_new / rr;
      for (size_t q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
      rr = rr_new;
    }
  }
  free(r);
  free(p);
  free(ap);
  return it;
}

/* ------------------------------------------------------------------------------------------ */
/* V-cycle (Sec. 3, Sec. 5.3): at level l < L-1:
 *   nu1 x (red, black);  r = f - A phi;  f_{l+1} = R r;  phi_{l+1} = 0;  V at l+1;
 *   phi += omega P phi_{l+1};  nu2 x (black, red).
 * At the coarsest level: CG from zero to rtol 1e-14 (cap 2 N_c iterations). */

typedef struct {
  int L;
  int dims[OR_MAX_LEVELS][3];
  double* phi[OR_MAX_LEVELS]; /* level 0 is the caller's array */
  double* f[OR_MAX_LEVELS];   /* level 0 is the caller's array */
  double* r;                  /* scratch, finest size */
  float* phif[OR_MAX_LEVELS]; /* single-precision hierarchy (mixed mode) */
  float* ff[OR_MAX_LEVELS];
  float* rf;
} hierarchy;

static size_t ncells(const int* d) { return (size_t)d[0] * d[1] * d[2]; }

static void hier_init(hierarchy* H, int nx, int ny, int nz, int single) {
  int dims[3 * OR_MAX_LEVELS];
  memset(H, 0, sizeof(*H));
  H->L = ccmg_or_levels(nx, ny, nz, dims);
  for (int l = 0; l < H->L; ++l) {
    for (int a = 0; a < 3; ++a) H->dims[l][a] = dims[3 * l + a];
    const size_t n = ncells(H->dims[l]);
    if (l > 0) {
      H->phi[l] = (double*)calloc(n, sizeof(double));
      H->f[l] = (double*)calloc(n, sizeof(double));
    }
    if (single) {
      H->phif[l] = (float*)calloc(n, sizeof(float));
      H->ff[l] = (float*)calloc(n, sizeof(float));
    }
  }
  H->r = (double*)calloc(ncells(H->dims[0]), sizeof(double));
  if (single) H->rf = (float*)calloc(ncells(H->dims[0]), sizeof(float));
}

static void hier_free(hierarchy* H) {
  for (int l = 0; l < H->L; ++l) {
    if (l > 0) {
      free(H->phi[l]);
      free(H->f[l]);
    }
    free(H->phif[l]);
    free(H->ff[l]);
  }
  free(H->r);
  free(H->rf);
}

#define CG_RTOL 1e-14
#define CG_RTOL_F32 1e-5 /* the single-precision inner cycles' coarsest CG (float cannot reach 1e-14) */

static void vcycle_d(hierarchy* H, int l, double h, const int* bc, int nu1, int nu2, double omega,
                     int* cg_iters) {
  const int* d = H->dims[l];
  const double c = level_coeff(h, l);
  if (l == H->L - 1) {
    const int it = ccmg_or_cg(H->phi[l], H->f[l], d[0], d[1], d[2], c, bc, CG_RTOL, 2 * (int)ncells(d));
    if (cg_iters) *cg_iters = it;
    return;
  }
  for (int s = 0; s < nu1; ++s) {
    rbgs_half_d(H->phi[l], H->f[l], d[0], d[1], d[2], c, bc, 0);
    rbgs_half_d(H->phi[l], H->f[l], d[0], d[1], d[2], c, bc, 1);
  }
  residual_d(H->phi[l], H->f[l], H->r, d[0], d[1], d[2], c, bc);
  restrict_avg_d(H->r, H->f[l + 1], d[0], d[1], d[2]);
  memset(H->phi[l + 1], 0, ncells(H->dims[l + 1]) * sizeof(double));
  vcycle_d(H, l + 1, h, bc, nu1, nu2, omega, cg_iters);
  prolong_correct_d(H->phi[l], H->phi[l + 1], d[0], d[1], d[2], omega);
  for (int s = 0; s < nu2; ++s) {
    rbgs_half_d(H->phi[l], H->f[l], d[0], d[1], d[2], c, bc, 1);
    rbgs_half_d(H->phi[l], H->f[l], d[0], d[1], d[2], c, bc, 0);
  }
}

/* Same cycle in single precision; the coarsest-grid CG stays in double. */
static void vcycle_f(hierarchy* H, int l, double h, const int* bc, int nu1, int nu2, float omega,
                     int* cg_iters) {
  const int* d = H->dims[l];
  const size_t n = ncells(d);
  if (l == H->L - 1) {
    const int it = ccmg_or_cg_f(H->phif[l], H->ff[l], d[0], d[1], d[2], (float)level_coeff(h, l), bc, CG_RTOL_F32,
                                2 * (int)n);
    if (cg_iters) *cg_iters = it;
    return;
  }
  const float c = (float)level_coeff(h, l);
  for (int s = 0; s < nu1; ++s) {
    rbgs_half_f(H->phif[l], H->ff[l], d[0], d[1], d[2], c, bc, 0);
    rbgs_half_f(H->phif[l], H->ff[l], d[0], d[1], d[2], c, bc, 1);
  }
  residual_f(H->phif[l], H->ff[l], H->rf, d[0], d[1], d[2], c, bc);
  restrict_avg_f(H->rf, H->ff[l + 1], d[0], d[1], d[2]);
  memset(H->phif[l + 1], 0, ncells(H->dims[l + 1]) * sizeof(float));
  vcycle_f(H, l + 1, h, bc, nu1, nu2, omega, cg_iters);
  prolong_correct_f(H->phif[l], H->phif[l + 1], d[0], d[1], d[2], omega);
  for (int s = 0; s < nu2; ++s) {
    rbgs_half_f(H->phif[l], H->ff[l], d[0], d[1], d[2], c, bc, 1);
    rbgs_half_f(H->phif[l], H->ff[l], d[0], d[1], d[2], c, bc, 0);
  }
}

/* Euclidean norm of a field (Algorithm 1's L2 norm): blocks of 2^16 values summed in index order,
 * the block sums added in block order. */
#define OR_NORM_BLOCK ((size_t)1 << 16)
static double norm2_d(const double* a, size_t n) {
  const size_t nb = (n + OR_NORM_BLOCK - 1) / OR_NORM_BLOCK;
  double* part = (double*)malloc((nb ? nb : 1) * sizeof(double));
  OR_PAR_FOR
  for (size_t b = 0; b < nb; ++b) {
    const size_t e = (b + 1) * OR_NORM_BLOCK < n ? (b + 1) * OR_NORM_BLOCK : n;
    double t = 0.0;
    for (size_t p = b * OR_NORM_BLOCK; p < e; ++p) t = t + a[p] * a[p];
    part[b] = t;
  }
  double s = 0.0;
  for (size_t b = 0; b < nb; ++b) s = s + part[b];
  free(part);
  return sqrt(s);
}

/* ncycles V-cycles on A_0 phi = f (f already BC-adapted), phi updated in place. Returns the
 * CG iteration count of the last coarse solve. */
int ccmg_or_vcycles(double* phi, const double* f, int nx, int ny, int nz, double h, const int* bc,
                    int nu1, int nu2, double omega, int ncycles) {
  hierarchy H;
  hier_init(&H, nx, ny, nz, 0);
  H.phi[0] = phi;
  H.f[0] = (double*)f;
  int cg = 0;
  for (int k = 0; k < ncycles; ++k) vcycle_d(&H, 0, h, bc, nu1, nu2, omega, &cg);
  H.phi[0] = NULL;
  H.f[0] = NULL;
  hier_free(&H);
  return cg;
}

/* Relative residual ||f - A_0 phi||_2 / ||f||_2 (Algorithm 1 termination test, L2 norm). */
double ccmg_or_rel_residual(const double* phi, const double* f, int nx, int ny, int nz, double h,
                            const int* bc) {
  const size_t n = (size_t)nx * ny * nz;
  double* r = (double*)malloc(n * sizeof(double));
  residual_d(phi, f, r, nx, ny, nz, level_coeff(h, 0), bc);
  const double fn = norm2_d(f, n);
  const double rn = norm2_d(r, n);
  free(r);
  return fn > 0.0 ? rn / fn : rn;
}

/* Algorithm 1: while ||r|| / ||f|| >= tol and fewer than max_cycles cycles: one V-cycle.
 * phi is the start value (warm start) and the result. Returns the number of cycles. */
int ccmg_or_solve(double* phi, const double* f, int nx, int ny, int nz, double h, const int* bc, int nu1,
                  int nu2, double omega, double tol, int max_cycles, double* rel_res_out) {
  hierarchy H;
  hier_init(&H, nx, ny, nz, 0);
  H.phi[0] = phi;
  H.f[0] = (double*)f;
  const size_t n = (size_t)nx * ny * nz;
  const double fn = norm2_d(f, n);
  int k = 0;
  double rel;
  for (;;) {
    residual_d(phi, f, H.r, nx, ny, nz, level_coeff(h, 0), bc);
    rel = fn > 0.0 ? norm2_d(H.r, n) / fn : norm2_d(H.r, n);
    if (!(rel >= tol) || k >= max_cycles) break;
    vcycle_d(&H, 0, h, bc, nu1, nu2, omega, NULL);
    ++k;
  }
  if (rel_res_out) *rel_res_out = rel;
  H.phi[0] = NULL;
  H.f[0] = NULL;
  hier_free(&H);
  return k;
}

/* Largest power of two not above v (for finite v > 0; exponent clamped to [-1000, 1000]),
 * else 1. */
static double pow2_floor(double v) {
  if (!(v > 0.0) || !(v < 1e300)) return 1.0;
  int e = 0;
  frexp(v, &e); /* v = m 2^e with 0.5 <= m < 1 */
  e -= 1;
  if (e < -1000) e = -1000;
  if (e > 1000) e = 1000;
  return ldexp(1.0, e);
}

/* Mixed-precision defect correction (not in the paper; the cycle is the paper's):
 *   loop: r = f - A_0 phi (double); stop if ||r||/||f|| < tol;
 *         s = the largest power of two not above the RMS of the previous residual (of f on
 *         the first pass), so that r / s and s e are exact;
 *         `inner` single-precision V-cycles on A_0 e = r / s, the first from e = 0 (double CG
 *         at the bottom);
 *         phi += s * e (double).
 * Returns the number of outer iterations. */
/* ncycles single-precision V-cycles (the mixed solver's inner cycles, its coarsest CG in float) on
 * A phi = f at the finest level, from phi as given; float arrays in natural order. */
int ccmg_or_vcycles_f(float* phi, const float* f, int nx, int ny, int nz, double h, const int* bc, int nu1,
                      int nu2, double omega, int ncycles) {
  hierarchy H;
  hier_init(&H, nx, ny, nz, 1);
  const size_t n = ncells(H.dims[0]);
  memcpy(H.ff[0], f, n * sizeof(float));
  memcpy(H.phif[0], phi, n * sizeof(float));
  for (int it = 0; it < ncycles; ++it) vcycle_f(&H, 0, h, bc, nu1, nu2, (float)omega, NULL);
  memcpy(phi, H.phif[0], n * sizeof(float));
  hier_free(&H);
  return ncycles;
}

int ccmg_or_solve_mixed(double* phi, const double* f, int nx, int ny, int nz, double h, const int* bc,
                        int nu1, int nu2, double omega, double tol, int max_cycles, int inner,
                        double* rel_res_out) {
  hierarchy H;
  hier_init(&H, nx, ny, nz, 1);
  const size_t n = (size_t)nx * ny * nz;
  const double fn = norm2_d(f, n);
  double scale = pow2_floor(fn / sqrt((double)n));
  int k = 0;
  double rel;
  for (;;) {
    residual_d(phi, f, H.r, nx, ny, nz, level_coeff(h, 0), bc);
    const double rn = norm2_d(H.r, n);
    rel = fn > 0.0 ? rn / fn : rn;
    if (!(rel >= tol) || k >= max_cycles) break;
    OR_PAR_FOR
    for (size_t q = 0; q < n; ++q) {
      H.ff[0][q] = (float)(H.r[q] / scale);
      H.phif[0][q] = 0.0f;
    }
    for (int it = 0; it < inner; ++it) vcycle_f(&H, 0, h, bc, nu1, nu2, (float)omega, NULL);
    OR_PAR_FOR
    for (size_t q = 0; q < n; ++q) phi[q] = phi[q] + scale * (double)H.phif[0][q];
    ++k;
    const double next = rn / sqrt((double)n);
    if (next > 0.0) scale = pow2_floor(next);
  }
  if (rel_res_out) *rel_res_out = rel;
  hier_free(&H);
  return k;
}

/* ------------------------------------------------------------------------------------------ */
/* E-field and Coulomb force (Sec. 2.4, Eq. ElectrostatForce; D3Q7 central differences).       */

/* phi at a neighbour of (i,j,k) along axis a (0,1,2) in direction dir (-1/+1); outside the
 * domain it is the ghost value of the face BC: Dirichlet 2g - phi, Neumann phi + h g. */
static double phi_nb(const double* phi, int i, int j, int k, int nx, int ny, int nz, int a, int dir,
                     double h, const int* bc, const double* bcv) {
  int q[3] = {i, j, k};
  const int n[3] = {nx, ny, nz};
  q[a] += dir;
  const double here = phi[idx3(i, j, k, nx, ny)];
  if (q[a] < 0 || q[a] >= n[a]) {
    const int face = 2 * a + (dir > 0 ? 1 : 0);
    if (bc[face] == BC_PERIODIC) {
      q[a] = wrap_index(q[a], n[a]);
      return phi[idx3(q[0], q[1], q[2], nx, ny)];
    }
    if (bc[face] == BC_DIRICHLET) return 2.0 * bcv[face] - here;
    return here + h * bcv[face];
  }
  return phi[idx3(q[0], q[1], q[2], nx, ny)];
}

/* phi_nb with per-cell boundary values (bc_at). */
static double phi_nb_f(const double* phi, int i, int j, int k, int nx, int ny, int nz, int a, int dir, double h,
                       const int* bc, const double* bcv, const double* bcf, const int* bcf_on) {
  int q[3] = {i, j, k};
  const int n[3] = {nx, ny, nz};
  q[a] += dir;
  const double here = phi[idx3(i, j, k, nx, ny)];
  if (q[a] < 0 || q[a] >= n[a]) {
    const int face = 2 * a + (dir > 0 ? 1 : 0);
    if (bc[face] == BC_PERIODIC) {
      q[a] = wrap_index(q[a], n[a]);
      return phi[idx3(q[0], q[1], q[2], nx, ny)];
    }
    const double g = bc_at(face, i, j, k, nx, ny, nz, bcv, bcf, bcf_on);
    if (bc[face] == BC_DIRICHLET) return 2.0 * g - here;
    return here + h * g;
  }
  return phi[idx3(q[0], q[1], q[2], nx, ny)];
}

/* E = -grad phi, E_a(i) = -(phi(i + e_a) - phi(i - e_a)) / (2h); out is [3][N] (SoA). */
void ccmg_or_efield(const double* phi, double* E, int nx, int ny, int nz, double h, const int* bc,
                    const double* bcv) {
  const size_t n = (size_t)nx * ny * nz;
  OR_PAR_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        for (int a = 0; a < 3; ++a) {
          const double up = phi_nb(phi, i, j, k, nx, ny, nz, a, +1, h, bc, bcv);
          const double dn = phi_nb(phi, i, j, k, nx, ny, nz, a, -1, h, bc, bcv);
          E[(size_t)a * n + p] = -(up - dn) / (2.0 * h);
        }
      }
}

/* The isotropy-preserving D3Q19 gradient (Sec. 2.4, "Coulomb force"): with lattice directions
 * e_q (6 face directions of weight 1/18, 12 edge directions of weight 1/36; the rest weight
 * w_1 = 1/3), grad phi(x) ~ (1/w_1) sum_q w_q phi(x + e_q h) e_q / h. Used where all 18
 * neighbours lie inside the domain; at the other cells the D3Q7 central differences with the
 * face ghosts above (the paper applies D3Q19 wherever it can). The directions are taken face directions first
 * (+x,-x,+y,-y,+z,-z), then the edge directions (+a+b, -a-b, +a-b, -a+b) for the axis pairs
 * (x,y), (x,z), (y,z); E_a = -grad_a phi. */
static const int d3q19_dir[18][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                     {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                     {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Whether all 18 neighbours of (i,j,k) exist: inside the domain, or across a periodic axis. */
static int d3q19_inside(int i, int j, int k, int nx, int ny, int nz, const int* bc) {
  const int q[3] = {i, j, k}, n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a)
    if (bc[2 * a] != BC_PERIODIC && (q[a] == 0 || q[a] == n[a] - 1)) return 0;
  return 1;
}

static void efield_d3q19_at(const double* phi, int i, int j, int k, int nx, int ny, int nz, double h, double E[3]) {
  double g[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 18; ++q) {
    const int* e = d3q19_dir[q];
    const double w = q < 6 ? 1.0 / 18.0 : 1.0 / 36.0;
    /* d3q19_inside holds: an index leaves the domain only along a periodic axis */
    const double v = phi[idx3(wrap_index(i + e[0], nx), wrap_index(j + e[1], ny), wrap_index(k + e[2], nz), nx, ny)];
    for (int a = 0; a < 3; ++a)
      if (e[a] != 0) g[a] = g[a] + w * v * (double)e[a];
  }
  for (int a = 0; a < 3; ++a) E[a] = -(3.0 * g[a]) / h;  /* 1 / w_1 = 3 */
}

/* E-field with the chosen gradient stencil, 7 (D3Q7 everywhere) or 19 (D3Q19 wherever it fits),
 * and per-cell boundary values (bc_at; NULL bcf: the uniform ones). */
void ccmg_or_efield_field(const double* phi, double* E, int nx, int ny, int nz, double h, const int* bc,
                          const double* bcv, const double* bcf, const int* bcf_on, int stencil) {
  const size_t n = (size_t)nx * ny * nz;
  OR_PAR_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        for (int a = 0; a < 3; ++a) {
          const double up = phi_nb_f(phi, i, j, k, nx, ny, nz, a, +1, h, bc, bcv, bcf, bcf_on);
          const double dn = phi_nb_f(phi, i, j, k, nx, ny, nz, a, -1, h, bc, bcv, bcf, bcf_on);
          E[(size_t)a * n + p] = -(up - dn) / (2.0 * h);
        }
      }
  if (stencil != 19) return;
  OR_PAR_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        if (!d3q19_inside(i, j, k, nx, ny, nz, bc)) continue;
        double e[3];
        efield_d3q19_at(phi, i, j, k, nx, ny, nz, h, e);
        for (int a = 0; a < 3; ++a) E[(size_t)a * n + idx3(i, j, k, nx, ny)] = e[a];
      }
}

void ccmg_or_efield_stencil(const double* phi, double* E, int nx, int ny, int nz, double h, const int* bc,
                            const double* bcv, int stencil) {
  ccmg_or_efield_field(phi, E, nx, ny, nz, h, bc, bcv, NULL, NULL, stencil);
}

/* Subsampled overlap count of sphere (centre c, radius R) with cell (i,j,k): the cell is cut
 * into sf^3 equal sub-cells and a sub-cell counts when its centre x satisfies |x - c|^2 <= R^2
 * (Sec. 2.4, "Subsampling"; sf = 1 is the plain cell-centre mapping of Sec. 2.2). Sub-cell
 * centre coordinate: (i + (2m+1)/(2 sf)) * h. */
static int overlap_count(int i, int j, int k, double h, const double* c, double R, int sf) {
  int cnt = 0;
  const double R2 = R * R;
  for (int mk = 0; mk < sf; ++mk) {
    const double z = ((double)k + (double)(2 * mk + 1) / (double)(2 * sf)) * h;
    const double dz = z - c[2];
    for (int mj = 0; mj < sf; ++mj) {
      const double y = ((double)j + (double)(2 * mj + 1) / (double)(2 * sf)) * h;
      const double dy = y - c[1];
      for (int mi = 0; mi < sf; ++mi) {
        const double x = ((double)i + (double)(2 * mi + 1) / (double)(2 * sf)) * h;
        const double dx = x - c[0];
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 <= R2) ++cnt;
      }
    }
  }
  return cnt;
}

/* Cell range [lo, hi] along one axis that can touch a sphere (all other cells have count 0);
 * clipped to the domain unless the axis is periodic, where cells beyond an end stand for those at
 * the opposite side (the sphere's periodic image). */
static void cell_range(double c, double R, double h, int n, int periodic, int* lo, int* hi) {
  int a = (int)floor((c - R) / h) - 1;
  int b = (int)floor((c + R) / h) + 1;
  if (!periodic && a < 0) a = 0;
  if (!periodic && b > n - 1) b = n - 1;
  *lo = a;
  *hi = b;
}

/* The cell ranges of sphere s on the three axes (bc NULL: no periodic axis). */
static void sphere_range(const double* c, double R, double h, const int* n, const int* bc, int* lo, int* hi) {
  for (int a = 0; a < 3; ++a) cell_range(c[a], R, h, n[a], bc && bc[2 * a] == BC_PERIODIC, &lo[a], &hi[a]);
}

/* Storage index of the cell a (possibly periodic-image) coordinate stands for. */
static size_t cell_index(int i, int j, int k, int nx, int ny, int nz) {
  return idx3(wrap_index(i, nx), wrap_index(j, ny), wrap_index(k, nz), nx, ny);
}

/* Volume-overlap weight w_{s,b} = count / sf^3 of sphere s in cell b. */
static double overlap_weight(int i, int j, int k, double h, const double* c, double R, int sf) {
  const int cnt = overlap_count(i, j, k, h, c, R, sf);
  return (double)cnt / (double)(sf * sf * sf);
}

/* Charge density field: rho(b) = sum_s density_s * w_{s,b} (spheres in index order); bc (NULL:
 * none) marks the periodic axes, across which a sphere's charge reaches the opposite side. */
void ccmg_or_sphere_density_bc(double* rho, int nx, int ny, int nz, double h, int P, const double* centers,
                               const double* radius, const double* density, int sf, const int* bc) {
  memset(rho, 0, (size_t)nx * ny * nz * sizeof(double));
  const int n[3] = {nx, ny, nz};
  for (int s = 0; s < P; ++s) {
    const double* c = centers + 3 * s;
    int lo[3], hi[3];
    sphere_range(c, radius[s], h, n, bc, lo, hi);
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int cnt = overlap_count(i, j, k, h, c, radius[s], sf);
          if (cnt == 0) continue;
          const size_t p = cell_index(i, j, k, nx, ny, nz);
          rho[p] = rho[p] + density[s] * ((double)cnt / (double)(sf * sf * sf));
        }
  }
}

void ccmg_or_sphere_density(double* rho, int nx, int ny, int nz, double h, int P, const double* centers,
                            const double* radius, const double* density, int sf) {
  ccmg_or_sphere_density_bc(rho, nx, ny, nz, h, P, centers, radius, density, sf, NULL);
}

/* Adjoint of the density map: g_s += sum_b w_{s,b} gfield(b). */
void ccmg_or_sphere_density_adjoint_bc(const double* gfield, double* gdensity, int nx, int ny, int nz, double h,
                                       int P, const double* centers, const double* radius, int sf, const int* bc) {
  const int n[3] = {nx, ny, nz};
  for (int s = 0; s < P; ++s) {
    const double* c = centers + 3 * s;
    int lo[3], hi[3];
    sphere_range(c, radius[s], h, n, bc, lo, hi);
    double acc = 0.0;
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const double w = overlap_weight(i, j, k, h, c, radius[s], sf);
          if (w == 0.0) continue;
          acc = acc + w * gfield[cell_index(i, j, k, nx, ny, nz)];
        }
    gdensity[s] = gdensity[s] + acc;
  }
}

void ccmg_or_sphere_density_adjoint(const double* gfield, double* gdensity, int nx, int ny, int nz,
                                    double h, int P, const double* centers, const double* radius, int sf) {
  ccmg_or_sphere_density_adjoint_bc(gfield, gdensity, nx, ny, nz, h, P, centers, radius, sf, NULL);
}

/* Coulomb force on each sphere (Eq. ElectrostatForce with E = -grad phi):
 *   F_s = h^3 * sum_b w_{s,b} density_s E(x_b),
 * E by the gradient stencil of ccmg_or_efield_stencil (7: central differences everywhere; 19:
 * D3Q19 wherever it fits), taken at the cell a periodic-image coordinate stands for. forces is
 * [P][3]. */
void ccmg_or_force_gather_field(const double* phi, int nx, int ny, int nz, double h, const int* bc,
                                const double* bcv, const double* bcf, const int* bcf_on, int P,
                                const double* centers, const double* radius, const double* density, int sf,
                                int stencil, double* forces) {
  const double h3 = h * h * h;
  const int n[3] = {nx, ny, nz};
  OR_PAR_FOR
  for (int s = 0; s < P; ++s) {
    const double* c = centers + 3 * s;
    int lo[3], hi[3];
    sphere_range(c, radius[s], h, n, bc, lo, hi);
    double F[3] = {0.0, 0.0, 0.0};
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const double w = overlap_weight(i, j, k, h, c, radius[s], sf);
          if (w == 0.0) continue;
          const int iw = wrap_index(i, nx), jw = wrap_index(j, ny), kw = wrap_index(k, nz);
          double E[3];
          if (stencil == 19 && d3q19_inside(iw, jw, kw, nx, ny, nz, bc)) {
            efield_d3q19_at(phi, iw, jw, kw, nx, ny, nz, h, E);
          } else {
            for (int a = 0; a < 3; ++a) {
              const double up = phi_nb_f(phi, iw, jw, kw, nx, ny, nz, a, +1, h, bc, bcv, bcf, bcf_on);
              const double dn = phi_nb_f(phi, iw, jw, kw, nx, ny, nz, a, -1, h, bc, bcv, bcf, bcf_on);
              E[a] = -(up - dn) / (2.0 * h);
            }
          }
          for (int a = 0; a < 3; ++a) F[a] = F[a] + w * E[a];
        }
    for (int a = 0; a < 3; ++a) forces[3 * s + a] = h3 * density[s] * F[a];
  }
}

void ccmg_or_force_gather_stencil(const double* phi, int nx, int ny, int nz, double h, const int* bc,
                                  const double* bcv, int P, const double* centers, const double* radius,
                                  const double* density, int sf, int stencil, double* forces) {
  ccmg_or_force_gather_field(phi, nx, ny, nz, h, bc, bcv, NULL, NULL, P, centers, radius, density, sf, stencil,
                             forces);
}

void ccmg_or_force_gather(const double* phi, int nx, int ny, int nz, double h, const int* bc,
                          const double* bcv, int P, const double* centers, const double* radius,
                          const double* density, int sf, double* forces) {
  const double h3 = h * h * h;
  const int n[3] = {nx, ny, nz};
  for (int s = 0; s < P; ++s) {
    const double* c = centers + 3 * s;
    int lo[3], hi[3];
    sphere_range(c, radius[s], h, n, bc, lo, hi);
    double F[3] = {0.0, 0.0, 0.0};
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const double w = overlap_weight(i, j, k, h, c, radius[s], sf);
          if (w == 0.0) continue;
          const int iw = wrap_index(i, nx), jw = wrap_index(j, ny), kw = wrap_index(k, nz);
          for (int a = 0; a < 3; ++a) {
            const double up = phi_nb(phi, iw, jw, kw, nx, ny, nz, a, +1, h, bc, bcv);
            const double dn = phi_nb(phi, iw, jw, kw, nx, ny, nz, a, -1, h, bc, bcv);
            const double Ea = -(up - dn) / (2.0 * h);
            F[a] = F[a] + w * Ea;
          }
        }
    for (int a = 0; a < 3; ++a) forces[3 * s + a] = h3 * density[s] * F[a];
  }
}

/* Adjoint of ccmg_or_force_gather for J = sum_{s,a} wF[s][a] * F_s[a]:
 *   gphi   (N)  += dJ/dphi      (scatter of the central differences, ghosts included; across a
 *                               periodic axis to the cell at the opposite side)
 *   gdens  (P)  += dJ/ddensity_s through the explicit density factor
 *   gbc    (6)  += dJ/dbc_value through the ghost values used by the differences. */
void ccmg_or_force_gather_adjoint(const double* phi, int nx, int ny, int nz, double h, const int* bc,
                                  const double* bcv, int P, const double* centers, const double* radius,
                                  const double* density, int sf, const double* wF, double* gphi,
                                  double* gdens, double* gbc) {
  const double h3 = h * h * h;
  const int n[3] = {nx, ny, nz};
  for (int s = 0; s < P; ++s) {
    const double* c = centers + 3 * s;
    int lo[3], hi[3];
    sphere_range(c, radius[s], h, n, bc, lo, hi);
    double Fsum[3] = {0.0, 0.0, 0.0};
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const double w = overlap_weight(i, j, k, h, c, radius[s], sf);
          if (w == 0.0) continue;
          const int cell[3] = {wrap_index(i, nx), wrap_index(j, ny), wrap_index(k, nz)};
          const size_t p = idx3(cell[0], cell[1], cell[2], nx, ny);
          for (int a = 0; a < 3; ++a) {
            const double up = phi_nb(phi, cell[0], cell[1], cell[2], nx, ny, nz, a, +1, h, bc, bcv);
            const double dn = phi_nb(phi, cell[0], cell[1], cell[2], nx, ny, nz, a, -1, h, bc, bcv);
            Fsum[a] = Fsum[a] + w * (-(up - dn) / (2.0 * h));
            /* dJ/dE_a(b) = wF[s][a] * h3 * density_s * w; E_a = -(up - dn)/(2h). */
            const double gE = wF[3 * s + a] * h3 * density[s] * w;
            const double g_up = -gE / (2.0 * h);
            const double g_dn = +gE / (2.0 * h);
            for (int side = 0; side < 2; ++side) {
              const int dir = side == 0 ? +1 : -1;
              const double g = side == 0 ? g_up : g_dn;
              int qn[3] = {cell[0], cell[1], cell[2]};
              qn[a] += dir;
              const int face = 2 * a + (dir > 0 ? 1 : 0);
              if ((qn[a] < 0 || qn[a] >= n[a]) && bc[face] != BC_PERIODIC) {
                if (bc[face] == BC_DIRICHLET) {
                  gbc[face] = gbc[face] + 2.0 * g;
                  gphi[p] = gphi[p] - g;
                } else {
                  gbc[face] = gbc[face] + h * g;
                  gphi[p] = gphi[p] + g;
                }
              } else {
                const size_t pn = cell_index(qn[0], qn[1], qn[2], nx, ny, nz);
                gphi[pn] = gphi[pn] + g;
              }
            }
          }
        }
    for (int a = 0; a < 3; ++a) gdens[s] = gdens[s] + wF[3 * s + a] * h3 * Fsum[a];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Variable permittivity (Sec. 3: the solver extends to discontinuous dielectricity by Galerkin
 * coarsening with the averaging restriction and the nearest-neighbour prolongation, after
 * Alcouffe et al.). The equation is -div(eps grad phi) = rho; the finite-volume flux between two
 * cells has the weight of the harmonic mean of their permittivities (the flux-continuous choice
 * for a jump at the face). Each level carries, in natural order and scaled like the constant
 * case (A_l = c_l * (D phi - sum of w phi_neighbour), c_l = 1/(2^l h^2)):
 *   wx[i,j,k]  weight of the face between cells i-1 and i (at i = 0: the -x wall face, or across
 *              a periodic axis the face to cell nx-1); wy, wz likewise;
 *   D[i,j,k]   the diagonal: the weights of the cell's six faces, a Dirichlet wall face counted
 *              twice (ghost 2 g - phi), a Neumann wall face not at all (ghost phi + h g).
 * The wall face of a cell has the weight of the cell's own permittivity. With eps = 1 the
 * weights are 1 and D = 6 + d, the constant operator above.
 * Galerkin: A_{l+1} = R A_l P with R = P^T / 8, so in scaled form (c_{l+1} = c_l / 2)
 *   w_{l+1}(coarse face) = (1/4) * (sum of the 4 fine face weights on it),
 *   D_{l+1}(I) = (1/4) * (sum of the 8 children's D - 2 * the 12 faces inside I),
 * the entries of (1/4) P^T A~_l P written out (checked against the literal product by the tests). */

typedef struct {
  int n[3];
  double *D, *wx, *wy, *wz;
  double *Dw, *M; /* D = Dw + M: the diffusion part and the reaction (mass) part */
} var_level;

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

static void var_alloc(var_level* V, const int* d) {
  const size_t n = (size_t)d[0] * d[1] * d[2];
  for (int a = 0; a < 3; ++a) V->n[a] = d[a];
  V->D = (double*)calloc(n, sizeof(double));
  V->wx = (double*)calloc(n, sizeof(double));
  V->wy = (double*)calloc(n, sizeof(double));
  V->wz = (double*)calloc(n, sizeof(double));
  V->Dw = (double*)calloc(n, sizeof(double));
  V->M = (double*)calloc(n, sizeof(double));
}

static void var_free(var_level* V) {
  free(V->D);
  free(V->wx);
  free(V->wy);
  free(V->wz);
  free(V->Dw);
  free(V->M);
}

/* Level-0 weights from the cell permittivities. */
static void var_fine(const double* eps, const int* bc, var_level* V) {
  const int nx = V->n[0], ny = V->n[1], nz = V->n[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        const double e = eps[p];
        V->wx[p] = i > 0 ? harmonic(eps[idx3(i - 1, j, k, nx, ny)], e)
                         : (bc[0] == BC_PERIODIC ? harmonic(eps[idx3(nx - 1, j, k, nx, ny)], e) : e);
        V->wy[p] = j > 0 ? harmonic(eps[idx3(i, j - 1, k, nx, ny)], e)
                         : (bc[2] == BC_PERIODIC ? harmonic(eps[idx3(i, ny - 1, k, nx, ny)], e) : e);
        V->wz[p] = k > 0 ? harmonic(eps[idx3(i, j, k - 1, nx, ny)], e)
                         : (bc[4] == BC_PERIODIC ? harmonic(eps[idx3(i, j, nz - 1, nx, ny)], e) : e);
      }
  /* the diagonal: six faces in the order -x,+x,-y,+y,-z,+z */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        const double e = eps[p];
        const int pos[3] = {i, j, k};
        const double* w[3] = {V->wx, V->wy, V->wz};
        double D = 0.0;
        for (int a = 0; a < 3; ++a) {
          const int n = V->n[a];
          /* minus face */
          if (pos[a] > 0 || bc[2 * a] == BC_PERIODIC) D = D + w[a][p];
          else if (bc[2 * a] == BC_DIRICHLET) D = D + 2.0 * e;
          /* plus face: the minus face of the next cell (of cell 0 across a periodic axis) */
          int q[3] = {i, j, k};
          if (pos[a] < n - 1) {
            q[a] += 1;
            D = D + w[a][idx3(q[0], q[1], q[2], nx, ny)];
          } else if (bc[2 * a + 1] == BC_PERIODIC) {
            q[a] = 0;
            D = D + w[a][idx3(q[0], q[1], q[2], nx, ny)];
          } else if (bc[2 * a + 1] == BC_DIRICHLET) {
            D = D + 2.0 * e;
          }
        }
        V->Dw[p] = D;
        V->M[p] = 0.0;
        V->D[p] = D;
      }
}

/* Coarse weights (fine level F, coarse level C with half the dimensions): the Galerkin product
 * of the diffusion part divided by the correction factor omega, and that of the reaction part.
 * The paper magnifies the coarse-grid correction of the Poisson operator by about two because
 * the averaging restriction and constant prolongation are of too low order for a second-order
 * operator; taking the factor into the coarse operator instead (A_c = R A_diff P / omega +
 * R M P, correction weight 1) gives the same iterates for the Poisson operator (omega a power of
 * two: bit for bit) and leaves the zeroth-order reaction term, which these transfers coarsen
 * exactly, without magnification. */
static void var_coarsen(const var_level* F, var_level* C, double omega) {
  const int nx = F->n[0], ny = F->n[1];
  for (int K = 0; K < C->n[2]; ++K)
    for (int J = 0; J < C->n[1]; ++J)
      for (int I = 0; I < C->n[0]; ++I) {
        double sx = 0.0, sy = 0.0, sz = 0.0, sd = 0.0, sm = 0.0, inner = 0.0;
        for (int u = 0; u < 2; ++u)
          for (int v = 0; v < 2; ++v) {
            sx = sx + F->wx[idx3(2 * I, 2 * J + u, 2 * K + v, nx, ny)];
            sy = sy + F->wy[idx3(2 * I + u, 2 * J, 2 * K + v, nx, ny)];
            sz = sz + F->wz[idx3(2 * I + u, 2 * J + v, 2 * K, nx, ny)];
          }
        for (int dk = 0; dk < 2; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              sd = sd + F->Dw[idx3(2 * I + di, 2 * J + dj, 2 * K + dk, nx, ny)];
              sm = sm + F->M[idx3(2 * I + di, 2 * J + dj, 2 * K + dk, nx, ny)];
            }
        for (int u = 0; u < 2; ++u)
          for (int v = 0; v < 2; ++v) {
            inner = inner + F->wx[idx3(2 * I + 1, 2 * J + u, 2 * K + v, nx, ny)];
            inner = inner + F->wy[idx3(2 * I + u, 2 * J + 1, 2 * K + v, nx, ny)];
            inner = inner + F->wz[idx3(2 * I + u, 2 * J + v, 2 * K + 1, nx, ny)];
          }
        const size_t p = idx3(I, J, K, C->n[0], C->n[1]);
        C->wx[p] = sx / 4.0 / omega;
        C->wy[p] = sy / 4.0 / omega;
        C->wz[p] = sz / 4.0 / omega;
        C->Dw[p] = (sd - 2.0 * inner) / 4.0 / omega;
        C->M[p] = sm / 4.0;
        C->D[p] = C->Dw[p] + C->M[p];
      }
}

/* Weighted sum of the neighbours, in the order -x,+x,-y,+y,-z,+z (walls: none). */
static double var_nbsum(const double* phi, const var_level* V, const int* bc, int i, int j, int k) {
  const int nx = V->n[0], ny = V->n[1], nz = V->n[2];
  const size_t p = idx3(i, j, k, nx, ny);
  double s = 0.0;
  if (i > 0) s = s + V->wx[p] * phi[idx3(i - 1, j, k, nx, ny)];
  else if (bc[0] == BC_PERIODIC) s = s + V->wx[p] * phi[idx3(nx - 1, j, k, nx, ny)];
  if (i < nx - 1) s = s + V->wx[idx3(i + 1, j, k, nx, ny)] * phi[idx3(i + 1, j, k, nx, ny)];
  else if (bc[1] == BC_PERIODIC) s = s + V->wx[idx3(0, j, k, nx, ny)] * phi[idx3(0, j, k, nx, ny)];
  if (j > 0) s = s + V->wy[p] * phi[idx3(i, j - 1, k, nx, ny)];
  else if (bc[2] == BC_PERIODIC) s = s + V->wy[p] * phi[idx3(i, ny - 1, k, nx, ny)];
  if (j < ny - 1) s = s + V->wy[idx3(i, j + 1, k, nx, ny)] * phi[idx3(i, j + 1, k, nx, ny)];
  else if (bc[3] == BC_PERIODIC) s = s + V->wy[idx3(i, 0, k, nx, ny)] * phi[idx3(i, 0, k, nx, ny)];
  if (k > 0) s = s + V->wz[p] * phi[idx3(i, j, k - 1, nx, ny)];
  else if (bc[4] == BC_PERIODIC) s = s + V->wz[p] * phi[idx3(i, j, nz - 1, nx, ny)];
  if (k < nz - 1) s = s + V->wz[idx3(i, j, k + 1, nx, ny)] * phi[idx3(i, j, k + 1, nx, ny)];
  else if (bc[5] == BC_PERIODIC) s = s + V->wz[idx3(i, j, 0, nx, ny)] * phi[idx3(i, j, 0, nx, ny)];
  return s;
}

static void var_apply(const double* phi, double* out, const var_level* V, double c, const int* bc) {
  for (int k = 0; k < V->n[2]; ++k)
    for (int j = 0; j < V->n[1]; ++j)
      for (int i = 0; i < V->n[0]; ++i) {
        const size_t p = idx3(i, j, k, V->n[0], V->n[1]);
        out[p] = c * (V->D[p] * phi[p] - var_nbsum(phi, V, bc, i, j, k));
      }
}

static void var_residual(const double* phi, const double* f, double* r, const var_level* V, double c,
                         const int* bc) {
  for (int k = 0; k < V->n[2]; ++k)
    for (int j = 0; j < V->n[1]; ++j)
      for (int i = 0; i < V->n[0]; ++i) {
        const size_t p = idx3(i, j, k, V->n[0], V->n[1]);
        r[p] = f[p] - c * (V->D[p] * phi[p] - var_nbsum(phi, V, bc, i, j, k));
      }
}

/* One colour of red-black Gauss-Seidel: phi_i = (f_i / c + weighted neighbours) / D_i. */
static void var_rbgs_half(double* phi, const double* f, const var_level* V, double c, const int* bc, int colour) {
  for (int k = 0; k < V->n[2]; ++k)
    for (int j = 0; j < V->n[1]; ++j)
      for (int i = 0; i < V->n[0]; ++i) {
        if (((i + j + k) & 1) != colour) continue;
        const size_t p = idx3(i, j, k, V->n[0], V->n[1]);
        phi[p] = (f[p] / c + var_nbsum(phi, V, bc, i, j, k)) / V->D[p];
      }
}

/* CG on the coarsest level, as ccmg_or_cg with the weighted operator. */
static int var_cg(double* x, const double* b, const var_level* V, double c, const int* bc, double rtol, int maxit) {
  const size_t n = (size_t)V->n[0] * V->n[1] * V->n[2];
  double* r = (double*)malloc(n * sizeof(double));
  double* p = (double*)malloc(n * sizeof(double));
  double* ap = (double*)malloc(n * sizeof(double));
  for (size_t q = 0; q < n; ++q) {
    x[q] = 0.0;
    r[q] = b[q];
    p[q] = b[q];
  }
  const double bnorm = sqrt(dot_d(b, b, n));
  double rr = dot_d(r, r, n);
  int it = 0;
  if (bnorm > 0.0) {
    while (it < maxit) {
      var_apply(p, ap, V, c, bc);
      const double alpha = rr / dot_d(p, ap, n);
      for (size_t q = 0; q < n; ++q) {
        x[q] = x[q] + alpha * p[q];
        r[q] = r[q] - alpha * ap[q];
      }
      ++it;
      const double rr_new = dot_d(r, r, n);
      if (sqrt(rr_new) <= rtol * bnorm) break;
      const double beta = rr_new / rr;
      for (size_t q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
      rr = rr_new;
    }
  }
  free(r);
  free(p);
  free(ap);
  return it;
}

typedef struct {
  hierarchy H;
  var_level V[OR_MAX_LEVELS];
} var_hierarchy;

/* The weighted hierarchy of eps, with the reaction coefficient r (NULL: none) on level 0, coarse
 * levels by var_coarsen with the correction factor omega. */
static void var_hier_init_r(var_hierarchy* G, const double* eps, const double* r, double h, int nx, int ny, int nz,
                            const int* bc, double omega) {
  hier_init(&G->H, nx, ny, nz, 0);
  for (int l = 0; l < G->H.L; ++l) var_alloc(&G->V[l], G->H.dims[l]);
  var_fine(eps, bc, &G->V[0]);
  if (r) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t p = 0; p < n; ++p) {
      G->V[0].M[p] = r[p] * (h * h);
      G->V[0].D[p] = G->V[0].Dw[p] + G->V[0].M[p];
    }
  }
  for (int l = 1; l < G->H.L; ++l) var_coarsen(&G->V[l - 1], &G->V[l], omega);
}

static void var_hier_free(var_hierarchy* G) {
  for (int l = 0; l < G->H.L; ++l) var_free(&G->V[l]);
  hier_free(&G->H);
}

static void var_vcycle(var_hierarchy* G, int l, double h, const int* bc, int nu1, int nu2, double omega) {
  hierarchy* H = &G->H;
  const var_level* V = &G->V[l];
  const int* d = H->dims[l];
  const double c = level_coeff(h, l);
  if (l == H->L - 1) {
    var_cg(H->phi[l], H->f[l], V, c, bc, CG_RTOL, 2 * (int)ncells(d));
    return;
  }
  for (int s = 0; s < nu1; ++s) {
    var_rbgs_half(H->phi[l], H->f[l], V, c, bc, 0);
    var_rbgs_half(H->phi[l], H->f[l], V, c, bc, 1);
  }
  var_residual(H->phi[l], H->f[l], H->r, V, c, bc);
  restrict_avg_d(H->r, H->f[l + 1], d[0], d[1], d[2]);
  memset(H->phi[l + 1], 0, ncells(H->dims[l + 1]) * sizeof(double));
  var_vcycle(G, l + 1, h, bc, nu1, nu2, omega);
  prolong_correct_d(H->phi[l], H->phi[l + 1], d[0], d[1], d[2], 1.0); /* omega is in the coarse operator */
  for (int s = 0; s < nu2; ++s) {
    var_rbgs_half(H->phi[l], H->f[l], V, c, bc, 1);
    var_rbgs_half(H->phi[l], H->f[l], V, c, bc, 0);
  }
}

/* The scaled weights of level `level` (D, wx, wy, wz, each of that level's cell count) of the
 * hierarchy of eps with the reaction coefficient k2 (NULL: none) and correction factor omega. */
void ccmg_or_var_coeffs(const double* eps, const double* k2, double h, int nx, int ny, int nz, const int* bc,
                        double omega, int level, double* D, double* wx, double* wy, double* wz) {
  var_hierarchy G;
  var_hier_init_r(&G, eps, k2, h, nx, ny, nz, bc, omega);
  const size_t n = ncells(G.H.dims[level]);
  memcpy(D, G.V[level].D, n * sizeof(double));
  memcpy(wx, G.V[level].wx, n * sizeof(double));
  memcpy(wy, G.V[level].wy, n * sizeof(double));
  memcpy(wz, G.V[level].wz, n * sizeof(double));
  var_hier_free(&G);
}

/* out = A_l phi_l on level `level` of that hierarchy (fine dimensions nx, ny, nz). */
void ccmg_or_var_apply(const double* phi, double* out, const double* eps, const double* k2, int nx, int ny, int nz,
                       double h, const int* bc, double omega, int level) {
  var_hierarchy G;
  var_hier_init_r(&G, eps, k2, h, nx, ny, nz, bc, omega);
  var_apply(phi, out, &G.V[level], level_coeff(h, level), bc);
  var_hier_free(&G);
}

/* Right-hand side of -div(eps grad phi) (+ reaction) = rho with the walls folded in once on the
 * finest grid: f = rho; Dirichlet face cells f += 2 eps g / h^2; Neumann face cells f += eps g / h
 * (eps of the boundary cell, the weight of its wall face); periodic faces add nothing. */
void ccmg_or_var_rhs(const double* rho, const double* eps, double* f, int nx, int ny, int nz, double h, const int* bc,
                     const double* bcv) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        double v = rho[p];
        const int on_face[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, k == 0, k == nz - 1};
        for (int q = 0; q < 6; ++q) {
          if (!on_face[q] || bc[q] == BC_PERIODIC) continue;
          if (bc[q] == BC_DIRICHLET)
            v = v + 2.0 * eps[p] * bcv[q] / (h * h);
          else
            v = v + eps[p] * bcv[q] / h;
        }
        f[p] = v;
      }
}

/* ncycles V-cycles (as ccmg_or_vcycles) with the weighted operators. */
void ccmg_or_var_vcycles(double* phi, const double* f, const double* eps, const double* k2, int nx, int ny, int nz,
                         double h, const int* bc, int nu1, int nu2, double omega, int ncycles) {
  var_hierarchy G;
  var_hier_init_r(&G, eps, k2, h, nx, ny, nz, bc, omega);
  G.H.phi[0] = phi;
  G.H.f[0] = (double*)f;
  for (int k = 0; k < ncycles; ++k) var_vcycle(&G, 0, h, bc, nu1, nu2, omega);
  G.H.phi[0] = NULL;
  G.H.f[0] = NULL;
  var_hier_free(&G);
}

/* Algorithm 1 with the weighted operators; returns the cycle count. */
int ccmg_or_var_solve(double* phi, const double* f, const double* eps, const double* k2, int nx, int ny, int nz,
                      double h, const int* bc, int nu1, int nu2, double omega, double tol, int max_cycles,
                      double* rel_res_out) {
  var_hierarchy G;
  var_hier_init_r(&G, eps, k2, h, nx, ny, nz, bc, omega);
  G.H.phi[0] = phi;
  G.H.f[0] = (double*)f;
  const size_t n = (size_t)nx * ny * nz;
  const double fn = norm2_d(f, n);
  int k = 0;
  double rel;
  for (;;) {
    var_residual(phi, f, G.H.r, &G.V[0], level_coeff(h, 0), bc);
    rel = fn > 0.0 ? norm2_d(G.H.r, n) / fn : norm2_d(G.H.r, n);
    if (!(rel >= tol) || k >= max_cycles) break;
    var_vcycle(&G, 0, h, bc, nu1, nu2, omega);
    ++k;
  }
  if (rel_res_out) *rel_res_out = rel;
  G.H.phi[0] = NULL;
  G.H.f[0] = NULL;
  var_hier_free(&G);
  return k;
}

/* Relative residual ||f - A_0 phi|| / ||f|| with the weighted operator. */
double ccmg_or_var_rel_residual(const double* phi, const double* f, const double* eps, const double* k2, int nx,
                                int ny, int nz, double h, const int* bc) {
  var_hierarchy G;
  var_hier_init_r(&G, eps, k2, h, nx, ny, nz, bc, 2.0);
  const size_t n = (size_t)nx * ny * nz;
  double* r = (double*)malloc(n * sizeof(double));
  var_residual(phi, f, r, &G.V[0], level_coeff(h, 0), bc);
  const double fn = norm2_d(f, n), rn = norm2_d(r, n);
  free(r);
  var_hier_free(&G);
  return fn > 0.0 ? rn / fn : rn;
}

/* ------------------------------------------------------------------------------------------ */
/* Screened and Poisson-Boltzmann operators (the paper names the Poisson-Boltzmann equation as
 * the next application of the solver module, Sec. 9): with a reaction coefficient k2 >= 0 per
 * cell (the squared inverse Debye length times the permittivity in the electrolyte, zero where
 * ions are excluded) the equation is
 *   -div(eps grad phi) + k2 phi = rho          (linear, Debye-Hueckel), or
 *   -div(eps grad phi) + k2 sinh(phi) = rho    (nonlinear, symmetric 1:1 electrolyte, phi in
 *                                                units of the thermal voltage).
 * The reaction term is cell-local: it adds k2 h^2 to the scaled diagonal of level 0 (A_0 =
 * c_0 (D phi - sum w phi) + k2 phi, c_0 = 1/h^2), and the Galerkin coarsening carries it to the
 * coarse levels as part of D (R M P of a diagonal M is the diagonal of the children's means).
 * The nonlinear equation is solved by Newton's method: F(phi) = f - A_eps phi - k2 sinh(phi);
 * stop when ||F|| / ||f|| < tol; else solve (A_eps + k2 cosh(phi)) delta = F (homogeneous walls)
 * to the inner tolerance with the multigrid of that linear operator, phi += delta. */

/* F = f - A_eps phi - k2 sinh(phi) (the nonlinear residual); returns ||F||_2. */
static double pb_residual(const double* phi, const double* f, const var_level* V0, const double* k2, double h,
                          const int* bc, double* F) {
  const size_t n = (size_t)V0->n[0] * V0->n[1] * V0->n[2];
  var_residual(phi, f, F, V0, level_coeff(h, 0), bc);
  for (size_t p = 0; p < n; ++p) F[p] = F[p] - k2[p] * sinh(phi[p]);
  return norm2_d(F, n);
}

/* Newton's method for -div(eps grad phi) + k2 sinh(phi) = f (f with the wall terms, as from
 * ccmg_or_var_rhs); phi is the start value and the result. Each step solves the linearised
 * equation to inner_tol (relative) by V-cycles. Returns the number of Newton steps; the final
 * ||F|| / ||f|| in rel_out. */
int ccmg_or_pb_newton(double* phi, const double* f, const double* eps, const double* k2, int nx, int ny, int nz,
                      double h, const int* bc, int nu1, int nu2, double omega, double tol, int max_newton,
                      double inner_tol, int max_cycles, double* rel_out) {
  const size_t n = (size_t)nx * ny * nz;
  const int d[3] = {nx, ny, nz};
  var_level V0;
  var_alloc(&V0, d);
  var_fine(eps, bc, &V0);
  double* F = (double*)malloc(n * sizeof(double));
  double* kl = (double*)malloc(n * sizeof(double));
  double* delta = (double*)malloc(n * sizeof(double));
  const double fn = norm2_d(f, n);
  int it = 0;
  double rel;
  for (;;) {
    const double Fn = pb_residual(phi, f, &V0, k2, h, bc, F);
    rel = fn > 0.0 ? Fn / fn : Fn;
    if (!(rel >= tol) || it >= max_newton) break;
    for (size_t p = 0; p < n; ++p) {
      kl[p] = k2[p] * cosh(phi[p]);
      delta[p] = 0.0;
    }
    ccmg_or_var_solve(delta, F, eps, kl, nx, ny, nz, h, bc, nu1, nu2, omega, inner_tol, max_cycles, NULL);
    for (size_t p = 0; p < n; ++p) phi[p] = phi[p] + delta[p];
    ++it;
  }
  if (rel_out) *rel_out = rel;
  free(F);
  free(kl);
  free(delta);
  var_free(&V0);
  return it;
}

/* The nonlinear residual F of phi (for checks), written to F_out; returns ||F|| / ||f||. */
double ccmg_or_pb_residual(const double* phi, const double* f, const double* eps, const double* k2, int nx, int ny,
                           int nz, double h, const int* bc, double* F_out) {
  const int d[3] = {nx, ny, nz};
  var_level V0;
  var_alloc(&V0, d);
  var_fine(eps, bc, &V0);
  const double Fn = pb_residual(phi, f, &V0, k2, h, bc, F_out);
  const double fn = norm2_d(f, (size_t)nx * ny * nz);
  var_free(&V0);
  return fn > 0.0 ? Fn / fn : Fn;
}

/* Adjoint of ccmg_or_var_rhs: given lambda = dJ/df, dJ/drho = lambda and dJ/dbc_value[q] = the sum
 * over the face-q cells of lambda * (2 eps / h^2 Dirichlet, eps / h Neumann; periodic: none). */
void ccmg_or_var_rhs_adjoint(const double* lam, const double* eps, double* grho, double* gbc, int nx, int ny, int nz,
                             double h, const int* bc) {
  for (int q = 0; q < 6; ++q) gbc[q] = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t p = idx3(i, j, k, nx, ny);
        grho[p] = lam[p];
        const int on_face[6] = {i == 0, i == nx - 1, j == 0, j == ny - 1, k == 0, k == nz - 1};
        for (int q = 0; q < 6; ++q) {
          if (!on_face[q] || bc[q] == BC_PERIODIC) continue;
          gbc[q] = gbc[q] + lam[p] * (bc[q] == BC_DIRICHLET ? 2.0 * eps[p] / (h * h) : eps[p] / h);
        }
      }
}
