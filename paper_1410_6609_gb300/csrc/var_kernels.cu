// var_kernels.cu -- the solver with a variable permittivity (sm_103a), FP64.
//
// Sec. 3 of the paper: the cell-centred solver extends to discontinuous dielectricity through
// Galerkin coarsening with the averaging restriction and the nearest-neighbour prolongation (after
// Alcouffe et al.). The equation becomes -div(eps grad phi) = rho; the flux through the face of
// two cells has the weight of the harmonic mean of their permittivities, and a wall face the
// weight of its cell's permittivity (Dirichlet: counted twice, ghost 2 g - phi; Neumann: not at
// all, ghost phi + h g; periodic: the face to the cell at the opposite side). Every level stores,
// in its own order (packed colours, or natural order on the coarsest level), four arrays of its
// cell count: the diagonal D and the weights wx, wy, wz of each cell's -x, -y, -z faces, scaled as
// in the constant case (A_l = c_l (D phi - sum w phi_neighbour), c_l = 1/(2^l h^2)). The +x face
// of a cell is the -x face of its +x neighbour, so its weight sits at that neighbour's index:
// the same index as the neighbour's potential. Galerkin coarsening, A_{l+1} = R A_l P with
// R = P^T / 8, keeps this form:
//   w_{l+1}(coarse face) = (1/4) (sum of the 4 fine face weights on it),
//   D_{l+1}(I) = (1/4) (sum of the 8 children's D - 2 (sum of the 12 faces inside I)).
// A reaction term k2 phi (screened and Poisson-Boltzmann operators) adds M = k2 h^2 to the
// level-0 diagonal; the coarse levels carry the diffusion part divided by the coarse-grid
// correction factor omega (the factor of Sec. 3 taken into the operator, so the correction
// itself is not magnified: the same iterates for the Poisson operator) and the reaction part,
// which these transfers coarsen exactly, as its plain Galerkin product (1/4) (sum of the 8
// children's M). D = Dw + M is kept with its parts Dw and M.
// The setup kernels evaluate these in the oracle's order with rounded operations, so the
// coefficients agree bit for bit; the cycle kernels are the FP64 cell-by-cell forms of the
// smoother, the fused residual and restriction, the residual norm and the coarse CG.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "ccmg_internal.cuh"
#include "level_ops.cuh"

namespace ccmg {
namespace {

using ops::block_sum;
using ops::coarse_index;
using ops::nb_has;
using ops::nb_off;

// The coefficient arrays of a level at vc: D, wx, wy, wz, 1/D, Dw and M, each of `n` entries
// (the smoother multiplies by the stored reciprocal: FP64 division is many times slower than a
// multiply on this GPU, and the half-sweep would be bound by it).
constexpr int kVarArrays = 7;
struct VarCoef {
  const double* D;
  const double* wx;
  const double* wy;
  const double* wz;
  const double* invD;
  const double* Dw;
  const double* M;
};
__device__ __forceinline__ VarCoef var_coef(const double* vc, long long n) {
  return VarCoef{vc, vc + n, vc + 2 * n, vc + 3 * n, vc + 4 * n, vc + 5 * n, vc + 6 * n};
}

// The cycle's view of a level's coefficients in precision T (the first five arrays: D, wx, wy,
// wz, 1/D); the single-precision copies (kVarArrays32 arrays) serve the inner cycle of the
// mixed-precision defect correction.
constexpr int kVarArrays32 = 5;
template <typename T>
struct VarW {
  const T* D;
  const T* wx;
  const T* wy;
  const T* wz;
  const T* invD;
};
template <typename T>
__device__ __forceinline__ VarW<T> var_w(const T* vc, long long n) {
  return VarW<T>{vc, vc + n, vc + 2 * n, vc + 3 * n, vc + 4 * n};
}
__device__ __forceinline__ VarW<double> var_w(const VarCoef& W) { return VarW<double>{W.D, W.wx, W.wy, W.wz, W.invD}; }
using ops::fmat;

__device__ __forceinline__ double harmonic(double a, double b) { return __ddiv_rn(__dmul_rn(2.0 * a, b), a + b); }

__device__ __forceinline__ long long natural(const Geom& G, int i, int j, int k) {
  return (long long)i + (long long)G.nx * ((long long)j + (long long)G.ny * k);
}

// Level-0 coefficients from the cell permittivities eps and the reaction coefficients react
// (natural order; react null: none).
__global__ void __launch_bounds__(256) k_var_fine(const double* __restrict__ eps, const double* __restrict__ react,
                                                  double h2, Geom G, FaceBC bc, double* __restrict__ vc, long long n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const int nn[3] = {G.nx, G.ny, G.nz}, pos[3] = {i, j, k};
  const double e = __ldg(eps + natural(G, i, j, k));
  double w[3], D = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int q[3] = {i, j, k};
    const bool per = (G.per >> a) & 1;
    // the -a face
    double wm;
    if (pos[a] > 0 || per) {
      q[a] = pos[a] > 0 ? pos[a] - 1 : nn[a] - 1;
      wm = harmonic(__ldg(eps + natural(G, q[0], q[1], q[2])), e);
    } else {
      wm = e;
    }
    w[a] = wm;
    if (pos[a] > 0 || per) D = __dadd_rn(D, wm);
    else if (bc.type[2 * a] == 0) D = __dadd_rn(D, __dmul_rn(2.0, e));
    // the +a face: the -a face of the next cell (of cell 0 across a periodic axis)
    if (pos[a] < nn[a] - 1 || per) {
      q[a] = pos[a] < nn[a] - 1 ? pos[a] + 1 : 0;
      const double en = __ldg(eps + natural(G, q[0], q[1], q[2]));
      D = __dadd_rn(D, harmonic(e, en));
    } else if (bc.type[2 * a + 1] == 0) {
      D = __dadd_rn(D, __dmul_rn(2.0, e));
    }
  }
  const long long o = coarse_index(G, i, j, k);
  const double M = react ? __dmul_rn(__ldg(react + natural(G, i, j, k)), h2) : 0.0;
  const double Dt = __dadd_rn(D, M);
  vc[o] = Dt;
  vc[n + o] = w[0];
  vc[2 * n + o] = w[1];
  vc[3 * n + o] = w[2];
  vc[4 * n + o] = __ddiv_rn(1.0, Dt);
  vc[5 * n + o] = D;
  vc[6 * n + o] = M;
}

// Coefficients of coarse level Gc from fine level Gf (the oracle's summation order): the Galerkin
// product of the diffusion part divided by omega, that of the reaction part as it is.
__global__ void __launch_bounds__(256) k_var_coarsen(const double* __restrict__ vf, Geom Gf, long long nf,
                                                     double* __restrict__ vcc, Geom Gc, long long nc, double omega) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  const VarCoef F = var_coef(vf, nf);
  auto at = [&](const double* a, int i, int j, int k) { return __ldg(a + coarse_index(Gf, i, j, k)); };
  double sx = 0.0, sy = 0.0, sz = 0.0, sd = 0.0, sm = 0.0, inner = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      sx = __dadd_rn(sx, at(F.wx, 2 * I, 2 * J + u, 2 * K + v));
      sy = __dadd_rn(sy, at(F.wy, 2 * I + u, 2 * J, 2 * K + v));
      sz = __dadd_rn(sz, at(F.wz, 2 * I + u, 2 * J + v, 2 * K));
    }
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        sd = __dadd_rn(sd, at(F.Dw, 2 * I + di, 2 * J + dj, 2 * K + dk));
        sm = __dadd_rn(sm, at(F.M, 2 * I + di, 2 * J + dj, 2 * K + dk));
      }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      inner = __dadd_rn(inner, at(F.wx, 2 * I + 1, 2 * J + u, 2 * K + v));
      inner = __dadd_rn(inner, at(F.wy, 2 * I + u, 2 * J + 1, 2 * K + v));
      inner = __dadd_rn(inner, at(F.wz, 2 * I + u, 2 * J + v, 2 * K + 1));
    }
  const long long o = coarse_index(Gc, I, J, K);
  const double Dw = __ddiv_rn(__ddiv_rn(__dsub_rn(sd, __dmul_rn(2.0, inner)), 4.0), omega);
  const double M = __ddiv_rn(sm, 4.0);
  const double Dc = __dadd_rn(Dw, M);
  vcc[o] = Dc;
  vcc[nc + o] = __ddiv_rn(__ddiv_rn(sx, 4.0), omega);
  vcc[2 * nc + o] = __ddiv_rn(__ddiv_rn(sy, 4.0), omega);
  vcc[3 * nc + o] = __ddiv_rn(__ddiv_rn(sz, 4.0), omega);
  vcc[4 * nc + o] = __ddiv_rn(1.0, Dc);
  vcc[5 * nc + o] = Dw;
  vcc[6 * nc + o] = M;
}


// Weighted neighbour sum of cell m of colour c, row (j, k), on a packed level, in the order
// -x,+x,-y,+y,-z,+z (walls: none; periodic axes wrap). The weight of a + face is read at the
// neighbour's index, where its potential is.
template <typename T>
__device__ __forceinline__ T var_nbsum_packed(const T* __restrict__ x, const VarW<T>& W, const Geom& G, int c, int m,
                                              int j, int k) {
  const int s = (j + k + c) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)c * G.csz + row + m;
  const long long oth = (long long)(1 - c) * G.csz + row;
  const bool px = (G.per & 1) != 0;
  T acc = T(0);
  if (!(m == 0 && s == 0)) acc = fmat(__ldg(W.wx + own), __ldg(x + oth + m + s - 1), acc);
  else if (px) acc = fmat(__ldg(W.wx + own), __ldg(x + oth + G.hx - 1), acc);
  if (!(m == G.hx - 1 && s == 1)) {
    const long long q = oth + m + s;
    acc = fmat(__ldg(W.wx + q), __ldg(x + q), acc);
  } else if (px) {
    acc = fmat(__ldg(W.wx + oth), __ldg(x + oth), acc);
  }
  if (nb_has<0, true>(G, j, k)) acc = fmat(__ldg(W.wy + own), __ldg(x + oth + m + nb_off<0, true>(G, j, k)), acc);
  if (nb_has<1, true>(G, j, k)) {
    const long long q = oth + m + nb_off<1, true>(G, j, k);
    acc = fmat(__ldg(W.wy + q), __ldg(x + q), acc);
  }
  if (nb_has<2, true>(G, j, k)) acc = fmat(__ldg(W.wz + own), __ldg(x + oth + m + nb_off<2, true>(G, j, k)), acc);
  if (nb_has<3, true>(G, j, k)) {
    const long long q = oth + m + nb_off<3, true>(G, j, k);
    acc = fmat(__ldg(W.wz + q), __ldg(x + q), acc);
  }
  return acc;
}

// The same on a natural-order level, values of type V and weights of type C, summed in V.
template <typename V, typename C>
__device__ __forceinline__ V var_nbsum_natural(const V* __restrict__ x, const VarW<C>& W, const Geom& G, int i, int j,
                                               int k) {
  const long long p = natural(G, i, j, k);
  const long long sy = G.nx, sz = (long long)G.nx * G.ny;
  const bool px = (G.per & 1) != 0, py = (G.per & 2) != 0, pz = (G.per & 4) != 0;
  V acc = V(0);
  if (i > 0) acc = fmat(V(W.wx[p]), x[p - 1], acc);
  else if (px) acc = fmat(V(W.wx[p]), x[p + G.nx - 1], acc);
  if (i < G.nx - 1) acc = fmat(V(W.wx[p + 1]), x[p + 1], acc);
  else if (px) acc = fmat(V(W.wx[p - (G.nx - 1)]), x[p - (G.nx - 1)], acc);
  if (j > 0) acc = fmat(V(W.wy[p]), x[p - sy], acc);
  else if (py) acc = fmat(V(W.wy[p]), x[p + (G.ny - 1) * sy], acc);
  if (j < G.ny - 1) acc = fmat(V(W.wy[p + sy]), x[p + sy], acc);
  else if (py) acc = fmat(V(W.wy[p - (G.ny - 1) * sy]), x[p - (G.ny - 1) * sy], acc);
  if (k > 0) acc = fmat(V(W.wz[p]), x[p - sz], acc);
  else if (pz) acc = fmat(V(W.wz[p]), x[p + (G.nz - 1) * sz], acc);
  if (k < G.nz - 1) acc = fmat(V(W.wz[p + sz]), x[p + sz], acc);
  else if (pz) acc = fmat(V(W.wz[p - (G.nz - 1) * sz]), x[p - (G.nz - 1) * sz], acc);
  return acc;
}

// Red-black Gauss-Seidel half-sweep: phi = (g + weighted neighbours) (1/D) for the cells of
// `colour` (ZERO: the iterate is zero, phi = g (1/D)).
template <typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_var_smooth(T* __restrict__ x, const T* __restrict__ g,
                                                    const T* __restrict__ vc, Geom G, int colour) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (m >= G.hx || j >= G.ny) return;
  const VarW<T> W = var_w(vc, 2 * G.csz);
  const long long own = (long long)colour * G.csz + ((long long)k * G.ny + j) * G.hx + m;
  const T S = ZERO ? T(0) : var_nbsum_packed<T>(x, W, G, colour, m, j, k);
  x[own] = (__ldg(g + own) + S) * __ldg(W.invD + own);
}

// The same half-sweep for V consecutive cells m0 .. m0+V-1 of a colour row (rows of whole
// 16-byte vectors): every array is read as one vector per row segment, the x-neighbour beyond the
// segment (and its + face weight) as one scalar, as in the constant-coefficient vector sweep.
// Each cell's sum is formed in var_nbsum_packed's order: identical results.
template <typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_var_smooth_vec(T* __restrict__ x, const T* __restrict__ g,
                                                        const T* __restrict__ vc, Geom G, int colour) {
  constexpr int V = 16 / sizeof(T);
  const int mv = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (mv >= G.hx / V || j >= G.ny) return;
  const int m0 = mv * V;
  const VarW<T> W = var_w(vc, 2 * G.csz);
  const int s = (j + k + colour) & 1;
  const long long row = ((long long)k * G.ny + j) * G.hx;
  const long long own = (long long)colour * G.csz + row + m0;
  const long long oth = (long long)(1 - colour) * G.csz + row;  // the other colour's row
  T gv[V], inv[V], out[V];
  ops::load_vec(g + own, gv);
  ops::load_vec(W.invD + own, inv);
  if (ZERO) {
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = (gv[v] + T(0)) * inv[v];
    ops::store_vec(x + own, out);
    return;
  }
  T wxs[V], wys[V], wzs[V], yc[V], wxo[V];
  ops::load_vec(W.wx + own, wxs);
  ops::load_vec(W.wy + own, wys);
  ops::load_vec(W.wz + own, wzs);
  ops::load_vec(x + oth + m0, yc);
  ops::load_vec(W.wx + oth + m0, wxo);
  // the x-neighbour beyond the segment and, for s = 1, the weight of its face
  const bool px = (G.per & 1) != 0;
  T xe = T(0), we = T(0);
  if (s == 0) {
    if (m0 > 0) xe = __ldg(x + oth + m0 - 1);
    else if (px) xe = __ldg(x + oth + G.hx - 1);
  } else {
    if (m0 + V < G.hx) {
      xe = __ldg(x + oth + m0 + V);
      we = __ldg(W.wx + oth + m0 + V);
    } else if (px) {
      xe = __ldg(x + oth);
      we = __ldg(W.wx + oth);
    }
  }
  const bool hxm = (s == 0) ? (m0 > 0 || px) : true;        // cell m0 has its -x neighbour
  const bool hxp = (s == 1) ? (m0 + V < G.hx || px) : true;  // cell m0+V-1 has its +x neighbour
  T ym[V], yp[V], zm[V], zp[V], wyp[V], wzp[V];
  const bool hym = nb_has<0, true>(G, j, k), hyp = nb_has<1, true>(G, j, k);
  const bool hzm = nb_has<2, true>(G, j, k), hzp = nb_has<3, true>(G, j, k);
  if (hym) ops::load_vec(x + oth + m0 + nb_off<0, true>(G, j, k), ym);
  if (hyp) {
    ops::load_vec(x + oth + m0 + nb_off<1, true>(G, j, k), yp);
    ops::load_vec(W.wy + oth + m0 + nb_off<1, true>(G, j, k), wyp);
  }
  if (hzm) ops::load_vec(x + oth + m0 + nb_off<2, true>(G, j, k), zm);
  if (hzp) {
    ops::load_vec(x + oth + m0 + nb_off<3, true>(G, j, k), zp);
    ops::load_vec(W.wz + oth + m0 + nb_off<3, true>(G, j, k), wzp);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    T acc = T(0);
    if (s == 0) {  // -x neighbour at m-1 (segment or xe), +x neighbour at m with its weight wxo[v]
      if (v > 0) acc = fmat(wxs[v], yc[v - 1], acc);
      else if (hxm) acc = fmat(wxs[v], xe, acc);
      acc = fmat(wxo[v], yc[v], acc);
    } else {  // -x neighbour at m, +x neighbour at m+1 with the weight of that cell's face
      acc = fmat(wxs[v], yc[v], acc);
      if (v < V - 1) acc = fmat(wxo[v + 1], yc[v + 1], acc);
      else if (hxp) acc = fmat(we, xe, acc);
    }
    if (hym) acc = fmat(wys[v], ym[v], acc);
    if (hyp) acc = fmat(wyp[v], yp[v], acc);
    if (hzm) acc = fmat(wzs[v], zm[v], acc);
    if (hzp) acc = fmat(wzp[v], zp[v], acc);
    out[v] = (gv[v] + acc) * inv[v];
  }
  ops::store_vec(x + own, out);
}

// Fused residual and averaging restriction: gc(I,J,K) = (1/4) sum of the 8 children's scaled
// residuals g + sum w phi - D phi, in the order (dk, dj, di).
template <typename T>
__global__ void __launch_bounds__(256) k_var_resid_restrict(const T* __restrict__ x, const T* __restrict__ g,
                                                            const T* __restrict__ vc, Geom G, T* __restrict__ gc,
                                                            Geom Gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Gc.nx || J >= Gc.ny) return;
  const VarW<T> W = var_w(vc, 2 * G.csz);
  T acc = T(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int j = 2 * J + dj, k = 2 * K + dk;
        const int c = (di + dj + dk) & 1;
        const long long own = (long long)c * G.csz + ((long long)k * G.ny + j) * G.hx + I;
        const T S = var_nbsum_packed<T>(x, W, G, c, I, j, k);
        acc = acc + fmat(-__ldg(W.D + own), __ldg(x + own), __ldg(g + own) + S);
      }
  gc[coarse_index(Gc, I, J, K)] = acc * T(0.25);
}

// The fused residual and restriction for V consecutive coarse cells I0 = V iv .. I0+V-1 of coarse
// row (J, K) (fine rows of whole vectors): their children in fine row (j, k) are entries I0.. of both
// colour arrays, so every array is read as one vector per row segment (the x-neighbours beyond
// the segment as scalars); each child's residual is formed in var_nbsum_packed's order and the
// 8 summed in the order (dk, dj, di) of k_var_resid_restrict: identical results.
template <typename T>
__global__ void __launch_bounds__(256) k_var_resid_restrict_vec(const T* __restrict__ x, const T* __restrict__ g,
                                                                const T* __restrict__ vc, Geom G,
                                                                T* __restrict__ gc, Geom Gc) {
  constexpr int V = 16 / sizeof(T);
  const int iv = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (iv >= Gc.nx / V || J >= Gc.ny) return;
  const int I0 = iv * V;
  const VarW<T> W = var_w(vc, 2 * G.csz);
  const bool px = (G.per & 1) != 0;
  T acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = T(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const int j = 2 * J + dj, k = 2 * K + dk;
      const long long row = ((long long)k * G.ny + j) * G.hx;
      const int c0 = (dj + dk) & 1, c1 = c0 ^ 1;  // colours of the children di = 0 (s = 0) and di = 1 (s = 1)
      const long long r0 = (long long)c0 * G.csz + row, r1 = (long long)c1 * G.csz + row;
      T x0[V], x1[V], g0[V], g1[V], D0[V], D1[V], wx0[V], wx1[V], wy0[V], wy1[V], wz0[V], wz1[V];
      ops::load_vec(x + r0 + I0, x0);
      ops::load_vec(x + r1 + I0, x1);
      ops::load_vec(g + r0 + I0, g0);
      ops::load_vec(g + r1 + I0, g1);
      ops::load_vec(W.D + r0 + I0, D0);
      ops::load_vec(W.D + r1 + I0, D1);
      ops::load_vec(W.wx + r0 + I0, wx0);
      ops::load_vec(W.wx + r1 + I0, wx1);
      ops::load_vec(W.wy + r0 + I0, wy0);
      ops::load_vec(W.wy + r1 + I0, wy1);
      ops::load_vec(W.wz + r0 + I0, wz0);
      ops::load_vec(W.wz + r1 + I0, wz1);
      // x-neighbours beyond the segment: cell 2 I0 - 1 (colour c1, index I0 - 1) and cell 2 (I0+V)
      // (colour c0, index I0 + V) with the weight of its face
      T left = T(0), right = T(0), wright = T(0);
      const bool hl = I0 > 0 || px, hr = I0 + V < G.hx || px;
      if (I0 > 0) left = __ldg(x + r1 + I0 - 1);
      else if (px) left = __ldg(x + r1 + G.hx - 1);
      if (I0 + V < G.hx) {
        right = __ldg(x + r0 + I0 + V);
        wright = __ldg(W.wx + r0 + I0 + V);
      } else if (px) {
        right = __ldg(x + r0);
        wright = __ldg(W.wx + r0);
      }
      const bool hym = nb_has<0, true>(G, j, k), hyp = nb_has<1, true>(G, j, k);
      const bool hzm = nb_has<2, true>(G, j, k), hzp = nb_has<3, true>(G, j, k);
      // neighbour rows of both colours (child di = 0 reads colour c1's, di = 1 colour c0's), and
      // the + face weights stored there
      T ym0[V], ym1[V], yp0[V], yp1[V], zm0[V], zm1[V], zp0[V], zp1[V], wyp0[V], wyp1[V], wzp0[V], wzp1[V];
      if (hym) {
        const long long o = nb_off<0, true>(G, j, k);
        ops::load_vec(x + r0 + I0 + o, ym0);
        ops::load_vec(x + r1 + I0 + o, ym1);
      }
      if (hyp) {
        const long long o = nb_off<1, true>(G, j, k);
        ops::load_vec(x + r0 + I0 + o, yp0);
        ops::load_vec(x + r1 + I0 + o, yp1);
        ops::load_vec(W.wy + r0 + I0 + o, wyp0);
        ops::load_vec(W.wy + r1 + I0 + o, wyp1);
      }
      if (hzm) {
        const long long o = nb_off<2, true>(G, j, k);
        ops::load_vec(x + r0 + I0 + o, zm0);
        ops::load_vec(x + r1 + I0 + o, zm1);
      }
      if (hzp) {
        const long long o = nb_off<3, true>(G, j, k);
        ops::load_vec(x + r0 + I0 + o, zp0);
        ops::load_vec(x + r1 + I0 + o, zp1);
        ops::load_vec(W.wz + r0 + I0 + o, wzp0);
        ops::load_vec(W.wz + r1 + I0 + o, wzp1);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        // child di = 0 (colour c0, s = 0): -x at index m-1 of c1, +x at index m of c1
        T S = T(0);
        if (v > 0) S = fmat(wx0[v], x1[v - 1], S);
        else if (hl) S = fmat(wx0[v], left, S);
        S = fmat(wx1[v], x1[v], S);
        if (hym) S = fmat(wy0[v], ym1[v], S);
        if (hyp) S = fmat(wyp1[v], yp1[v], S);
        if (hzm) S = fmat(wz0[v], zm1[v], S);
        if (hzp) S = fmat(wzp1[v], zp1[v], S);
        acc[v] = acc[v] + fmat(-D0[v], x0[v], g0[v] + S);
        // child di = 1 (colour c1, s = 1): -x at index m of c0, +x at index m+1 of c0
        S = T(0);
        S = fmat(wx1[v], x0[v], S);
        if (v < V - 1) S = fmat(wx0[v + 1], x0[v + 1], S);
        else if (hr) S = fmat(wright, right, S);
        if (hym) S = fmat(wy1[v], ym0[v], S);
        if (hyp) S = fmat(wyp0[v], yp0[v], S);
        if (hzm) S = fmat(wz1[v], zm0[v], S);
        if (hzp) S = fmat(wzp0[v], zp0[v], S);
        acc[v] = acc[v] + fmat(-D1[v], x1[v], g1[v] + S);
      }
    }
#pragma unroll
  for (int v = 0; v < V; ++v) gc[coarse_index(Gc, I0 + v, J, K)] = acc[v] * T(0.25);
}

// Scaled residual of every cell with per-block partial sums of its square; MODE 1: also the
// residual field r = r~ c0 in natural order; MODE 2: also float(r~ isc) in the level's order (the
// right-hand side of the single-precision inner cycle, by exponent arithmetic when isc is a power
// of two).
template <int MODE>
__global__ void __launch_bounds__(256) k_var_resid_norm(const double* __restrict__ x, const double* __restrict__ g,
                                                        const double* __restrict__ vc, Geom G, double c0,
                                                        double* __restrict__ partials, double* __restrict__ outn,
                                                        float* __restrict__ outp, const double* __restrict__ inv_scale) {
  __shared__ double red[33];
  const VarW<double> W = var_w(vc, G.packed ? 2 * G.csz : G.csz);
  const long long n = G.packed ? 2 * G.csz : G.csz;
  const double isc = MODE == 2 ? inv_scale[0] : 0.0;
  const int p2 = MODE == 2 ? ops::pow2_exponent(isc) : ops::kBadPow2;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double rd;
    long long nat;
    if (G.packed) {
      const int c = (int)(t / G.csz);
      const long long r = t - (long long)c * G.csz;
      const int m = (int)(r % G.hx);
      const long long rw = r / G.hx;
      const int j = (int)(rw % G.ny), k = (int)(rw / G.ny);
      const double S = var_nbsum_packed<double>(x, W, G, c, m, j, k);
      rd = fma(-__ldg(W.D + t), __ldg(x + t), __ldg(g + t) + S);
      nat = (long long)(2 * m + ((j + k + c) & 1)) + (long long)G.nx * ((long long)j + (long long)G.ny * k);
    } else {
      const int i = (int)(t % G.nx), j = (int)((t / G.nx) % G.ny), k = (int)(t / ((long long)G.nx * G.ny));
      const double S = var_nbsum_natural<double, double>(x, W, G, i, j, k);
      rd = fma(-W.D[t], x[t], g[t] + S);
      nat = t;
    }
    acc = fma(rd, rd, acc);
    if (MODE == 1) outn[nat] = rd * c0;
    if (MODE == 2) outp[t] = p2 != ops::kBadPow2 ? ops::f32_of_scaled(rd, p2) : (float)(rd * isc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Unpreconditioned CG on the coarsest (natural-order) level with the weighted operator, one CTA,
// in double whatever T (the level's precision), vectors in shared memory (4 n doubles); stops at
// ||r|| <= rtol ||b|| or maxit iterations.
template <typename T>
__global__ void __launch_bounds__(256) k_var_coarse_cg(T* __restrict__ xo, const T* __restrict__ bi,
                                                       const T* __restrict__ vc, Geom G, double rtol, int maxit,
                                                       int* iters) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const int n = G.nx * G.ny * G.nz;
  const VarW<T> W = var_w(vc, n);
  double* x = sm;
  double* r = x + n;
  double* p = r + n;
  double* ap = p + n;
  double loc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double b = (double)bi[i];
    x[i] = 0.0;
    r[i] = b;
    p[i] = b;
    loc += b * b;
  }
  double rr = block_sum(loc, red);
  const double bnorm = sqrt(rr);
  int it = 0;
  if (bnorm > 0.0) {
    while (it < maxit) {
      loc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ix = i % G.nx, iy = (i / G.nx) % G.ny, iz = i / (G.nx * G.ny);
        const double a = (double)W.D[i] * p[i] - var_nbsum_natural<double, T>(p, W, G, ix, iy, iz);
        ap[i] = a;
        loc += p[i] * a;
      }
      const double pap = block_sum(loc, red);
      const double alpha = rr / pap;
      loc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x[i] = x[i] + alpha * p[i];
        const double ri = r[i] - alpha * ap[i];
        r[i] = ri;
        loc += ri * ri;
      }
      const double rrn = block_sum(loc, red);
      ++it;
      if (sqrt(rrn) <= rtol * bnorm) break;
      const double beta = rrn / rr;
      for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = r[i] + beta * p[i];
      __syncthreads();
      rr = rrn;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xo[i] = (T)x[i];
  if (threadIdx.x == 0 && iters) *iters = it;
}

// Single-precision copies of the cycle's coefficient arrays of one level.
__global__ void __launch_bounds__(256) k_var_to_f32(const double* __restrict__ vc, float* __restrict__ v32,
                                                   long long n) {
  const long long total = (long long)kVarArrays32 * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    v32[t] = (float)vc[t];
}

// Right-hand side of -div(eps grad phi) = rho, scaled g = f h^2: f = rho, Dirichlet face cells
// += 2 eps g / h^2, Neumann face cells += eps g / h (the oracle's operations and face order).
__global__ void __launch_bounds__(256) k_var_set_rhs(double* __restrict__ gout, Geom G,
                                                     const double* __restrict__ rho,
                                                     const double* __restrict__ eps, double h, FaceBC bc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= G.nx || j >= G.ny) return;
  const long long p = natural(G, i, j, k);
  double v = rho[p];
  const bool on[6] = {i == 0, i == G.nx - 1, j == 0, j == G.ny - 1, k == 0, k == G.nz - 1};
  const double e = eps[p];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!on[q] || bc.type[q] == 2) continue;
    const double gv = face_value(bc, q, i, j, k, G.nx, G.ny);
    v = bc.type[q] == 0 ? __dadd_rn(v, __ddiv_rn(__dmul_rn(__dmul_rn(2.0, e), gv), __dmul_rn(h, h)))
                        : __dadd_rn(v, __ddiv_rn(__dmul_rn(e, gv), h));
  }
  gout[coarse_index(G, i, j, k)] = __dmul_rn(v, __dmul_rn(h, h));
}

// Newton step of the Poisson-Boltzmann equation on the (packed) finest level: the scaled
// nonlinear residual F~ = g0 + sum w phi - Dw phi - k2 h^2 sinh(phi) into f (the right-hand side
// of the correction equation), partial sums of F~^2, and the linearised diagonal
// M = k2 h^2 cosh(phi), D = Dw + M, 1/D for the next coarsening.
__global__ void __launch_bounds__(256) k_pb_update(const double* __restrict__ x, const double* __restrict__ g0,
                                                   double* __restrict__ vc, Geom G, const double* __restrict__ k2,
                                                   double h2, double* __restrict__ f,
                                                   double* __restrict__ partials) {
  __shared__ double red[33];
  const long long n = 2 * G.csz;
  const VarCoef W = var_coef(vc, n);
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / G.csz);
    const long long r = t - (long long)c * G.csz;
    const int m = (int)(r % G.hx);
    const long long rw = r / G.hx;
    const int j = (int)(rw % G.ny), k = (int)(rw / G.ny);
    const long long nat = (long long)(2 * m + ((j + k + c) & 1)) + (long long)G.nx * ((long long)j + (long long)G.ny * k);
    const double S = var_nbsum_packed<double>(x, var_w(W), G, c, m, j, k);
    const double p = x[t];
    const double kh = __dmul_rn(__ldg(k2 + nat), h2);
    const double F = fma(-kh, sinh(p), fma(-W.Dw[t], p, g0[t] + S));
    f[t] = F;
    acc = fma(F, F, acc);
    const double M = __dmul_rn(kh, cosh(p));
    const double D = __dadd_rn(W.Dw[t], M);
    vc[6 * n + t] = M;
    vc[t] = D;
    vc[4 * n + t] = __ddiv_rn(1.0, D);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) k_axpy(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = y[t] + x[t];
}

__global__ void __launch_bounds__(256) k_fill(double* __restrict__ y, double v, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = v;
}

void shape2(int nx, int ny, int nz, dim3& b, dim3& g) {
  const int bx = nx >= 64 ? 64 : (nx >= 32 ? 32 : 16);
  b = dim3(bx, 256 / bx, 1);
  g = dim3((nx + bx - 1) / bx, (ny + b.y - 1) / b.y, nz);
}

}  // namespace

long long var_cells(const Geom& G) { return G.packed ? 2 * G.csz : G.csz; }

int var_arrays() { return kVarArrays; }

cudaError_t launch_var_coarsen_all(const Geom* geo, int L, double* const* vc, double omega, cudaStream_t s) {
  dim3 b, g;
  for (int l = 1; l < L; ++l) {
    shape2(geo[l].nx, geo[l].ny, geo[l].nz, b, g);
    k_var_coarsen<<<g, b, 0, s>>>(vc[l - 1], geo[l - 1], var_cells(geo[l - 1]), vc[l], geo[l], var_cells(geo[l]),
                                  omega);
  }
  return cudaGetLastError();
}

cudaError_t launch_var_setup(const double* eps, const double* react, double h, double omega, const Geom* geo, int L,
                             const FaceBC& bc, double* const* vc, cudaStream_t s) {
  dim3 b, g;
  shape2(geo[0].nx, geo[0].ny, geo[0].nz, b, g);
  k_var_fine<<<g, b, 0, s>>>(eps, react, h * h, geo[0], bc, vc[0], var_cells(geo[0]));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_var_coarsen_all(geo, L, vc, omega, s);
}

cudaError_t launch_pb_update(const double* x, const double* g0, double* vc, const Geom& G, const double* k2, double h,
                             double* f, double* partials, int* nparts, cudaStream_t s) {
  const long long n = var_cells(G);
  long long blocks = (n + 255) / 256;
  if (blocks > kMaxPartials) blocks = kMaxPartials;
  k_pb_update<<<(int)blocks, 256, 0, s>>>(x, g0, vc, G, k2, h * h, f, partials);
  *nparts = (int)blocks;
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t s) {
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  k_axpy<<<(int)blocks, 256, 0, s>>>(y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* y, double v, long long n, cudaStream_t s) {
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  k_fill<<<(int)blocks, 256, 0, s>>>(y, v, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_var_smooth(T* x, const T* g, const T* vc, const Geom& G, int colour, bool zero, cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  dim3 b, gr;
  // single precision: the vector sweep (HBM-bound); double: the per-cell sweep, which the FP64
  // pipe bounds either way and which keeps more warps resident (measured 1.08 vs 1.17 ms at 512^3).
  // CCMG_VAR_SWEEP=cell keeps the per-cell sweep everywhere (for comparing the two).
  static const bool cell_only = [] {
    const char* e = std::getenv("CCMG_VAR_SWEEP");
    return e && std::strcmp(e, "cell") == 0;
  }();
  if (sizeof(T) == 4 && G.hx % V == 0 && !cell_only) {
    const int nvec = G.hx / V;
    int bx = 1;
    while (bx < nvec && bx < 128) bx *= 2;
    b = dim3(bx, 256 / bx, 1);
    gr = dim3((nvec + bx - 1) / bx, (G.ny + b.y - 1) / b.y, G.nz);
    if (zero) k_var_smooth_vec<T, true><<<gr, b, 0, s>>>(x, g, vc, G, colour);
    else k_var_smooth_vec<T, false><<<gr, b, 0, s>>>(x, g, vc, G, colour);
    return cudaGetLastError();
  }
  shape2(G.hx, G.ny, G.nz, b, gr);
  if (zero) k_var_smooth<T, true><<<gr, b, 0, s>>>(x, g, vc, G, colour);
  else k_var_smooth<T, false><<<gr, b, 0, s>>>(x, g, vc, G, colour);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_var_resid_restrict(const T* x, const T* g, const T* vc, const Geom& G, T* gc, const Geom& Gc,
                                      cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  dim3 b, gr;
  static const bool cell_only = [] {
    const char* e = std::getenv("CCMG_VAR_SWEEP");
    return e && std::strcmp(e, "cell") == 0;
  }();
  if (sizeof(T) == 4 && G.hx % V == 0 && !cell_only) {  // single precision: the vector form
    const int nvec = Gc.nx / V;
    int bx = 1;
    while (bx < nvec && bx < 64) bx *= 2;
    b = dim3(bx, 256 / bx, 1);
    gr = dim3((nvec + bx - 1) / bx, (Gc.ny + b.y - 1) / b.y, Gc.nz);
    k_var_resid_restrict_vec<T><<<gr, b, 0, s>>>(x, g, vc, G, gc, Gc);
    return cudaGetLastError();
  }
  shape2(Gc.nx, Gc.ny, Gc.nz, b, gr);
  k_var_resid_restrict<T><<<gr, b, 0, s>>>(x, g, vc, G, gc, Gc);
  return cudaGetLastError();
}

cudaError_t launch_var_resid_norm(const double* x, const double* g, const double* vc, const Geom& G, double c0,
                                  double* partials, int* nparts, int mode, double* out_natural, float* out_packed,
                                  const double* inv_scale, cudaStream_t s) {
  const long long n = var_cells(G);
  long long blocks = (n + 255) / 256;
  if (blocks > kMaxPartials) blocks = kMaxPartials;
  if (mode == 1) k_var_resid_norm<1><<<(int)blocks, 256, 0, s>>>(x, g, vc, G, c0, partials, out_natural, nullptr, nullptr);
  else if (mode == 2)
    k_var_resid_norm<2><<<(int)blocks, 256, 0, s>>>(x, g, vc, G, c0, partials, nullptr, out_packed, inv_scale);
  else k_var_resid_norm<0><<<(int)blocks, 256, 0, s>>>(x, g, vc, G, c0, partials, nullptr, nullptr, nullptr);
  *nparts = (int)blocks;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_var_coarse_cg(T* x, const T* b, const T* vc, const Geom& Gc, double rtol, int maxit, int* d_iters,
                                 cudaStream_t s) {
  const int n = Gc.nx * Gc.ny * Gc.nz;
  int threads = ((n + 31) / 32) * 32;
  if (threads > 256) threads = 256;
  const size_t smem = (size_t)4 * n * sizeof(double);
  k_var_coarse_cg<T><<<1, threads, smem, s>>>(x, b, vc, Gc, rtol, maxit, d_iters);
  return cudaGetLastError();
}

cudaError_t prepare_var_coarse_cg() {
  const int bytes = (int)(4 * kMaxCoarseCells * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_var_coarse_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_var_coarse_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int var_arrays32() { return kVarArrays32; }

cudaError_t launch_var_to_f32(const double* const* vc, float* const* v32, const Geom* geo, int L, cudaStream_t s) {
  for (int l = 0; l < L; ++l) {
    const long long n = var_cells(geo[l]);
    const long long blocks = std::min<long long>((kVarArrays32 * n + 255) / 256, 152LL * 16);
    k_var_to_f32<<<(int)blocks, 256, 0, s>>>(vc[l], v32[l], n);
  }
  return cudaGetLastError();
}

template cudaError_t launch_var_smooth<double>(double*, const double*, const double*, const Geom&, int, bool,
                                               cudaStream_t);
template cudaError_t launch_var_smooth<float>(float*, const float*, const float*, const Geom&, int, bool, cudaStream_t);
template cudaError_t launch_var_resid_restrict<double>(const double*, const double*, const double*, const Geom&,
                                                       double*, const Geom&, cudaStream_t);
template cudaError_t launch_var_resid_restrict<float>(const float*, const float*, const float*, const Geom&, float*,
                                                      const Geom&, cudaStream_t);
template cudaError_t launch_var_coarse_cg<double>(double*, const double*, const double*, const Geom&, double, int, int*,
                                                  cudaStream_t);
template cudaError_t launch_var_coarse_cg<float>(float*, const float*, const float*, const Geom&, double, int, int*,
                                                 cudaStream_t);

cudaError_t launch_var_set_rhs(double* g, const Geom& G, const double* rho, const double* eps, double h,
                               const FaceBC& bc, cudaStream_t s) {
  dim3 b, gr;
  shape2(G.nx, G.ny, G.nz, b, gr);
  k_var_set_rhs<<<gr, b, 0, s>>>(g, G, rho, eps, h, bc);
  return cudaGetLastError();
}

}  // namespace ccmg
