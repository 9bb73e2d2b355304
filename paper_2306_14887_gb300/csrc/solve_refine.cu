// Refined truncation solve (TN_SOLVE_REFINED): FP64 result from an FP32 start.
//
// The truncated SVD of the bond matrix K = R_v R_w^T (Methods, "The simple
// update procedure") is taken as the eigen-decomposition
// H = K K^H = R_v conj(G_w) R_v^H = U diag(sigma^2) U^H, where G_v = R_v^H R_v
// and G_w are the Gram matrices of the gate-split environment-weighted site
// matrices, built from the open-p environments N_p of both sides.  The gate is
// split on the projectors of v's physical index as in solve32.cu, which makes
// G_v block diagonal.  Phases:
//
//   1. chol64_kernel: FP64 pivoted Cholesky of the two chi x chi blocks of G_v,
//      P^T G_b P = L_b L_b^H, so that R_b = L_b^H P^T.
//   2. solve32_kernel in basis mode: the same R_v rounded to FP32, the FP32
//      Cholesky of G_w, K^T = R_w R_v^T and the one-sided Jacobi of K in FP32
//      shared memory.  It yields only a starting basis: the columns of K J
//      normalised (U_0, n x n, by decreasing sigma, the columns below
//      1e-3 sigma_1 re-orthonormalised in FP32) and sigma^2.
//   3. refine_kernel: one Newton step in FP64 for the kept chi columns, the
//      refinement of Ogita and Aishima ("Iterative refinement for symmetric
//      eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018), in
//      the basis U_A of the active columns of U_0 (sigma above 1e-6 sigma_1):
//        P = H U_k,  S = U_A^H P,  R = I - U_A^H U_k               (FP64)
//        lambda_j = S_jj / (1 - R_jj)
//        E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)  for i != j,
//               R_ij / 2 when the pair is not separated; E_jj = R_jj / 2
//        u_j' = u_j + U_A E_Aj + (I - P_A) P_j / lambda_j
//      The last term is the Newton correction toward the complement of
//      span(U_A), on which H is about zero; to first order it is
//      P_j / lambda_j - U_A (S_Aj / lambda_j + R_Aj).  The step converges
//      quadratically: a start orthogonal to about 1e-6 leaves an error of
//      order (1e-6 / relative gap)^2.  It is taken for the head columns
//      (sigma >= 1e-3 sigma_1).  Below that the FP32 start is limited by the
//      FP32 Gram inputs themselves, and the Rayleigh quotients of the squared
//      problem are dominated by the head's rounding, so tail columns keep
//      their start's eigenvalues and take only the corrections that keep
//      them orthogonal to the head (E_ij = R_ij - conj(E_ji)) and to each
//      other (R_ij / 2).
//   4. legs_kernel: FP64 leg matrices from the refined basis,
//      C_v = R_v^+ U_k sqrt(S) by triangular solves and
//      C_w = R_v^T conj(U_k) / sqrt(sigma ||sigma||); the outputs D_v[p] and
//      D_w[q] (FP32 planar), the spectrum S = sigma / ||sigma|| in decreasing
//      order, and both gate-edge messages diag(S).
//
// Only phase 2 computes in FP32.  The quantities the outputs are computed from
// (R_v, H U, the Rayleigh quotients, the corrected eigenvectors and the leg
// matrices) are FP64.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tnbp.h"

namespace tnbp {
namespace {

struct cd {
  double x, y;
};
__device__ __forceinline__ cd cz() { return {0.0, 0.0}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.x, -a.y}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cd cmul(cd a, cd b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// acc += a * b
__device__ __forceinline__ void cfma(cd& acc, cd a, cd b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cd shfl_xor(cd v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kJG = 8;              // output columns accumulated together per warp row
constexpr int kJU = 4;              // output columns per thread in the basis update
constexpr int kSmemChi = 64;   // up to here the FP32 basis and the FP64 Cholesky run in
                               // shared memory; above, in the edge's global workspace
constexpr int kMaxChi = 256;
constexpr int kSmemBudget = 200 * 1024;
// Head columns, sigma >= 1e-3 sigma_1: the FP32 start is accurate enough there
// for one Newton step to reach FP64 accuracy.  Below, the start is limited by
// the FP32 Gram inputs themselves (their rounding puts an absolute floor of
// about sqrt(eps_32) sigma_1 under the singular values), and the Rayleigh
// quotient of the squared problem H would be dominated by the head's
// rounding, so tail columns keep their start's values and are only kept
// orthogonal.
constexpr double kHead = 1e-6;
// Separation test of a pair: the start's eigenvalue lambda_0[i] carries the
// FP32 rounding of its column, about kNoise sqrt(lambda_0[0] lambda_0[i])
// (a few FP32 ulps of sigma_1 times sigma_i, with a margin).  A pair whose gap
// is not clearly above that, or whose Newton correction would exceed 1/4, is
// treated as degenerate: only kept orthogonal (R_ij / 2).  Rotations inside
// the kept set are a gauge freedom of the two-site matrix, so leaving such a
// pair unrotated changes no contraction of the state.
constexpr double kNoise = 2e-6;

// ------------------------------------------------------------ FP64 Cholesky
// Pivoted Cholesky of the Hermitian PSD m x m matrix A (row stride ld, both
// triangles stored) in place by the whole block: afterwards the first `rank`
// columns of the lower triangle hold L with P^T A P = L L^H, perm[t] is the
// original index of pivot t, and everything else is zero.  A pivot at or below
// rel_tol * (largest initial diagonal) ends the factorisation.
__device__ void pivoted_cholesky64(cd* A, int m, int ld, int* perm, double rel_tol, int* rank_out,
                                   int* piv_s, double* pv_s, double* d0_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < m; i += blockDim.x) perm[i] = i;
  __syncthreads();
  int r = m;
  for (int k = 0; k < m; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int i = k + lane; i < m; i += 32) {
        const double d = A[i * ld + i].x;
        if (d > best) { best = d; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        *pv_s = best;
        *piv_s = bi;
        if (k == 0) *d0_s = best > 0.0 ? best : 0.0;
      }
    }
    __syncthreads();
    const double pv = *pv_s;
    const int piv = *piv_s;
    const double d0 = *d0_s;
    if (!(d0 > 0.0) || !(pv > rel_tol * d0)) { r = k; break; }
    if (piv != k) {
      // symmetric exchange of rows and columns k and piv (the 2 x 2 block of
      // the two indices by one thread afterwards)
      for (int j = tid; j < m; j += blockDim.x) {
        if (j == k || j == piv) continue;
        const cd t = A[k * ld + j];
        A[k * ld + j] = A[piv * ld + j];
        A[piv * ld + j] = t;
        const cd u = A[j * ld + k];
        A[j * ld + k] = A[j * ld + piv];
        A[j * ld + piv] = u;
      }
      __syncthreads();
      if (tid == 0) {
        const cd kk = A[k * ld + k], pp = A[piv * ld + piv];
        const cd kp = A[k * ld + piv], pk = A[piv * ld + k];
        A[k * ld + k] = pp;
        A[piv * ld + piv] = kk;
        A[k * ld + piv] = pk;
        A[piv * ld + k] = kp;
        const int t = perm[k];
        perm[k] = perm[piv];
        perm[piv] = t;
      }
      __syncthreads();
    }
    const double d = sqrt(A[k * ld + k].x);
    const double inv = 1.0 / d;
    for (int i = k + 1 + tid; i < m; i += blockDim.x) A[i * ld + k] = cscale(A[i * ld + k], inv);
    __syncthreads();
    if (tid == 0) A[k * ld + k] = {d, 0.0};
    // trailing update of the full Hermitian block: A[i][j] -= l_i conj(l_j)
    const int rem = m - k - 1;
    for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
      const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      const cd li = A[i * ld + k], lj = A[j * ld + k];
      cd v = A[i * ld + j];
      v.x = fma(-li.x, lj.x, v.x);
      v.x = fma(-li.y, lj.y, v.x);
      v.y = fma(-li.y, lj.x, v.y);
      v.y = fma(li.x, lj.y, v.y);
      A[i * ld + j] = v;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    if (j > i || j >= r) A[i * ld + j] = cz();
  }
  if (tid == 0) *rank_out = r;
  __syncthreads();
}

// Block b = blockIdx.x of edge blockIdx.y: G_b = conj(N_b^v) -> L_b, perm_b, rank_b.
__global__ void __launch_bounds__(kThreads) chol64_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int piv_s, rank_s;
  __shared__ double pv_s, d0_s;
  const int b = blockIdx.x, edge = blockIdx.y, chi = a.chi;
  const int64_t c2 = (int64_t)chi * chi;
  const float* g = a.gram + (int64_t)edge * 8 * c2 + (int64_t)b * 2 * c2;
  const RefineLayout lay = refine_layout(chi);
  double* base = a.work + (int64_t)edge * lay.stride;
  int* ints = reinterpret_cast<int*>(base + lay.ints);
  // the factorisation runs in shared memory (padded rows) up to kSmemChi and in
  // place in the edge's L block of the workspace above
  // the basis kernel that follows may start (its first phase does not read
  // these factors; it waits for this grid before it does)
  cudaTriggerProgrammaticLaunchCompletion();
  const bool in_smem = chi <= kSmemChi;
  const int ld = in_smem ? chi + 1 : chi;
  cd* A = in_smem ? reinterpret_cast<cd*>(smem_raw)
                  : reinterpret_cast<cd*>(base + lay.L) + (int64_t)b * c2;
  for (int idx = threadIdx.x; idx < chi * chi; idx += blockDim.x) {
    const int i = idx / chi, j = idx - i * chi;
    A[i * ld + j] = {(double)g[idx], -(double)g[c2 + idx]};
  }
  __syncthreads();
  pivoted_cholesky64(A, chi, ld, ints + b * chi, a.gram_cut, &rank_s, &piv_s, &pv_s, &d0_s);
  cd* L = reinterpret_cast<cd*>(base + lay.L) + (int64_t)b * c2;
  if (in_smem)
    for (int idx = threadIdx.x; idx < chi * chi; idx += blockDim.x) {
      const int i = idx / chi, j = idx - i * chi;
      L[idx] = A[i * ld + j];
    }
  if (threadIdx.x == 0) ints[2 * chi + b] = rank_s;
}

// ------------------------------------------------------------ refinement
struct EdgeView {
  int chi, n, act;
  const cd* L;         // [2][chi][chi] lower triangular
  const int* perm;     // [2][chi]
  const int* rank;     // [2]
  const cd* U;         // [n][n]: column m at U + n m
  cd* U1;              // [chi][n]: refined kept columns
  const double* lam0;  // [n]
  double* lam1;        // [chi]
  const double* misc;  // [0] sum of sigma^2 of the start
  const float* gw;     // [q][re|im][chi][chi] the open-q environments N_q^w (FP32 inputs)
};

__device__ EdgeView edge_view(const SolveArgs& a, int edge) {
  const RefineLayout lay = refine_layout(a.chi);
  double* base = a.work + (int64_t)edge * lay.stride;
  EdgeView v;
  v.chi = a.chi;
  v.n = 2 * a.chi;
  const int* ints = reinterpret_cast<const int*>(base + lay.ints);
  v.perm = ints;
  v.rank = ints + 2 * a.chi;
  v.act = ints[2 * a.chi + 2];
  v.L = reinterpret_cast<const cd*>(base + lay.L);
  v.U = reinterpret_cast<const cd*>(base + lay.U);
  v.U1 = reinterpret_cast<cd*>(base + lay.U1);
  v.lam0 = base + lay.lam0;
  v.lam1 = base + lay.lam1;
  v.misc = base + lay.misc;
  v.gw = a.gram + (int64_t)edge * 8 * (int64_t)a.chi * a.chi + 4 * (int64_t)a.chi * a.chi;
  return v;
}

// out(i, j) = sum_{r in [lo(i), hi(i))} arow(i, r) * B[j * ldb + bidx(i, r)]
// for the rows i < nrows and the cw columns j of B; store(i, j, value).  Each
// row is taken by 8 lanes (4 rows per warp), each lane summing every 8th r in
// FP64 for kJG columns at a time; the 8 partial sums are then combined in a
// fixed order (3 shuffle levels) and lane jj of the row's group stores
// column jj.
template <class RF, class AF, class BF, class SF>
__device__ void rows8(int nrows, int cw, const cd* B, int ldb, RF range, AF arow, BF bidx,
                      SF store) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 7;
  for (int i0 = warp * 4; i0 < nrows; i0 += kWarps * 4) {
    const int i = i0 + (lane >> 3);
    int lo = 0, hi = 0;
    if (i < nrows) range(i, lo, hi);
    for (int j0 = 0; j0 < cw; j0 += kJG) {
      cd acc[kJG];
#pragma unroll
      for (int jj = 0; jj < kJG; ++jj) acc[jj] = cz();
      const int nj = min(kJG, cw - j0);
      for (int r = lo + sub; r < hi; r += 8) {
        const cd av = arow(i, r);
        const cd* bp = B + (int64_t)j0 * ldb + bidx(i, r);
        if (nj == kJG) {
#pragma unroll
          for (int jj = 0; jj < kJG; ++jj) cfma(acc[jj], av, bp[jj * ldb]);
        } else {
#pragma unroll
          for (int jj = 0; jj < kJG; ++jj)
            if (jj < nj) cfma(acc[jj], av, bp[jj * ldb]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < kJG; ++jj) {
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) acc[jj] = cadd(acc[jj], shfl_xor(acc[jj], o));
      }
      cd mine = cz();
#pragma unroll
      for (int jj = 0; jj < kJG; ++jj)
        if (sub == jj) mine = acc[jj];
      if (i < nrows && sub < nj) store(i, j0 + sub, mine);
    }
  }
}

// One Newton step for the kept columns [j0, j1) of one edge.  Shared-memory
// buffers (column-major, column j at j * n): Uc (the start's columns), B1
// (Y = R_v^H U_c, then P = H U_c), B2 (T = N_q^w Y'_q, then S, then the
// update coefficients), B3 (Y'_q, then Z = conj(G_w) Y, then R); lamc the
// columns' Rayleigh quotients (negated start eigenvalue for tail columns),
// lamf the final eigenvalues.
__device__ void refine_chunk(const SolveArgs& a, const EdgeView& v, int j0, int j1, cd* Uc, cd* B1,
                             cd* B2, cd* B3, double* lamc, double* lamf) {
  const int chi = v.chi, n = v.n, A = v.act;
  const int64_t c2 = (int64_t)chi * chi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jl = min(j1, min(chi, A));
  for (int j = max(j0, jl) + tid; j < j1; j += blockDim.x) v.lam1[j] = 0.0;
  if (j0 >= jl) return;
  const int cw = jl - j0;
  for (int idx = tid; idx < cw * n; idx += blockDim.x) Uc[idx] = v.U[(int64_t)j0 * n + idx];
  __syncthreads();
  // Y = R_v^H U_c: Y[(k, perm_k[s])] = sum_{t <= s, t < rank_k} L_k[s][t] U[(k, t)]
  rows8(
      n, cw, Uc, n,
      [&](int i, int& lo, int& hi) {
        const int k = i / chi, s = i - k * chi;
        lo = 0;
        hi = min(s + 1, v.rank[k]);
      },
      [&](int i, int t) {
        const int k = i / chi, s = i - k * chi;
        return v.L[k * c2 + (int64_t)s * chi + t];
      },
      [&](int i, int t) { return (i / chi) * chi + t; },
      [&](int i, int j, cd val) {
        const int k = i / chi, s = i - k * chi;
        B1[j * n + k * chi + v.perm[k * chi + s]] = val;
      });
  __syncthreads();
  // Z = conj(G_w) Y through the rank-one phase structure of G_w: with the
  // global phase of b(q) chosen so that b_q(q) = 1 and b_k(q) = -i s (k != q),
  // conj(G_w) = sum_q c(q) c(q)^H (x) N_q^w, c(0) = (1, -i s), c(1) = (-i s, 1),
  // so Z = sum_q c(q) (x) N_q^w Y'_q with Y'_q = c(q)^H Y:
  //   Y'_0 = Y_0 + i s Y_1,  Y'_1 = i s Y_0 + Y_1      (into B3)
  //   T_q = N_q^w Y'_q                                  (into B2; two chi x chi products)
  //   Z_0 = T_0 - i s T_1,   Z_1 = -i s T_0 + T_1       (into B3)
  // The factors +-i s are exact, so this is conj(G_w) Y with half the products.
  const double sg = (double)a.sign;
  for (int idx = tid; idx < cw * n; idx += blockDim.x) {
    const int j = idx / n, i = idx - j * n;
    const int q = i / chi, e = i - q * chi;
    const cd y0 = B1[j * n + e], y1 = B1[j * n + chi + e];
    const cd other = q == 0 ? y1 : y0;             // the term multiplied by i s
    const cd mine = q == 0 ? y0 : y1;
    B3[j * n + i] = {mine.x - sg * other.y, mine.y + sg * other.x};
  }
  __syncthreads();
  rows8(
      n, cw, B3, n, [&](int, int& lo, int& hi) { lo = 0; hi = chi; },
      [&](int i, int r) {
        const int q = i / chi, e = i - q * chi;
        const int64_t o = (int64_t)q * 2 * c2 + (int64_t)e * chi + r;
        return cd{(double)v.gw[o], (double)v.gw[c2 + o]};
      },
      [&](int i, int r) { return (i / chi) * chi + r; },
      [&](int i, int j, cd val) { B2[j * n + i] = val; });
  __syncthreads();
  for (int idx = tid; idx < cw * n; idx += blockDim.x) {
    const int j = idx / n, i = idx - j * n;
    const int k = i / chi, e = i - k * chi;
    const cd t0 = B2[j * n + e], t1 = B2[j * n + chi + e];
    const cd other = k == 0 ? t1 : t0;             // the term multiplied by -i s
    const cd mine = k == 0 ? t0 : t1;
    B3[j * n + i] = {mine.x + sg * other.y, mine.y - sg * other.x};
  }
  __syncthreads();
  // P = R_v Z: P[(b, t)] = sum_{s >= t} conj(L_b[s][t]) Z[(b, perm_b[s])], zero for t >= rank_b
  rows8(
      n, cw, B3, n,
      [&](int i, int& lo, int& hi) {
        const int b = i / chi, t = i - b * chi;
        lo = t;
        hi = t < v.rank[b] ? chi : t;
      },
      [&](int i, int s) {
        const int b = i / chi, t = i - b * chi;
        return cconj(v.L[b * c2 + (int64_t)s * chi + t]);
      },
      [&](int i, int s) {
        const int b = i / chi;
        return b * chi + v.perm[b * chi + s];
      },
      [&](int i, int j, cd val) { B1[j * n + i] = val; });
  __syncthreads();
  // S = U_A^H P and R = I - U_A^H U_c
  rows8(
      A, cw, B1, n, [&](int, int& lo, int& hi) { lo = 0; hi = n; },
      [&](int i, int r) { return cconj(v.U[(int64_t)i * n + r]); }, [&](int, int r) { return r; },
      [&](int i, int j, cd val) { B2[j * n + i] = val; });
  rows8(
      A, cw, Uc, n, [&](int, int& lo, int& hi) { lo = 0; hi = n; },
      [&](int i, int r) { return cconj(v.U[(int64_t)i * n + r]); }, [&](int, int r) { return r; },
      [&](int i, int j, cd val) {
        B3[j * n + i] = {(i == j0 + j ? 1.0 : 0.0) - val.x, -val.y};
      });
  __syncthreads();
  // head columns (lambda_0 >= kHead lambda_0[0]) take the Newton step with
  // the Rayleigh quotient lambda_j = S_jj / (1 - R_jj); tail columns keep
  // their start's eigenvalue (lamc = -lambda_0 marks them)
  const double lhead = kHead * v.lam0[0];
  for (int j = tid; j < cw; j += blockDim.x) {
    const int jg = j0 + j;
    if (v.lam0[jg] >= lhead) {
      const double s = B2[j * n + jg].x, r = B3[j * n + jg].x;
      const double lam = s / (1.0 - r);
      lamc[j] = (lam > 0.0 && isfinite(lam)) ? lam : 0.0;
    } else {
      lamc[j] = -v.lam0[jg];
    }
  }
  __syncthreads();
  // Update coefficients c_ij (into B2), one warp per column j.  Head column:
  // c_ij = E_ij - S_ij / lambda_j - R_ij with the Newton E_ij (R_ij / 2 for
  // pairs that are not separated), and the final eigenvalue
  // lambda_j - sum_i |E_ij|^2 (lambda_i - lambda_j): the Rayleigh quotient of
  // the start carries that second-order contamination from the components
  // the step removes.  Tail column: c_ij = R_ij - conj(E_ji) against a head
  // column i (the mirror of the head column's correction, which keeps the
  // pair orthogonal to first order) and R_ij / 2 against a tail column.
  const double s00 = sqrt(fmax(v.lam0[0], 0.0));
  for (int j = warp; j < cw; j += kWarps) {
    const int jg = j0 + j;
    const double lj = lamc[j];
    const double ilj = lj > 0.0 ? 1.0 / lj : 0.0;
    double corr = 0.0;
    for (int i = lane; i < A; i += 32) {
      const cd s = B2[j * n + i], r = B3[j * n + i];
      const double li = v.lam0[i];
      cd c = cz();
      if (lj > 0.0) {
        cd e;
        if (i == jg) {
          e = cscale(r, 0.5);
        } else {
          const cd num = cadd(s, cscale(r, lj));
          const double den = lj - li;
          const double noise = kNoise * s00 * sqrt(fmax(li, 0.0));
          if (16.0 * cabs2(num) < den * den && fabs(den) > noise) {
            e = cscale(num, 1.0 / den);
            corr += cabs2(e) * (li - lj);
          } else {
            e = cscale(r, 0.5);
          }
        }
        c = csub(csub(e, cscale(s, ilj)), r);
      } else if (lj < 0.0) {
        if (i != jg && li >= lhead) {
          const cd num = cadd(cconj(s), cscale(cconj(r), li));
          const double den = li + lj;  // lambda_i - lambda_j
          const double noise = kNoise * s00 * (sqrt(li) + sqrt(-lj));
          const cd eji = (16.0 * cabs2(num) < den * den && fabs(den) > noise)
                             ? cscale(num, 1.0 / den)
                             : cscale(cconj(r), 0.5);
          c = csub(r, cconj(eji));
        } else {
          c = cscale(r, 0.5);
        }
      }
      B2[j * n + i] = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) corr += __shfl_xor_sync(0xffffffffu, corr, o);
    if (lane == 0) lamf[j] = lj > 0.0 ? lj - corr : v.lam0[jg];
  }
  __syncthreads();
  // u_j' = u_j + P_j / lambda_j + sum_{i < A} u_i c_ij for head columns,
  // u_j + sum_i u_i c_ij for tail columns; a head column without a positive
  // Rayleigh quotient keeps its start
  const int ng = (cw + kJU - 1) / kJU;
  for (int idx = tid; idx < n * ng; idx += blockDim.x) {
    const int r = idx % n, jb = (idx / n) * kJU;
    cd acc[kJU];
#pragma unroll
    for (int jj = 0; jj < kJU; ++jj) acc[jj] = cz();
    const int nj = min(kJU, cw - jb);
    for (int i = 0; i < A; ++i) {
      const cd u = v.U[(int64_t)i * n + r];
#pragma unroll
      for (int jj = 0; jj < kJU; ++jj)
        if (jj < nj) cfma(acc[jj], u, B2[(jb + jj) * n + i]);
    }
#pragma unroll
    for (int jj = 0; jj < kJU; ++jj) {
      const int j = jb + jj;
      if (jj >= nj) continue;
      const double lj = lamc[j];
      cd out = Uc[j * n + r];
      if (lj > 0.0) out = cadd(cadd(out, cscale(B1[j * n + r], 1.0 / lj)), acc[jj]);
      else if (lj < 0.0) out = cadd(out, acc[jj]);
      v.U1[(int64_t)(j0 + j) * n + r] = out;
    }
  }
  for (int j = tid; j < cw; j += blockDim.x) v.lam1[j0 + j] = lamf[j];
  __syncthreads();
}

// The kept-column slots of all edges, ne * chi, split evenly over the grid: each
// block takes a contiguous range (split further at edge boundaries and into
// pieces of at most cwmax columns).
__global__ void __launch_bounds__(kThreads, 1) refine_kernel(SolveArgs a, int cwmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi, n = 2 * chi;
  cd* Uc = reinterpret_cast<cd*>(smem_raw);
  cd* B1 = Uc + (int64_t)cwmax * n;
  cd* B2 = B1 + (int64_t)cwmax * n;
  cd* B3 = B2 + (int64_t)cwmax * n;
  double* lamc = reinterpret_cast<double*>(B3 + (int64_t)cwmax * n);
  double* lamf = lamc + cwmax;
  const int64_t T = (int64_t)a.n_edges * chi;
  const int64_t g0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t g1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  for (int64_t g = g0; g < g1;) {
    const int e = (int)(g / chi), j0 = (int)(g % chi);
    const int jend = (int)min((int64_t)chi, j0 + (g1 - g));
    const EdgeView v = edge_view(a, e);
    for (int s = j0; s < jend; s += cwmax) refine_chunk(a, v, s, min(jend, s + cwmax), Uc, B1, B2, B3, lamc, lamf);
    g += jend - j0;
  }
}

// ------------------------------------------------------------ leg matrices
// Same split of the kept-column slots.  Per edge: the kept set (the chi
// candidates with sigma above svd_cut * the largest), ||sigma||, and each
// column's slot in decreasing order.  Per chunk of refined columns u (both
// blocks b), in FP64:
//   Y = L_b u_b          (R_v^H u, so that C_w = R_v^T conj(u) = conj(Y)), and
//   W with L_b^H W = u_b (back substitution: C_v = R_v^+ u),
// then D_v[b][perm_b[s]][pos] = W[(b, s)] sqrt(sigma / ||sigma||) and
// D_w[q][e][pos] = sum_b b_b(q) conj(Y[(b, pinv_b(e))]) / sqrt(sigma ||sigma||)
// with b_b(q) = exp(s i pi/4 s_b s_q), as the gate split gives.
__global__ void __launch_bounds__(kThreads, 2) legs_kernel(SolveArgs a, int cwmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi, n = 2 * chi;
  cd* Ub = reinterpret_cast<cd*>(smem_raw);        // [cwmax][n] refined columns
  cd* Yb = Ub + (int64_t)cwmax * n;                // [cwmax][n]
  double* lam_s = reinterpret_cast<double*>(Yb + (int64_t)cwmax * n);  // [chi]
  int* pos_s = reinterpret_cast<int*>(lam_s + chi);                     // [chi]
  int* pinv = pos_s + chi;                                             // [2][chi]
  unsigned char* keep_s = reinterpret_cast<unsigned char*>(pinv + 2 * chi);  // [chi]
  __shared__ double scal[4];  // nrm, smax, kept count, discarded weight
  const int64_t c2 = (int64_t)chi * chi;
  const int tid = threadIdx.x;
  const int64_t T = (int64_t)a.n_edges * chi;
  const int64_t g0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t g1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const double sg = (double)a.sign;
  const double c45 = 0.70710678118654752440;
  for (int64_t g = g0; g < g1;) {
    const int e = (int)(g / chi), j0 = (int)(g % chi);
    const int j1 = (int)min((int64_t)chi, j0 + (g1 - g));
    g += j1 - j0;
    const EdgeView v = edge_view(a, e);
    const int cand = min(chi, v.act);
    for (int m = tid; m < chi; m += blockDim.x) lam_s[m] = m < cand ? v.lam1[m] : 0.0;
    for (int i = tid; i < 2 * chi; i += blockDim.x) pinv[(i / chi) * chi + v.perm[i]] = i % chi;
    __syncthreads();
    if (tid == 0) {
      double smax = 0.0;
      for (int m = 0; m < cand; ++m) smax = fmax(smax, lam_s[m] > 0.0 ? sqrt(lam_s[m]) : 0.0);
      double kept = 0.0, tot = 0.0;
      int nk = 0;
      for (int m = 0; m < chi; ++m) {
        const double s = lam_s[m] > 0.0 ? sqrt(lam_s[m]) : 0.0;
        const bool k = m < cand && s > 0.0 && s > a.svd_cut * smax;
        keep_s[m] = k;
        if (k) { kept += lam_s[m]; ++nk; }
        tot += m < cand ? fmax(lam_s[m], 0.0) : fmax(v.lam0[m], 0.0);
      }
      for (int m = chi; m < n; ++m) tot += fmax(v.lam0[m], 0.0);
      scal[0] = sqrt(kept);
      scal[1] = smax;
      scal[2] = nk;
      scal[3] = tot > 0.0 ? fmax(tot - kept, 0.0) / tot : 0.0;
    }
    __syncthreads();
    const int nk = (int)scal[2];
    for (int m = tid; m < chi; m += blockDim.x) {
      int p = 0;
      if (keep_s[m]) {
        for (int q = 0; q < chi; ++q)
          p += keep_s[q] && (lam_s[q] > lam_s[m] || (lam_s[q] == lam_s[m] && q < m));
      } else {
        p = nk;
        for (int q = 0; q < m; ++q) p += !keep_s[q];
      }
      pos_s[m] = p;
    }
    const double nrm = scal[0];
    const bool ok = nrm > 0.0 && isfinite(nrm);
    if (j0 == 0 && tid == 0) {
      double* st = a.stats + 4 * e;
      st[0] = scal[3];
      st[1] = nk;
      st[2] = scal[1];
      if (!ok) atomicOr(a.flags, 1);
    }
    float* dv = a.dmat + (int64_t)e * 8 * c2;
    float* dw = dv + 4 * c2;
    for (int js = j0; js < j1; js += cwmax) {
      const int cw = min(cwmax, j1 - js);
      for (int idx = tid; idx < cw * n; idx += blockDim.x) {
        const int jj = idx / n;
        Ub[idx] = keep_s[js + jj] ? v.U1[(int64_t)js * n + idx] : cz();
      }
      __syncthreads();
      // Y = L_b u_b (from the unmodified columns) first
      rows8(
          n, cw, Ub, n,
          [&](int i, int& lo, int& hi) {
            const int b = i / chi, t = i - b * chi;
            lo = 0;
            hi = min(t + 1, v.rank[b]);
          },
          [&](int i, int k) {
            const int b = i / chi, t = i - b * chi;
            return v.L[b * c2 + (int64_t)t * chi + k];
          },
          [&](int i, int k) { return (i / chi) * chi + k; },
          [&](int i, int j, cd val) { Yb[j * n + i] = val; });
      __syncthreads();
      // W: solve L_b^H w = u_b for every column of the chunk by back
      // substitution over s = rank_b - 1 .. 0, in place in Ub: w[s] = u[s] /
      // L[s][s], then u[t] -= conj(L[s][t]) w[s] for t < s (both blocks and all
      // columns at once, one pass per s)
      const int rmax = max(v.rank[0], v.rank[1]);
      for (int sidx = rmax - 1; sidx >= 0; --sidx) {
        for (int idx = tid; idx < 2 * cw; idx += blockDim.x) {
          const int b = idx / cw, jj = idx - b * cw;
          if (sidx < v.rank[b]) {
            const cd d = v.L[b * c2 + (int64_t)sidx * chi + sidx];
            Ub[jj * n + b * chi + sidx] = cscale(Ub[jj * n + b * chi + sidx], 1.0 / d.x);
          }
        }
        __syncthreads();
        for (int idx = tid; idx < 2 * cw * sidx; idx += blockDim.x) {
          const int b = idx / (cw * sidx), rem = idx - b * cw * sidx;
          const int jj = rem / sidx, t = rem - jj * sidx;
          if (sidx < v.rank[b]) {
            const cd l = cconj(v.L[b * c2 + (int64_t)sidx * chi + t]);
            const cd w = Ub[jj * n + b * chi + sidx];
            cd& u = Ub[jj * n + b * chi + t];
            u.x = fma(-l.x, w.x, u.x);
            u.x = fma(l.y, w.y, u.x);
            u.y = fma(-l.x, w.y, u.y);
            u.y = fma(-l.y, w.x, u.y);
          }
        }
        __syncthreads();
      }
      cd* Wb_ = Ub;  // W now occupies Ub (entries past each block's rank unused)
      // D_v and D_w columns, one thread per (column, e)
      for (int idx = tid; idx < cw * chi; idx += blockDim.x) {
        const int jj = idx / chi, ei = idx - jj * chi, m = js + jj;
        const int p = pos_s[m];
        const bool keep = ok && keep_s[m];
        const double sgm = keep ? sqrt(lam_s[m]) : 0.0;
        const double fv = keep ? sqrt(sgm / nrm) : 0.0;
        const double fw = keep ? 1.0 / sqrt(sgm * nrm) : 0.0;
        const int64_t o = (int64_t)ei * chi + p;
        cd w0 = cz(), w1 = cz();
        for (int b = 0; b < 2; ++b) {
          const int s = pinv[b * chi + ei];
          const cd z = (keep && s < v.rank[b]) ? cscale(Wb_[jj * n + b * chi + s], fv) : cz();
          dv[(int64_t)b * 2 * c2 + o] = (float)z.x;
          dv[(int64_t)b * 2 * c2 + c2 + o] = (float)z.y;
          const cd y = Yb[jj * n + b * chi + s];
          const cd cwv = {y.x * fw, -y.y * fw};
          const double sb = (b == 0) ? 1.0 : -1.0;
          w0 = cadd(w0, cmul({c45, sg * sb * c45}, cwv));
          w1 = cadd(w1, cmul({c45, -sg * sb * c45}, cwv));
        }
        dw[o] = (float)w0.x;
        dw[c2 + o] = (float)w0.y;
        dw[2 * c2 + o] = (float)w1.x;
        dw[3 * c2 + o] = (float)w1.y;
      }
      for (int jj = tid; jj < cw; jj += blockDim.x) {
        const int m = js + jj, p = pos_s[m];
        const bool keep = ok && keep_s[m];
        if (a.s_out) a.s_out[(int64_t)e * chi + p] = keep ? sqrt(lam_s[m]) / nrm : 0.0;
      }
      if (ok && a.msg) {
        float* m0 = a.msg + (int64_t)a.msg_vw[2 * e] * 2 * c2;
        float* m1 = a.msg + (int64_t)a.msg_vw[2 * e + 1] * 2 * c2;
        for (int idx = tid; idx < cw * chi; idx += blockDim.x) {
          const int jj = idx / chi, k = idx - jj * chi, m = js + jj;
          const int p = pos_s[m];
          const float val = (k == p && keep_s[m]) ? (float)(sqrt(lam_s[m]) / nrm) : 0.f;
          m0[(int64_t)p * chi + k] = val; m0[c2 + (int64_t)p * chi + k] = 0.f;
          m1[(int64_t)p * chi + k] = val; m1[c2 + (int64_t)p * chi + k] = 0.f;
        }
      }
      __syncthreads();
    }
  }
}

// Shared-memory limits of the refined solve's kernels, raised once to the
// largest request any chi <= kMaxChi makes, so that concurrent launches (the
// job server's slots) never lower a limit another thread relies on.
constexpr size_t kCholSmemMax = sizeof(cd) * kSmemChi * (kSmemChi + 1);
constexpr size_t kRefineSmemMax = kSmemBudget + 4096;
constexpr size_t kLegsSmemMax = kSmemBudget / 2 + 8192;

cudaError_t refine_prepare() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    result = cudaFuncSetAttribute(chol64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kCholSmemMax);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRefineSmemMax);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(legs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kLegsSmemMax);
  });
  return result;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return sms > 0 ? sms : 148;
}

}  // namespace

bool solve_refined_supported(int chi) {
  if (chi >= 1 && chi <= kSmemChi) return solve32_supported(chi);
  return chi <= kMaxChi && (2 * chi) % 32 == 0;  // the global-memory basis kernel
}

cudaError_t launch_solve_refined_basis(const SolveArgs& a, cudaStream_t st) {
  if (a.n_edges <= 0) return cudaSuccess;
  if (!solve_refined_supported(a.chi)) return cudaErrorInvalidValue;
  const int chi = a.chi;
  // 1. FP64 Cholesky of the v-side Gram blocks
  const size_t sm_chol = chi <= kSmemChi ? sizeof(cd) * (size_t)chi * (chi + 1) : 0;
  cudaError_t e = refine_prepare();
  if (e != cudaSuccess) return e;
  chol64_kernel<<<dim3(2, a.n_edges), kThreads, sm_chol, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 2. FP32 starting basis
  SolveArgs b = a;
  b.basis = 1;
  return chi <= kSmemChi ? launch_solve32(b, st) : launch_basis_gmem(b, st);
}

cudaError_t launch_solve_refined_newton(const SolveArgs& a, cudaStream_t st) {
  if (a.n_edges <= 0) return cudaSuccess;
  if (!solve_refined_supported(a.chi)) return cudaErrorInvalidValue;
  const int chi = a.chi, n = 2 * chi;
  // 3. FP64 Newton step, the kept-column slots balanced over the SMs
  const int64_t T = (int64_t)a.n_edges * chi;
  const int cw_fit = (int)(kSmemBudget / (sizeof(cd) * 4 * (size_t)n + 2 * sizeof(double)));
  int grid = (int)std::min<int64_t>(T, sm_count());
  grid = (int)std::max<int64_t>(grid, (T + cw_fit - 1) / cw_fit);
  const int cwmax = (int)((T + grid - 1) / grid);
  const size_t sm_ref = sizeof(cd) * 4 * (size_t)cwmax * n + 2 * sizeof(double) * cwmax;
  cudaError_t e = refine_prepare();
  if (e != cudaSuccess) return e;
  if (sm_ref > kRefineSmemMax) return cudaErrorInvalidValue;
  refine_kernel<<<grid, kThreads, sm_ref, st>>>(a, cwmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 4. FP64 leg matrices, spectrum and messages.  The back substitution is a
  // chain of chi dependent passes: two CTAs per SM (half the columns each)
  // overlap their latencies.
  int grid_l = (int)std::min<int64_t>(T, 2 * (int64_t)sm_count());
  const int cw_fit_l = (int)((kLegsSmemMax - 8192) / (sizeof(cd) * 2 * (size_t)n));
  grid_l = (int)std::max<int64_t>(grid_l, (T + cw_fit_l - 1) / cw_fit_l);
  const int cw_l = (int)((T + grid_l - 1) / grid_l);
  const size_t sm_legs = sizeof(cd) * 2 * (size_t)cw_l * n + sizeof(double) * chi +
                         sizeof(int) * 3 * chi + chi + 16;
  if (sm_legs > kLegsSmemMax) return cudaErrorInvalidValue;
  legs_kernel<<<grid_l, kThreads, sm_legs, st>>>(a, cw_l);
  return cudaGetLastError();
}

cudaError_t launch_solve_refined(const SolveArgs& a, cudaStream_t st) {
  cudaError_t e = launch_solve_refined_basis(a, st);
  if (e != cudaSuccess) return e;
  return launch_solve_refined_newton(a, st);
}

}  // namespace tnbp
