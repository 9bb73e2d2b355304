// Shared-memory truncation solve with FP32 rotations (chi <= 64).
//
// Same inputs and outputs as the FP64 solve in solve.cu (open-p environments
// of both sides of each gate edge in; per-p leg matrices D, the new bond
// spectrum and the gate-edge messages out), organised so that every O(chi^3)
// step runs from shared memory on the FP32 pipes.  Norms, the spectrum and its
// normalisation are accumulated in FP64.
//
// The gate exp(s i pi/4 ZZ) is split on the projectors of v's physical index:
// exp(s i pi/4 ZZ) = sum_p |p><p| (x) B_p, B_p = exp(s i pi/4 s_p Z), s_0 = +1,
// s_1 = -1 (Eq. 1's two-site gate).  The gate-split matrix of the v side,
// Xv[(p', r), (e, k)] = delta_{k p'} X_v[p', r, e], then has the block-diagonal
// Gram matrix G_v = diag(conj N_0, conj N_1); on the w side
// G_w[(e,k), (e',k')] = sum_q conj(b_k(q)) b_k'(q) conj(N_q^w)[e, e'] with
// b_k(q) = exp(s i pi/4 s_k s_q).  Steps per edge (one CTA):
//   1. pivoted Cholesky of the two chi x chi blocks of G_v and of G_w (2chi):
//      P^T G P = L L^H, so G = R^H R with R = L^H P^T;
//   2. K^T = R_w R_v^T (the bond matrix K = R_v R_w^T, transposed);
//   3. one-sided Jacobi on the columns of K (rows of K^T) until every pair is
//      orthogonal to FP32 precision: K V = U diag(sigma), with no squaring of
//      the condition number;
//   4. keep the chi largest sigma (above svd_cut * sigma_1), S = sigma/||sigma||;
//   5. C_v = R_v^+ U sqrt(S) (any z with R_v z = u serves: solutions differ by
//      null(R_v) = null(Xv), invisible in Xv z), C_w = R_v^T conj(U) / sqrt(sigma ||sigma||);
//   6. D_v[p] = C_v[block p], D_w[q] = sum_k b_k(q) C_w[block k]; both gate-edge
//      messages <- diag(S).
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "tnbp.h"

namespace tnbp {
namespace {

constexpr int kThreads = 1024;

constexpr int kWarps = kThreads / 32;
constexpr int kMaxChi = 64;
constexpr double kAbsTol = 1e-12;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconjf(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
// (a, b, c, d) -> (a, c, b, d): two interleaved complex values <-> their real
// pair and imaginary pair (the same permutation both ways)
__device__ __forceinline__ float4 pair_swap(float4 v) { return make_float4(v.x, v.z, v.y, v.w); }

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// A group of threads [t0, t0 + nt) of the block synchronised by a named barrier.
struct Group {
  int t0, nt, bar;
  __device__ int tid() const { return (int)threadIdx.x - t0; }
  __device__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory"); }
};

// Pivoted Cholesky of the Hermitian PSD m x m matrix A (row stride ld, full
// storage) in place, FP32 in shared memory, by the threads of group g:
// afterwards A's lower triangle holds L with P^T A P = L L^H, perm[t] =
// original index of pivot t, and *rank the number of pivots above
// rel_tol * (largest initial diagonal); everything outside the first `rank`
// columns of the lower triangle is zeroed.  The trailing update keeps the full
// Hermitian block current, so each pivot's row and column exchange reads
// current values.  Per pivot: the group's first warp finds the pivot, one pass
// applies the symmetric exchange, one scales the column, one updates the
// trailing block (rows over warps, columns over lanes).
__device__ void pivoted_cholesky32(float2* A, int m, int ld, int* perm, float rel_tol, int* rank,
                                   int* piv_s, float* pv_s, float* dmax0, float2* colk,
                                   const Group& g) {
  const int tid = g.tid(), lane = tid & 31, warp = tid >> 5, nw = g.nt >> 5;
  for (int i = tid; i < m; i += g.nt) perm[i] = i;
  g.sync();
  int r = m;
  for (int k = 0; k < m; ++k) {
    if (warp == 0) {
      float best = -1.f;
      int bi = k;
      for (int i = k + lane; i < m; i += 32) {
        const float d = A[i * ld + i].x;
        if (d > best) { best = d; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        *pv_s = best;
        *piv_s = bi;
        if (k == 0) *dmax0 = best > 0.f ? best : 0.f;
      }
    }
    g.sync();
    const float pv = *pv_s;
    const int piv = *piv_s;
    const float d0 = *dmax0;
    if (!(d0 > 0.f) || !(pv > rel_tol * d0)) { r = k; break; }
    if (piv != k) {
      // symmetric exchange of rows / columns k and piv: rows over all columns
      // (the L part included), columns over the trailing rows, the 2 x 2 block
      // {k, piv} by one thread
      for (int j = tid; j < m; j += g.nt) {
        if (j == k || j == piv) continue;
        const float2 t = A[k * ld + j];
        A[k * ld + j] = A[piv * ld + j];
        A[piv * ld + j] = t;
        if (j > k) {
          const float2 u = A[j * ld + k];
          A[j * ld + k] = A[j * ld + piv];
          A[j * ld + piv] = u;
        }
      }
      if (tid == 0) {
        const float2 kk = A[k * ld + k], pp = A[piv * ld + piv];
        const float2 kp = A[k * ld + piv], pk = A[piv * ld + k];
        A[k * ld + k] = pp;
        A[piv * ld + piv] = kk;
        A[k * ld + piv] = pk;
        A[piv * ld + k] = kp;
        const int t = perm[k];
        perm[k] = perm[piv];
        perm[piv] = t;
      }
      g.sync();
    }
    const float d = sqrtf(A[k * ld + k].x);
    const float inv = 1.f / d;
    for (int i = k + 1 + tid; i < m; i += g.nt) {
      const float2 a = A[i * ld + k];
      const float2 l = make_float2(a.x * inv, a.y * inv);
      A[i * ld + k] = l;
      colk[i] = l;
    }
    g.sync();
    if (tid == 0) A[k * ld + k] = make_float2(d, 0.f);
    for (int i = k + 1 + warp; i < m; i += nw) {
      const float2 ci = colk[i];
      for (int j = k + 1 + lane; j < m; j += 32) {
        const float2 cj = colk[j];
        float2 a = A[i * ld + j];
        a.x -= ci.x * cj.x + ci.y * cj.y;  // ci conj(cj)
        a.y -= ci.y * cj.x - ci.x * cj.y;
        A[i * ld + j] = a;
      }
    }
    g.sync();
  }
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < m; j += 32)
      if (j > i || j >= r) A[i * ld + j] = make_float2(0.f, 0.f);
  if (tid == 0) *rank = r;
  g.sync();
}

struct Smem {
  float2* X;       // n x n: G_w -> L_w -> K^T -> rotated columns of K
  float2* Lv;      // 2 blocks chi x (chi + 1): L_0, L_1 (padded rows)
  int* perm_w;     // n
  int* perm_v;     // 2 chi
  int* src;        // n: K^T gather map
  int* order;      // n: rows by decreasing norm
  int* rank;       // 4
  int* red_i;      // 32
  float* red_v;    // 32
  float* dmax0;    // 4
  int* counter;    // 4
  double* sig;     // n
  double* scal;    // 4
  double* red_d;   // 32
  float2* colk;    // 2 n (one column buffer per concurrent factorisation)
  float* nrm;      // n: squared row norms during the Jacobi
};

__device__ Smem carve(unsigned char* base, int chi) {
  const int n = 2 * chi;
  Smem s;
  unsigned char* p = base;
  s.X = reinterpret_cast<float2*>(p); p += sizeof(float2) * n * n;
  s.Lv = reinterpret_cast<float2*>(p); p += sizeof(float2) * 2 * chi * (chi + 1);
  s.sig = reinterpret_cast<double*>(p); p += sizeof(double) * n;
  s.scal = reinterpret_cast<double*>(p); p += sizeof(double) * 4;
  s.red_d = reinterpret_cast<double*>(p); p += sizeof(double) * 32;
  s.colk = reinterpret_cast<float2*>(p); p += sizeof(float2) * 2 * n;
  s.nrm = reinterpret_cast<float*>(p); p += sizeof(float) * n;
  s.perm_w = reinterpret_cast<int*>(p); p += sizeof(int) * n;
  s.perm_v = reinterpret_cast<int*>(p); p += sizeof(int) * 2 * chi;
  s.src = reinterpret_cast<int*>(p); p += sizeof(int) * n;
  s.order = reinterpret_cast<int*>(p); p += sizeof(int) * n;
  s.rank = reinterpret_cast<int*>(p); p += sizeof(int) * 4;
  s.red_i = reinterpret_cast<int*>(p); p += sizeof(int) * 32;
  s.red_v = reinterpret_cast<float*>(p); p += sizeof(float) * 32;
  s.dmax0 = reinterpret_cast<float*>(p); p += sizeof(float) * 4;
  s.counter = reinterpret_cast<int*>(p); p += sizeof(int) * 4;
  return s;
}

// Basis mode output (the refined solve's FP32 phase).  Column m of the
// starting basis is row order[m] of the rotated K^T over its norm; lam0[m] =
// sigma^2; the active count is the number of columns with sigma above 1e-6
// sigma_1; the sum of sigma^2 and the sweep count go to misc.  The Jacobi
// leaves pairs whose overlap is below its absolute floor unrotated, so
// columns far below sigma_1 (the tail, sigma < 1e-3 sigma_1) can be far from
// orthogonal; each active tail column is therefore orthogonalised against
// every column before it and normalised (modified Gram-Schmidt in FP32, two
// passes), which leaves the whole active basis orthonormal to about 1e-7.
// Overwrites X and s.sig.
__device__ __noinline__ void write_basis(const SolveArgs& a, const Smem& s, float2* X, int edge,
                                         int chi, int sweeps) {
  const int n = 2 * chi, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const RefineLayout lay = refine_layout(chi);
  double* rbase = a.work + (int64_t)edge * lay.stride;
  int* rints = reinterpret_cast<int*>(rbase + lay.ints);
  const double s0 = s.sig[s.order[0]];
  for (int m = tid; m < n; m += blockDim.x) {
    const double sj = s.sig[s.order[m]];
    rbase[lay.lam0 + m] = sj * sj;
  }
  if (tid == 0) {
    int act = 0, head = 0;
    double tot = 0.0;
    for (int m = 0; m < n; ++m) {
      const double sj = s.sig[s.order[m]];
      tot += sj * sj;
      act += (sj > 0.0 && sj > 1e-6 * s0) ? 1 : 0;
      head += (sj > 0.0 && sj >= 1e-3 * s0) ? 1 : 0;
    }
    rints[2 * chi + 2] = act;
    s.counter[0] = act;
    s.counter[1] = head;
    rbase[lay.misc] = tot;
    rbase[lay.misc + 1] = sweeps;
    a.stats[4 * edge + 3] = sweeps;
    if (!(s0 > 0.0) || !isfinite(tot)) atomicOr(a.flags, 1);
  }
  __syncthreads();
  const int act = s.counter[0], head = s.counter[1];
  // unit rows
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int j = idx / n;
    const double sj = s.sig[j];
    const float is = sj > 0.0 ? (float)(1.0 / sj) : 0.f;
    X[idx] = make_float2(X[idx].x * is, X[idx].y * is);
  }
  __syncthreads();
  if (head < act) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = 0; k < act; ++k) {
        const int rk = s.order[k];
        if (k >= head) {
          // normalise tail row k (warp 0), every row before it being final
          if (warp == 0) {
            float acc = 0.f;
            for (int c = lane; c < n; c += 32) {
              const float2 v = X[rk * n + c];
              acc += v.x * v.x + v.y * v.y;
            }
            acc = warp_sum(acc);
            const float inv = acc > 0.f ? rsqrtf(acc) : 0.f;
            for (int c = lane; c < n; c += 32) {
              const float2 v = X[rk * n + c];
              X[rk * n + c] = make_float2(v.x * inv, v.y * inv);
            }
          }
          __syncthreads();
        }
        // x_m -= <u_k, x_m> u_k for the tail rows after k
        for (int m = max(k + 1, head) + warp; m < act; m += nwarps) {
          const int rm = s.order[m];
          float gr = 0.f, gi = 0.f;
          for (int c = lane; c < n; c += 32) {
            const float2 u = X[rk * n + c], x = X[rm * n + c];
            gr += u.x * x.x + u.y * x.y;
            gi += u.x * x.y - u.y * x.x;
          }
          gr = warp_sum(gr);
          gi = warp_sum(gi);
          for (int c = lane; c < n; c += 32) {
            const float2 u = X[rk * n + c], x = X[rm * n + c];
            X[rm * n + c] = make_float2(x.x - (gr * u.x - gi * u.y), x.y - (gr * u.y + gi * u.x));
          }
        }
        __syncthreads();
      }
    }
  }
  double2* U = reinterpret_cast<double2*>(rbase + lay.U);
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int m = idx / n, r = idx % n;
    const float2 x = X[s.order[m] * n + r];
    U[idx] = make_double2((double)x.x, (double)x.y);
  }
}

__global__ void __launch_bounds__(kThreads) solve32_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int chi = a.chi, n = 2 * chi;
  const int64_t c2 = (int64_t)chi * chi;
  const int edge = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Smem s = carve(smem_raw, chi);
  float2* X = s.X;
  const float* gv = a.gram + (int64_t)edge * 8 * c2;
  const float* gw = gv + 4 * c2;
  const float sg = (float)a.sign;

  // 1. Gram matrices: G_v blocks conj(N_p^v) in Lv, G_w from conj(N_q^w) in X.
  //    In basis mode Lv receives the FP64 Cholesky factors of the G_v blocks
  //    (lower triangles, rounded) with their pivot orders and ranks instead.
  const int ldv = chi + 1;
  if (a.basis) {
    // the FP64 factors come from chol64_kernel, which may still be running
    // (programmatic dependent launch): they are read after the G_w Cholesky
  } else {
    for (int idx = tid; idx < 2 * chi * chi; idx += blockDim.x) {
      const int p = idx / (chi * chi), o = idx % (chi * chi);
      s.Lv[p * chi * ldv + (o / chi) * ldv + o % chi] =
          make_float2(gv[p * 2 * c2 + o], -gv[p * 2 * c2 + c2 + o]);
    }
  }
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    const int ki = i / chi, ei = i % chi, kj = j / chi, ej = j % chi;
    const int64_t o = (int64_t)ei * chi + ej;
    const float2 g0 = make_float2(gw[o], -gw[c2 + o]);
    const float2 g1 = make_float2(gw[2 * c2 + o], -gw[3 * c2 + o]);
    float2 v;
    if (ki == kj) {
      v = make_float2(g0.x + g1.x, g0.y + g1.y);
    } else {
      // conj(b_ki(q)) b_kj(q) = exp(s i pi/4 (s_kj - s_ki) s_q): (0,1) -> -s i s_q,
      // (1,0) -> +s i s_q, so the block is -+ s i (G_0 - G_1)
      const float2 d = make_float2(g0.x - g1.x, g0.y - g1.y);
      const float f = (ki == 0) ? -sg : sg;
      v = make_float2(-f * d.y, f * d.x);
    }
    X[idx] = v;
  }
  __syncthreads();
  const float ctol = 1e-7f;
  float2* colk = reinterpret_cast<float2*>(s.colk);
  {
    // the two v-side blocks concurrently on the two halves of the block, then G_w
    const int half_t = kThreads / 2;
    const int h = tid >= half_t;
    const Group gh{h * half_t, half_t, 1 + h};
    if (!a.basis)
      pivoted_cholesky32(s.Lv + h * chi * ldv, chi, ldv, s.perm_v + h * chi, ctol, &s.rank[h],
                         s.red_i + h, s.red_v + h, s.dmax0 + h, colk + h * n, gh);
    __syncthreads();
    const Group gall{0, kThreads, 0};
    pivoted_cholesky32(X, n, n, s.perm_w, ctol, &s.rank[2], s.red_i, s.red_v, s.dmax0 + 2, colk,
                       gall);
  }
  if (a.basis) {
    // wait for chol64_kernel (all of its writes visible), then take its factors
    cudaGridDependencySynchronize();
    const RefineLayout lay = refine_layout(chi);
    const double* rbase = a.work + (int64_t)edge * lay.stride;
    const int* rints = reinterpret_cast<const int*>(rbase + lay.ints);
    const double2* L64 = reinterpret_cast<const double2*>(rbase + lay.L);
    for (int idx = tid; idx < 2 * chi * chi; idx += blockDim.x) {
      const int p = idx / (chi * chi), o = idx % (chi * chi);
      const double2 l = L64[idx];
      s.Lv[p * chi * ldv + (o / chi) * ldv + o % chi] = make_float2((float)l.x, (float)l.y);
    }
    for (int i = tid; i < 2 * chi; i += blockDim.x) s.perm_v[i] = rints[i];
    if (tid < 2) s.rank[tid] = rints[2 * chi + tid];
    __syncthreads();
  }

  // 2. K^T = R_w R_v^T.  First X <- conj(L_w^T) so that row j of X holds
  //    R_w[j][perm_w[t]] at column t.  Then with c = perm_b[t'] (block b):
  //    K^T[j][(b, i)] = sum_t' X[j][pinv_w(b chi + perm_b[t'])] conj(L_b[t'][i]).
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    if (i < j) {
      const float2 u = X[i * n + j], l = X[j * n + i];
      X[i * n + j] = cconjf(l);
      X[j * n + i] = cconjf(u);
    } else if (i == j) {
      X[idx] = cconjf(X[idx]);
    }
  }
  // src[(b, t')] = pinv_w(b chi + perm_b[t'])
  for (int t = tid; t < n; t += blockDim.x) s.src[s.perm_w[t]] = -1 - t;  // temp: pinv_w
  __syncthreads();
  for (int bt = tid; bt < n; bt += blockDim.x) {
    const int b = bt / chi, tp = bt % chi;
    const int c = b * chi + s.perm_v[b * chi + tp];
    s.order[bt] = -1 - s.src[c];  // pinv_w(c), staged in order[]
  }
  __syncthreads();
  for (int bt = tid; bt < n; bt += blockDim.x) s.src[bt] = s.order[bt];
  __syncthreads();
  const int npl = n / 32 > 0 ? (n + 31) / 32 : 1;  // values per lane (<= 4)
  if (n % 32 == 0) {
    // Each warp owns n/32 whole rows j, each lane n/32 consecutive output
    // columns o = (b, i) (all in one block b): a register tile of rows x
    // columns over t', the rows' gathered values broadcast from shared memory,
    // the lane's L_b row segment read contiguously.  Rows are written back in
    // place once the warp has read them.
    const int cl = n / 32;            // columns per lane, rows per warp
    const int o0 = lane * cl;
    const int b = o0 / chi, i0 = o0 - b * chi;
    const float2* Lb = s.Lv + b * chi * ldv;
    const int* srcb = s.src + b * chi;
    for (int r0 = 0; r0 < cl; r0 += 2) {
      const int j0 = warp * cl + r0;
      const int nr = cl - r0 < 2 ? cl - r0 : 2;
      float2 acc[2][4];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
      for (int tp = 0; tp < chi; ++tp) {
        const int col = srcb[tp];
        float2 y[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) y[r] = r < nr ? X[(j0 + r) * n + col] : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < cl) {
            const float2 z = cconjf(Lb[tp * ldv + i0 + c]);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const float2 pz = cmulf(y[r], z);
              acc[r][c].x += pz.x;
              acc[r][c].y += pz.y;
            }
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (r < nr && c < cl) X[(j0 + r) * n + o0 + c] = acc[r][c];
      __syncwarp();
    }
  } else {
  for (int j = warp; j < n; j += kWarps) {
    float2 y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int bt = u * 32 + lane;
      y[u] = (u < npl && bt < n) ? X[j * n + s.src[bt]] : make_float2(0.f, 0.f);
    }
    float2 out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = make_float2(0.f, 0.f);
    for (int bt = 0; bt < n; ++bt) {
      const float2 yv = shfl2(y[bt >> 5], bt & 31);
      const int b = bt / chi, tp = bt % chi;
      const float2* Lb = s.Lv + b * chi * ldv;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = u * 32 + lane;  // output (b, i) = o
        if (u < npl && o < n && o / chi == b) {
          const int i = o % chi;
          if (i <= tp) {
            const float2 p = cmulf(yv, cconjf(Lb[tp * ldv + i]));
            out[u].x += p.x;
            out[u].y += p.y;
          }
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = u * 32 + lane;
      if (u < npl && o < n) X[j * n + o] = out[u];
    }
  }
  }
  __syncthreads();

  // 3. One-sided Jacobi on the rows of X (columns of K), round-robin pairs.
  //    ||K||_F^2 (invariant under the rotations) sets an absolute floor: a pair
  //    whose overlap is below kAbsTol ||K||_F^2 cannot move any singular value
  //    above the truncation cut, and rotating rounding noise would never stop.
  {
    double acc = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const float2 v = X[idx];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc = warp_sum_d(acc);
    if (lane == 0) s.red_d[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s.red_d[w];
      s.scal[2] = t;
    }
    __syncthreads();
  }
  const float abs_floor = (float)(kAbsTol * s.scal[2]);
  const float orth_tol = a.orth_tol > 0.f ? a.orth_tol : 2e-6f;
  const float orth_tol2 = orth_tol * orth_tol, abs_floor2 = abs_floor * abs_floor;
  const int half = n / 2;
  int sweeps = 0;
  if (n % 32 == 0) {
    // Rows of 2 x 16-byte vectors, each pair owned by 16 lanes (two pairs per
    // warp, so the rotation arithmetic serves two pairs), lane l holding the
    // vectors l, l + 16, ... of a row (consecutive lanes, consecutive
    // addresses).  Pair order: recursive halving.  At level B (B = n/2, n/4,
    // .., 1) the rows form groups of 2B; slot s = g B + i keeps row g 2B + i
    // ("stationary") in registers for the B rounds of the level and meets
    // row g 2B + B + (i + r) mod B in round r, so every pair of rows meets
    // exactly once per sweep in n - 1 rounds, as in the round-robin order,
    // while only the partner row passes through shared memory each round
    // (shared-memory bandwidth bounds this loop).  Squared row norms:
    // recomputed exactly at the start of each sweep, updated by each rotation,
    // which moves t |gamma| of weight from row p to row q
    // (alpha' = alpha - t|g|, beta' = beta + t|g|).
    // Rows are held pair-split for the sweeps: each float4 carries the real
    // parts of two consecutive complex values, then their imaginary parts, so
    // that every complex dot product and rotation runs as paired FP32 FMAs
    // (two lanes of arithmetic per instruction) without operand shuffles.
    float4* X4 = reinterpret_cast<float4*>(X);
    const int row4 = n / 2, nq = n / 32;
    const int sub = lane >> 4, gl = lane & 15;
    const int slot = warp * 2 + sub;
    const bool active = 2 * warp < half;  // warp-uniform: half is even
    for (int idx = tid; idx < n * row4; idx += blockDim.x) X4[idx] = pair_swap(X4[idx]);
    __syncthreads();
    for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
      ++sweeps;
      for (int j = warp; j < n; j += kWarps) {
        float acc = 0.f;
        for (int c = lane; c < row4; c += 32) {
          const float4 v = X4[j * row4 + c];
          acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
        }
        acc = warp_sum(acc);
        if (lane == 0) s.nrm[j] = acc;
      }
      __syncthreads();
      // rows taken in order of decreasing norm this sweep (ties by index)
      for (int i = tid; i < n; i += blockDim.x) {
        const float ni = s.nrm[i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
          const float nj = s.nrm[j];
          rk += (nj > ni) || (nj == ni && j < i);
        }
        s.order[rk] = i;
      }
      __syncthreads();
      int any = 0;
      for (int B = half; B >= 1; B >>= 1) {
        const int g = slot / B, i = slot - g * B;
        const int prow = s.order[g * 2 * B + i];
        float4 xs[4];
        float al = 0.f;
        if (active) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < nq) xs[u] = X4[prow * row4 + gl + 16 * u];
          al = s.nrm[prow];
        }
        for (int r = 0; r < B; ++r) {
          int rot = 0;
          if (active) {
            const int ir = i + r >= B ? i + r - B : i + r;  // (i + r) mod B, i, r < B
            const int q = s.order[g * 2 * B + B + ir];
            float4 xq[4];
            // gamma = sum conj(x_p) x_q: Re = sum pr qr + pi qi, Im = sum pr qi - pi qr
            float2 ar = f2(0.f), ai = f2(0.f), aj = f2(0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (u < nq) {
                xq[u] = X4[q * row4 + gl + 16 * u];
                const float2 pr = make_float2(xs[u].x, xs[u].y), pi = make_float2(xs[u].z, xs[u].w);
                const float2 qr = make_float2(xq[u].x, xq[u].y), qi = make_float2(xq[u].z, xq[u].w);
                ar = __ffma2_rn(pr, qr, ar);
                ar = __ffma2_rn(pi, qi, ar);
                ai = __ffma2_rn(pr, qi, ai);
                aj = __ffma2_rn(pi, qr, aj);
              }
            }
            float gr = ar.x + ar.y, gi = (ai.x + ai.y) - (aj.x + aj.y);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
              gr += __shfl_xor_sync(0xffffffffu, gr, o);
              gi += __shfl_xor_sync(0xffffffffu, gi, o);
            }
            const float be = s.nrm[q];
            const float g2 = gr * gr + gi * gi;
            // |gamma| > orth_tol sqrt(al be) and |gamma| > abs_floor, compared squared
            if (g2 > orth_tol2 * al * be && g2 > abs_floor2 && g2 > 0.f) {
              // 1/|gamma| and cos = 1/sqrt(1 + t^2) from the hardware reciprocal
              // square root refined by one step of Newton's iteration
              // y <- y (3 - x y^2) / 2: the phase e^{-i phi} and the pair (cos, sin)
              // are then unit to about one ulp, so the rotations stay unitary and
              // the row norms do not drift.  t itself may be approximate: any t
              // gives a unitary rotation, and an inexact angle only leaves a
              // residual overlap that later rounds remove.
              float ig = rsqrtf(g2);
              ig = ig * (1.5f - 0.5f * g2 * ig * ig);
              const float gm = g2 * ig;
              const float2 ph = make_float2(gr * ig, -gi * ig);  // e^{-i phi}
              const float tau = (be - al) * 0.5f * ig;
              const float at = fabsf(tau);
              float t;
              if (at < 1e15f) {
                const float q1 = 1.f + at * at;
                t = __fdividef(1.f, at + q1 * rsqrtf(q1));  // 1 / (|tau| + sqrt(1 + tau^2))
              } else {
                t = 0.5f / at;
              }
              if (tau < 0.f) t = -t;
              const float q2 = 1.f + t * t;
              float cs = rsqrtf(q2);
              cs = cs * (1.5f - 0.5f * q2 * cs * cs);
              const float sn = t * cs;
              // pq = e^{-i phi} x_q; x_p <- cs x_p - sn pq, x_q <- sn x_p + cs pq,
              // two complex values per paired operation
              const float2 phr = f2(ph.x), phi = f2(ph.y), nphi = f2(-ph.y);
              const float2 cs2 = f2(cs), sn2 = f2(sn), nsn2 = f2(-sn);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (u < nq) {
                  const float2 pr = make_float2(xs[u].x, xs[u].y), pi = make_float2(xs[u].z, xs[u].w);
                  const float2 qr = make_float2(xq[u].x, xq[u].y), qi = make_float2(xq[u].z, xq[u].w);
                  const float2 pqr = __ffma2_rn(nphi, qi, __fmul2_rn(phr, qr));
                  const float2 pqi = __ffma2_rn(phi, qr, __fmul2_rn(phr, qi));
                  const float2 npr = __ffma2_rn(nsn2, pqr, __fmul2_rn(cs2, pr));
                  const float2 npi = __ffma2_rn(nsn2, pqi, __fmul2_rn(cs2, pi));
                  const float2 nqr = __ffma2_rn(sn2, pr, __fmul2_rn(cs2, pqr));
                  const float2 nqi = __ffma2_rn(sn2, pi, __fmul2_rn(cs2, pqi));
                  xs[u] = make_float4(npr.x, npr.y, npi.x, npi.y);
                  X4[q * row4 + gl + 16 * u] = make_float4(nqr.x, nqr.y, nqi.x, nqi.y);
                }
              }
              al = fmaxf(al - t * gm, 0.f);
              if (gl == 0) s.nrm[q] = be + t * gm;
              rot = 1;
            }
          }
          any |= __syncthreads_or(rot);
        }
        if (active) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < nq) X4[prow * row4 + gl + 16 * u] = xs[u];
          if (gl == 0) s.nrm[prow] = al;
        }
        __syncthreads();
      }
      if (!any) break;
    }
    for (int idx = tid; idx < n * row4; idx += blockDim.x) X4[idx] = pair_swap(X4[idx]);
    __syncthreads();
  } else
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    ++sweeps;
    if (tid == 0) s.counter[0] = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      for (int k = warp; k < half; k += kWarps) {
        int p, q;
        if (k == 0) { p = r; q = n - 1; }
        else { p = (r + k) % (n - 1); q = (r - k + (n - 1)) % (n - 1); }
        float2 xp[4], xq[4];
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = u * 32 + lane;
          if (u < npl && c < n) {
            xp[u] = X[p * n + c];
            xq[u] = X[q * n + c];
          } else {
            xp[u] = xq[u] = make_float2(0.f, 0.f);
          }
          al += xp[u].x * xp[u].x + xp[u].y * xp[u].y;
          be += xq[u].x * xq[u].x + xq[u].y * xq[u].y;
          // gamma = sum conj(xp) xq
          gr += xp[u].x * xq[u].x + xp[u].y * xq[u].y;
          gi += xp[u].x * xq[u].y - xp[u].y * xq[u].x;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const float gm = sqrtf(gr * gr + gi * gi);
        // pairs already orthogonal to FP32 precision are left alone; a sweep
        // that rotates no pair ends the iteration
        if (gm > orth_tol * sqrtf(al * be) && gm > abs_floor && gm > 0.f) {
          const float2 ph = make_float2(gr / gm, -gi / gm);  // e^{-i phi}, gamma = |g| e^{i phi}
          const float tau = (be - al) / (2.f * gm);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          // exactly rounded: an approximate reciprocal square root makes every
          // rotation slightly non-unitary and the column norms drift
          const float cs = 1.f / sqrtf(1.f + t * t);
          const float sn = t * cs;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = u * 32 + lane;
            if (u < npl && c < n) {
              const float2 pq = cmulf(ph, xq[u]);
              X[p * n + c] = make_float2(cs * xp[u].x - sn * pq.x, cs * xp[u].y - sn * pq.y);
              X[q * n + c] = make_float2(sn * xp[u].x + cs * pq.x, sn * xp[u].y + cs * pq.y);
            }
          }
          if (lane == 0) atomicAdd(s.counter, 1);
        }
      }
      __syncthreads();
    }
    if (s.counter[0] == 0) break;
    __syncthreads();
  }

  // 4. sigma_j = ||row j|| (FP64), order by decreasing sigma, truncate, normalise.
  for (int j = warp; j < n; j += kWarps) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) {
      const float2 v = X[j * n + c];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc = warp_sum_d(acc);
    if (lane == 0) s.sig[j] = sqrt(acc);
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const double si = s.sig[i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = s.sig[j];
      rk += (sj > si) || (sj == si && j < i);
    }
    s.order[rk] = i;
  }
  __syncthreads();
  if (a.basis) {
    write_basis(a, s, X, edge, chi, sweeps);
    return;
  }
  if (tid == 0) {
    double tot = 0.0, kept = 0.0;
    for (int i = 0; i < n; ++i) tot += s.sig[i] * s.sig[i];
    const double s0 = s.sig[s.order[0]];
    int nk = 0;
    for (int m = 0; m < chi; ++m) {
      const double v = s.sig[s.order[m]];
      if (v > 0.0 && v > a.svd_cut * s0) { kept += v * v; ++nk; }
    }
    s.scal[0] = sqrt(kept);
    s.scal[1] = nk;
    double* st = a.stats + 4 * edge;
    st[0] = tot > 0.0 ? (tot - kept) / tot : 0.0;
    st[1] = nk;
    st[2] = s0;
    st[3] = sweeps;
    if (!(kept > 0.0) || !isfinite(kept)) atomicOr(a.flags, 1);
  }
  __syncthreads();
  const double nrm = s.scal[0];
  const int nk = (int)s.scal[1];
  const bool ok = nrm > 0.0 && isfinite(nrm);

  // 5-6. One warp per kept column m: u = row_j / sigma (length n, index (b, i)).
  float* dv = a.dmat + (int64_t)edge * 8 * c2;
  float* dw = dv + 4 * c2;
  const float c45 = 0.70710678118654752f;
  for (int m = warp; m < chi; m += kWarps) {
    const bool keep = ok && m < nk;
    const int j = s.order[m];
    const double sgm = s.sig[j];
    const float fv = keep ? (float)sqrt(sgm / nrm) : 0.f;        // sqrt(S_m)
    const float fw = keep ? (float)(1.0 / sqrt(sgm * nrm)) : 0.f;  // 1/sqrt(sigma ||sigma||)
    const float inv_s = keep ? (float)(1.0 / sgm) : 0.f;
    for (int b = 0; b < 2; ++b) {
      const float2* Lb = s.Lv + b * chi * ldv;
      const int rb = s.rank[b];
      const int* pb = s.perm_v + b * chi;
      // u block b, lane owns entries i = lane, lane + 32
      float2 u[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = h * 32 + lane;
        u[h] = (keep && i < chi) ? X[j * n + b * chi + i] : make_float2(0.f, 0.f);
        u[h].x *= inv_s;
        u[h].y *= inv_s;
      }
      // C_v block b: solve L_b^H w = u by columns (t < rank, from the last):
      // w[t] = u[t] / L[t][t], then u[t'] -= conj(L[t][t']) w[t] for t' < t
      // (row t of L, contiguous over the lanes), z[perm[t]] = w[t]
      float2 w[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float2 uu[2] = {u[0], u[1]};
      for (int t = rb - 1; t >= 0; --t) {
        const float2 ut = shfl2(uu[t >> 5], t & 31);
        const float d = Lb[t * ldv + t].x;
        const float2 wt = make_float2(ut.x / d, ut.y / d);
        if ((t >> 5) == 0 && lane == (t & 31)) w[0] = wt;
        if ((t >> 5) == 1 && lane == (t & 31)) w[1] = wt;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int t2 = h * 32 + lane;
          if (t2 < t) {
            const float2 pr = cmulf(cconjf(Lb[t * ldv + t2]), wt);
            uu[h].x -= pr.x;
            uu[h].y -= pr.y;
          }
        }
      }
      // D_v[p = b][e][m] = z[e] * sqrt(S_m), e = perm_b[t]
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = h * 32 + lane;
        if (t < chi) {
          const int e = pb[t];
          const float2 z = (t < rb) ? make_float2(w[h].x * fv, w[h].y * fv) : make_float2(0.f, 0.f);
          dv[b * 2 * c2 + (int64_t)e * chi + m] = z.x;
          dv[b * 2 * c2 + c2 + (int64_t)e * chi + m] = z.y;
        }
      }
      // C_w block b: y[t] = sum_{i <= t} L_b[t][i] u[i] (lower-triangular matvec),
      // C_w[(b, perm_b[t])][m] = conj(y[t]) * fw.  D_w[q] = sum_k b_k(q) C_w[block k].
      float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      for (int i = 0; i < chi; ++i) {
        const float2 ui = shfl2(u[i >> 5], i & 31);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int t = h * 32 + lane;
          if (t < chi && i <= t) {
            const float2 pr = cmulf(Lb[t * ldv + i], ui);
            y[h].x += pr.x;
            y[h].y += pr.y;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = h * 32 + lane;
        if (t < chi) {
          const int e = pb[t];
          const float2 cw = make_float2(y[h].x * fw, -y[h].y * fw);
          // b_b(q) = exp(s i pi/4 s_b s_q): q = 0 -> exp(s i pi/4 s_b), q = 1 -> its conjugate
          const float sb = (b == 0) ? 1.f : -1.f;
          const float2 b0 = make_float2(c45, sg * sb * c45);
          const float2 b1 = make_float2(c45, -sg * sb * c45);
          const float2 v0 = cmulf(b0, cw), v1 = cmulf(b1, cw);
          float* d0 = dw + (int64_t)e * chi + m;
          float* d1 = dw + 2 * c2 + (int64_t)e * chi + m;
          if (b == 0) {
            d0[0] = v0.x; d0[c2] = v0.y;
            d1[0] = v1.x; d1[c2] = v1.y;
          } else {
            d0[0] += v0.x; d0[c2] += v0.y;
            d1[0] += v1.x; d1[c2] += v1.y;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (a.s_out) {
    for (int m = tid; m < chi; m += blockDim.x)
      a.s_out[(int64_t)edge * chi + m] = (ok && m < nk) ? s.sig[s.order[m]] / nrm : 0.0;
  }
  if (ok && a.msg) {
    float* m0 = a.msg + (int64_t)a.msg_vw[2 * edge] * 2 * c2;
    float* m1 = a.msg + (int64_t)a.msg_vw[2 * edge + 1] * 2 * c2;
    for (int idx = tid; idx < chi * chi; idx += blockDim.x) {
      const int i = idx / chi, j = idx % chi;
      const float val = (i == j && i < nk) ? (float)(s.sig[s.order[i]] / nrm) : 0.f;
      m0[idx] = val; m0[c2 + idx] = 0.f;
      m1[idx] = val; m1[c2 + idx] = 0.f;
    }
  }
}

// ----------------------------------------------------------------------
// The FP32 starting basis of the refined solve for 2 chi > 128, where the
// bond matrix no longer fits in shared memory: the same steps as basis mode of
// solve32_kernel, with G_w, its Cholesky factor and K^T in the edge's global
// workspace (L2-resident) and a round-robin pair order.  One CTA of
// kGThreads threads per edge.
constexpr int kGThreads = 512;
constexpr int kGMaxN = 512;           // 2 chi <= 512 (chi <= 256)
constexpr int kGVals = kGMaxN / 32;   // row values per lane

__global__ void __launch_bounds__(kGThreads, 1) basis_gmem_kernel(SolveArgs a) {
  __shared__ double sig[kGMaxN];
  __shared__ int order[kGMaxN], perm_w[kGMaxN], src[kGMaxN];
  __shared__ float2 colk[kGMaxN];
  __shared__ int counter[4], red_i[4], rank_s[4];
  __shared__ float red_v[4], dmax0[4];
  __shared__ double red_d[kGThreads / 32];
  const int chi = a.chi, n = 2 * chi, half = n / 2;
  const int64_t c2 = (int64_t)chi * chi;
  const int edge = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kGThreads / 32;
  const RefineLayout lay = refine_layout(chi);
  double* rbase = a.work + (int64_t)edge * lay.stride;
  const int* rints = reinterpret_cast<const int*>(rbase + lay.ints);
  const double2* L64 = reinterpret_cast<const double2*>(rbase + lay.L);
  float2* Gw = reinterpret_cast<float2*>(rbase + lay.S);   // n x n: G_w, then L_w
  float2* X = reinterpret_cast<float2*>(rbase + lay.U1);   // n x n: K^T, then its rotations
  const float* gw = a.gram + (int64_t)edge * 8 * c2 + 4 * c2;
  const float sg = (float)a.sign;
  // 1. G_w from conj(N_q^w) with the phases of the gate split (as solve32_kernel)
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    const int ki = i / chi, ei = i % chi, kj = j / chi, ej = j % chi;
    const int64_t o = (int64_t)ei * chi + ej;
    const float2 g0 = make_float2(gw[o], -gw[c2 + o]);
    const float2 g1 = make_float2(gw[2 * c2 + o], -gw[3 * c2 + o]);
    float2 v;
    if (ki == kj) {
      v = make_float2(g0.x + g1.x, g0.y + g1.y);
    } else {
      const float2 d = make_float2(g0.x - g1.x, g0.y - g1.y);
      const float f = (ki == 0) ? -sg : sg;
      v = make_float2(-f * d.y, f * d.x);
    }
    Gw[idx] = v;
  }
  __syncthreads();
  // 2. FP32 pivoted Cholesky of G_w in place (global memory)
  const Group gall{0, kGThreads, 0};
  pivoted_cholesky32(Gw, n, n, perm_w, 1e-7f, &rank_s[2], red_i, red_v, dmax0, colk, gall);
  // 3. K^T[j][(b, i)] = sum_{t' >= i} conj(L_w[src(b, t')][j]) conj(L_b[t'][i]) with
  //    src(b, t') = pinv_w(b chi + perm_b[t']) (as solve32_kernel, R_w = L_w^H P_w^T)
  for (int t = tid; t < n; t += blockDim.x) order[perm_w[t]] = t;  // pinv_w
  __syncthreads();
  for (int bt = tid; bt < n; bt += blockDim.x) {
    const int b = bt / chi, tp = bt % chi;
    src[bt] = order[b * chi + rints[b * chi + tp]];
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int o = idx / n, j = idx % n;   // output column (b, i) = o, row j: consecutive j per warp
    const int b = o / chi, i = o % chi;
    const double2* Lb = L64 + b * c2;
    float2 acc = make_float2(0.f, 0.f);
    for (int tp = i; tp < chi; ++tp) {
      const double2 l = Lb[(int64_t)tp * chi + i];
      const float2 w = Gw[(int64_t)src[b * chi + tp] * n + j];
      // conj(w) conj(l) = conj(w l)
      const float lx = (float)l.x, ly = (float)l.y;
      acc.x += w.x * lx - w.y * ly;
      acc.y -= w.x * ly + w.y * lx;
    }
    X[(int64_t)j * n + o] = acc;
  }
  __syncthreads();
  // 4. One-sided Jacobi on the rows of X (columns of K), round-robin pairs;
  //    pairs orthogonal to orth_tol, or with an overlap below 1e-12 ||K||_F^2,
  //    are left alone; a sweep that rotates nothing ends the iteration
  {
    double acc = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const float2 v = X[idx];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc = warp_sum_d(acc);
    if (lane == 0) red_d[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += red_d[w];
      sig[0] = t;
    }
    __syncthreads();
  }
  const float abs_floor = (float)(kAbsTol * sig[0]);
  const float orth_tol = a.orth_tol > 0.f ? a.orth_tol : 2e-6f;
  const int npl = n / 32;  // n is a multiple of 32 here
  int sweeps = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    ++sweeps;
    if (tid == 0) counter[0] = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      for (int k = warp; k < half; k += nwarps) {
        int p, q;
        if (k == 0) { p = r; q = n - 1; }
        else { p = (r + k) % (n - 1); q = (r - k + (n - 1)) % (n - 1); }
        float2 xp[kGVals], xq[kGVals];
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
        for (int u = 0; u < kGVals; ++u) {
          if (u < npl) {
            const int c = u * 32 + lane;
            xp[u] = X[(int64_t)p * n + c];
            xq[u] = X[(int64_t)q * n + c];
            al += xp[u].x * xp[u].x + xp[u].y * xp[u].y;
            be += xq[u].x * xq[u].x + xq[u].y * xq[u].y;
            gr += xp[u].x * xq[u].x + xp[u].y * xq[u].y;
            gi += xp[u].x * xq[u].y - xp[u].y * xq[u].x;
          }
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const float gm = sqrtf(gr * gr + gi * gi);
        if (gm > orth_tol * sqrtf(al * be) && gm > abs_floor && gm > 0.f) {
          const float2 ph = make_float2(gr / gm, -gi / gm);  // e^{-i phi}
          const float tau = (be - al) / (2.f * gm);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          const float cs = 1.f / sqrtf(1.f + t * t);
          const float sn = t * cs;
#pragma unroll
          for (int u = 0; u < kGVals; ++u) {
            if (u < npl) {
              const int c = u * 32 + lane;
              const float2 pq = cmulf(ph, xq[u]);
              X[(int64_t)p * n + c] = make_float2(cs * xp[u].x - sn * pq.x, cs * xp[u].y - sn * pq.y);
              X[(int64_t)q * n + c] = make_float2(sn * xp[u].x + cs * pq.x, sn * xp[u].y + cs * pq.y);
            }
          }
          if (lane == 0) atomicAdd(&counter[0], 1);
        }
      }
      __syncthreads();
    }
    const int rotated = counter[0];
    __syncthreads();
    if (rotated == 0) break;
  }
  // 5. sigma_j = ||row j|| (FP64), decreasing order, then the basis
  for (int j = warp; j < n; j += nwarps) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) {
      const float2 v = X[(int64_t)j * n + c];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    acc = warp_sum_d(acc);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const double si = sig[i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = sig[j];
      rk += (sj > si) || (sj == si && j < i);
    }
    order[rk] = i;
  }
  __syncthreads();
  Smem sm{};
  sm.sig = sig;
  sm.order = order;
  sm.counter = counter;
  write_basis(a, sm, X, edge, chi, sweeps);
}

size_t smem_bytes(int chi) {
  const int n = 2 * chi;
  return sizeof(float2) * (size_t)n * n + sizeof(float2) * 2 * chi * (chi + 1) +
         sizeof(double) * (n + 4 + 32) + sizeof(double) * 2 * n + sizeof(float2) * n +
         sizeof(int) * (n + 2 * chi + n + n + 4 + 32) + sizeof(float) * (32 + 4) + sizeof(int) * 4 +
         sizeof(float) * n + 64;
}

}  // namespace

bool solve32_supported(int chi) { return chi >= 1 && chi <= kMaxChi; }

cudaError_t launch_basis_gmem(const SolveArgs& a, cudaStream_t st) {
  if (a.n_edges <= 0) return cudaSuccess;
  if (a.chi < 16 || 2 * a.chi > kGMaxN || (2 * a.chi) % 32 != 0) return cudaErrorInvalidValue;
  basis_gmem_kernel<<<a.n_edges, kGThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_solve32(const SolveArgs& a, cudaStream_t st) {
  if (a.n_edges <= 0) return cudaSuccess;
  if (!solve32_supported(a.chi)) return cudaErrorInvalidValue;
  // the shared-memory limit is raised once, to the largest chi's need, so that
  // concurrent launches at different chi (the job server) never lower it
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(solve32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes(kMaxChi));
  });
  if (attr != cudaSuccess) return attr;
  const size_t sm = smem_bytes(a.chi);
  if (!a.basis) {
    solve32_kernel<<<a.n_edges, kThreads, sm, st>>>(a);
    return cudaGetLastError();
  }
  // basis mode follows chol64_kernel on the same stream: a programmatic
  // dependent launch, so that the G_w Cholesky runs while chol64 finishes
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.n_edges);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr_pdl[1];
  attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr_pdl;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, solve32_kernel, a);
}

}  // namespace tnbp
