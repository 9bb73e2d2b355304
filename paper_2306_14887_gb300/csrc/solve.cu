// FP64 truncation solve of the BP-gauged simple update (Methods, "The simple
// update procedure", and the reduced-tensor/message formulation it cites).
//
// For a gate edge e = (v, w) the inputs are the open-p environment matrices of
// both sides, N_p[e, e'] = sum T[p, .., e, ..] conj(T[p, .., e', ..]) prod_x M_{x->*}
// (the BP message contraction with the physical index left open).  With the
// gate split exp(s i pi/4 ZZ) = sum_k A_k (x) B_k, A_0 = B_0 = 2^-1/4 I,
// A_1 = 2^-1/4 Z, B_1 = s i 2^-1/4 Z, the env-weighted two-site matrix is
// Theta = Xv Xw^T with Xv[(p, rest), (k, e)] = a_k(p) X_v[p, rest, e], so the
// Gram matrices G_v = Xv^H Xv and G_w = Xw^H Xw (2chi x 2chi) are fixed by the
// N_p alone.  The solve, all in FP64:
//   G_v = W diag(lam) W^H                    (Hermitian Jacobi)
//   R_v = diag(lam)^1/2 W^H,  H = R_v conj(G_w) R_v^H = U diag(sigma^2) U^H
//   keep the chi largest sigma (above svd_cut * sigma_1), S = sigma / ||sigma||
//   C_v = W lam^-1/2 U sqrt(S),  C_w = conj(W) lam^1/2 conj(U) / sqrt(sigma ||sigma||)
// so that Xv C_v and Xw C_w are the two halves of the truncated SVD of Theta
// (H = K K^H for the bond matrix K = R_v R_w^T).  The outputs are the per-p
// chi x chi matrices D_v[p] = sum_k a_k(p) C_v[k], D_w[q] = sum_k b_k(q) C_w[k]
// that the rebuild contracts into the gate leg, and the new messages
// M_{v->w} = M_{w->v} = diag(S).
#include <math.h>

#include "common.cuh"
#include "tnbp.h"

namespace tnbp {

namespace {

struct cd { double x, y; };
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.x, -a.y}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }

__device__ double block_reduce_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

constexpr int kMaxN = 512;  // 2 * chi for chi <= 256

// Cyclic Jacobi for a Hermitian n x n matrix A (row-major, destroyed: its
// diagonal ends up holding the eigenvalues).  V receives the eigenvectors as
// columns.  The n/2 disjoint rotations of one round-robin round are applied
// together: all column updates (A J, V J), then all row updates (J^H A).
__device__ int jacobi_eig(cd* A, cd* V, int n, int max_sweeps, double* sh,
                          double* rc, double* rs, cd* rph) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    V[idx] = {i == j ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  const int half = n / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      const double a2 = A[idx].x * A[idx].x + A[idx].y * A[idx].y;
      if (i == j) dg += a2; else off += a2;
    }
    off = block_reduce_sum(off, sh);
    dg = block_reduce_sum(dg, sh);
    if (off <= 1e-30 * (dg + off) || off == 0.0) break;
    for (int r = 0; r < n - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = r; q = n - 1; }
        else { p = (r + k) % (n - 1); q = (r - k + (n - 1)) % (n - 1); }
        const double a = A[p * n + p].x, b = A[q * n + q].x;
        const cd c = A[p * n + q];
        const double rr = sqrt(c.x * c.x + c.y * c.y);
        double cs = 1.0, sn = 0.0;
        cd ph = {1.0, 0.0};
        if (rr > 1e-300 && rr > 1e-18 * (fabs(a) + fabs(b))) {
          ph = {c.x / rr, -c.y / rr};  // e^{-i phi}
          const double tau = (b - a) / (2.0 * rr);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          cs = 1.0 / sqrt(1.0 + t * t);
          sn = t * cs;
        }
        rc[k] = cs;
        rs[k] = sn;
        rph[k] = ph;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < half * n; w += blockDim.x) {
        const int k = w / n, i = w - k * n;
        int p, q;
        if (k == 0) { p = r; q = n - 1; }
        else { p = (r + k) % (n - 1); q = (r - k + (n - 1)) % (n - 1); }
        const double cs = rc[k], sn = rs[k];
        const cd ph = rph[k];
        const cd aip = A[i * n + p], aiq = cmul(ph, A[i * n + q]);
        A[i * n + p] = {cs * aip.x - sn * aiq.x, cs * aip.y - sn * aiq.y};
        A[i * n + q] = {sn * aip.x + cs * aiq.x, sn * aip.y + cs * aiq.y};
        const cd vip = V[i * n + p], viq = cmul(ph, V[i * n + q]);
        V[i * n + p] = {cs * vip.x - sn * viq.x, cs * vip.y - sn * viq.y};
        V[i * n + q] = {sn * vip.x + cs * viq.x, sn * vip.y + cs * viq.y};
      }
      __syncthreads();
      for (int w = threadIdx.x; w < half * n; w += blockDim.x) {
        const int k = w / n, j = w - k * n;
        int p, q;
        if (k == 0) { p = r; q = n - 1; }
        else { p = (r + k) % (n - 1); q = (r - k + (n - 1)) % (n - 1); }
        const double cs = rc[k], sn = rs[k];
        const cd phc = cconj(rph[k]);
        const cd apj = A[p * n + j], aqj = cmul(phc, A[q * n + j]);
        A[p * n + j] = {cs * apj.x - sn * aqj.x, cs * apj.y - sn * aqj.y};
        A[q * n + j] = {sn * apj.x + cs * aqj.x, sn * apj.y + cs * aqj.y};
      }
      __syncthreads();
    }
  }
  return sweep;  // rotation sweeps performed
}

// Sort eigenpairs by decreasing eigenvalue: lam[r] and column r of Vout.
__device__ void sort_eig(const cd* A, const cd* V, cd* Vout, int n, double* lam, int* perm) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = A[i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j * n + j].x;
      rank += (lj > li) || (lj == li && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = A[perm[i] * n + perm[i]].x;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, r = idx - i * n;
    Vout[idx] = V[i * n + perm[r]];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) solve_kernel(SolveArgs a) {
  __shared__ double sh[32];
  __shared__ double rc[kMaxN / 2], rs[kMaxN / 2];
  __shared__ cd rph[kMaxN / 2];
  __shared__ double lam[kMaxN], sig[kMaxN];
  __shared__ int perm[kMaxN];
  __shared__ double scal[4];

  const int edge = blockIdx.x;
  const int chi = a.chi, n = 2 * chi;
  const int64_t c2 = (int64_t)chi * chi;
  cd* base = reinterpret_cast<cd*>(a.work + (int64_t)edge * 12 * n * n);
  cd* Gv = base;
  cd* W = base + n * n;
  cd* Gw = base + 2 * n * n;
  cd* Z = base + 3 * n * n;
  cd* H = base + 4 * n * n;
  cd* U = base + 5 * n * n;
  const float* gv = a.gram + (int64_t)edge * 8 * c2;
  const float* gw = gv + 4 * c2;
  const double r2 = 0.70710678118654752440;  // (2^-1/4)^2
  const double sg = (double)a.sign;

  // 1. Gram matrices from the open-p environments (G_p = conj(N_p)).
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    const int ki = i / chi, ei = i - ki * chi, kj = j / chi, ej = j - kj * chi;
    const int64_t o = (int64_t)ei * chi + ej;
    const cd v0 = {gv[o], -gv[c2 + o]}, v1 = {gv[2 * c2 + o], -gv[3 * c2 + o]};
    const cd w0 = {gw[o], -gw[c2 + o]}, w1 = {gw[2 * c2 + o], -gw[3 * c2 + o]};
    const cd vs = cadd(v0, v1), vd = {v0.x - v1.x, v0.y - v1.y};
    Gv[idx] = cscale(((ki + kj) & 1) ? vd : vs, r2);
    const cd ws = cadd(w0, w1), wd = {w0.x - w1.x, w0.y - w1.y};
    cd g;
    if (ki == kj) g = ws;
    else if (ki == 0) g = {-sg * wd.y, sg * wd.x};   // +s i (G0 - G1)
    else g = {sg * wd.y, -sg * wd.x};                // -s i (G0 - G1)
    Gw[idx] = cscale(g, r2);
  }
  __syncthreads();

  // 2. G_v = W lam W^H.
  const int sweeps_v = jacobi_eig(Gv, Z, n, a.max_sweeps, sh, rc, rs, rph);
  sort_eig(Gv, Z, W, n, lam, perm);
  const double lmax = lam[0] > 0.0 ? lam[0] : 0.0;
  const double lcut = a.gram_cut * lmax;

  // 3. Z = conj(G_w) W ;  H = diag(lam)^1/2 W^H Z diag(lam)^1/2 on kept indices.
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    cd acc = {0.0, 0.0};
    for (int k = 0; k < n; ++k) acc = cadd(acc, cmul(cconj(Gw[i * n + k]), W[k * n + j]));
    Z[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    cd acc = {0.0, 0.0};
    if (lam[i] > lcut && lam[j] > lcut && lmax > 0.0) {
      for (int k = 0; k < n; ++k) acc = cadd(acc, cmul(cconj(W[k * n + i]), Z[k * n + j]));
      acc = cscale(acc, sqrt(lam[i] * lam[j]));
    }
    H[idx] = acc;
  }
  __syncthreads();
  // Hermitise H exactly before the eigen-solve.
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    if (i < j) {
      const cd hij = H[idx], hji = H[j * n + i];
      const cd m = {0.5 * (hij.x + hji.x), 0.5 * (hij.y - hji.y)};
      H[idx] = m;
      H[j * n + i] = cconj(m);
    } else if (i == j) {
      H[idx].y = 0.0;
    }
  }
  __syncthreads();

  // 4. H = U diag(sigma^2) U^H.
  const int sweeps_h = jacobi_eig(H, Z, n, a.max_sweeps, sh, rc, rs, rph);
  sort_eig(H, Z, U, n, sig, perm);

  // 5. Truncation to chi and normalisation (thread 0; n <= 512 values).
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += sig[i] > 0.0 ? sig[i] : 0.0;
    const double s0 = sig[0] > 0.0 ? sqrt(sig[0]) : 0.0;
    double kept = 0.0;
    int nk = 0;
    for (int i = 0; i < n; ++i) {
      const double s = (sig[i] > 0.0) ? sqrt(sig[i]) : 0.0;
      const bool keep = i < chi && s > 0.0 && s > a.svd_cut * s0;
      sig[i] = keep ? s : 0.0;
      if (keep) { kept += s * s; ++nk; }
    }
    const double nrm = sqrt(kept);
    scal[0] = nrm;
    double* st = a.stats + 4 * edge;
    st[0] = tot > 0.0 ? (tot - kept) / tot : 0.0;
    st[1] = nk;
    st[2] = s0;
    st[3] = sweeps_v + sweeps_h;
    if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(a.flags, 1);
  }
  __syncthreads();
  const double nrm = scal[0];
  const bool ok = nrm > 0.0 && isfinite(nrm);

  // 6. D_v[p][e][n], D_w[q][e][n] (FP32 planar) and the new messages diag(S).
  float* dv = a.dmat + (int64_t)edge * 8 * c2;
  float* dw = dv + 4 * c2;
  const double r = 0.84089641525371454303;  // 2^-1/4
  for (int idx = threadIdx.x; idx < chi * chi; idx += blockDim.x) {
    const int e = idx / chi, m = idx - e * chi;
    cd v0 = {0, 0}, v1 = {0, 0}, w0 = {0, 0}, w1 = {0, 0};
    if (ok && sig[m] > 0.0) {
      const double fv = sqrt(sig[m] / nrm);
      const double fw = 1.0 / sqrt(sig[m] * nrm);
      cd sv0 = {0, 0}, sv1 = {0, 0}, sw0 = {0, 0}, sw1 = {0, 0};
      for (int i = 0; i < n; ++i) {
        if (!(lam[i] > lcut) || !(lmax > 0.0)) continue;
        const double li = sqrt(lam[i]);
        const cd u = U[i * n + m];
        const cd cv = cscale(u, 1.0 / li);
        const cd cw = cscale(cconj(u), li);
        sv0 = cadd(sv0, cmul(W[e * n + i], cv));
        sv1 = cadd(sv1, cmul(W[(chi + e) * n + i], cv));
        sw0 = cadd(sw0, cmul(cconj(W[e * n + i]), cw));
        sw1 = cadd(sw1, cmul(cconj(W[(chi + e) * n + i]), cw));
      }
      // C_v[(k,e)][m] = sv_k * fv ; D_v[p] = r (C_v[0] + s_p C_v[1])
      v0 = cscale(cadd(sv0, sv1), r * fv);
      v1 = cscale({sv0.x - sv1.x, sv0.y - sv1.y}, r * fv);
      // D_w[q] = r (C_w[0] + s i s_q C_w[1])
      const cd isw1 = {-sg * sw1.y, sg * sw1.x};
      w0 = cscale(cadd(sw0, isw1), r * fw);
      w1 = cscale({sw0.x - isw1.x, sw0.y - isw1.y}, r * fw);
    }
    const int64_t o = (int64_t)e * chi + m;
    dv[o] = (float)v0.x; dv[c2 + o] = (float)v0.y;
    dv[2 * c2 + o] = (float)v1.x; dv[3 * c2 + o] = (float)v1.y;
    dw[o] = (float)w0.x; dw[c2 + o] = (float)w0.y;
    dw[2 * c2 + o] = (float)w1.x; dw[3 * c2 + o] = (float)w1.y;
  }
  if (a.s_out) {
    for (int i = threadIdx.x; i < chi; i += blockDim.x)
      a.s_out[(int64_t)edge * chi + i] = ok ? sig[i] / nrm : 0.0;
  }
  if (ok && a.msg) {
    float* m0 = a.msg + (int64_t)a.msg_vw[2 * edge] * 2 * c2;
    float* m1 = a.msg + (int64_t)a.msg_vw[2 * edge + 1] * 2 * c2;
    for (int idx = threadIdx.x; idx < chi * chi; idx += blockDim.x) {
      const int i = idx / chi, j = idx - i * chi;
      const float val = (i == j) ? (float)(sig[i] / nrm) : 0.f;
      m0[idx] = val; m0[c2 + idx] = 0.f;
      m1[idx] = val; m1[c2 + idx] = 0.f;
    }
  }
}

// Vidal gauge of one edge e = (u, w) from its two converged BP messages
// (Methods, "The Vidal gauge": at the BP fixed point the messages define the
// gauge transformation).  With P = sqrt(M_{u->w}), Q = sqrt(M_{w->u}) (the
// Hermitian square roots of the messages u and w send across e) and the SVD
// Q^T P = U diag(lambda) V^H, the bond matrices A = Q conj(U) lambda^-1/2 on
// u's leg and B = P V lambda^-1/2 on w's leg satisfy A B^T = 1 on the
// messages' support and turn both messages into diag(lambda).  The leg
// matrices written out carry one more lambda^-1/2, so that contracting them
// into the site tensors gives Gamma (T_v = Gamma_v with lambda^1/2 on every
// leg): G_u = Q conj(U) / lambda, G_w = P V / lambda, FP32 planar
// [side][re|im][i][k], and lambda / ||lambda||_2 (FP64, decreasing, zero past
// the support).  The SVD is taken as the eigen-decomposition of Z^H Z, Z =
// Q^T P, all in FP64; lambda below 1e-12 lambda_1 counts as zero.
__global__ void __launch_bounds__(256) vidal_edge_kernel(const float* msg, const int32_t* dir,
                                                         int chi, double* work, float* gout,
                                                         double* lam_out, int* flags) {
  __shared__ double sh[32];
  __shared__ double rc[kMaxN / 2], rs[kMaxN / 2];
  __shared__ cd rph[kMaxN / 2];
  __shared__ double lam[kMaxN];
  __shared__ int perm[kMaxN];
  __shared__ double scal[2];
  // the round-robin Jacobi pairs an even number of indices: odd chi is padded
  // with one zero row and column (one more zero singular value, sorted last)
  const int e = blockIdx.x, n = chi + (chi & 1);
  const int64_t c2 = (int64_t)chi * chi, nn = (int64_t)n * n;
  cd* base = reinterpret_cast<cd*>(work + (int64_t)e * 12 * nn);
  cd* A = base;
  cd* V = base + nn;
  cd* Vs = base + 2 * nn;
  cd* P = base + 3 * nn;
  cd* Q = base + 4 * nn;
  cd* Z = base + 5 * nn;
  // 1. Hermitian square roots of the two messages: side 0 (u -> w) into P,
  //    side 1 (w -> u) into Q.
  for (int side = 0; side < 2; ++side) {
    const float* m = msg + (int64_t)dir[2 * e + side] * 2 * c2;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      cd a = {0.0, 0.0};
      if (i < chi && j < chi) {
        const int64_t o = (int64_t)i * chi + j, t = (int64_t)j * chi + i;
        a = {0.5 * ((double)m[o] + (double)m[t]), 0.5 * ((double)m[c2 + o] - (double)m[c2 + t])};
      }
      A[idx] = a;
    }
    __syncthreads();
    jacobi_eig(A, V, n, 40, sh, rc, rs, rph);
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int i = 0; i < n; ++i) mx = fmax(mx, A[i * n + i].x);
      scal[0] = mx;
    }
    __syncthreads();
    const double cut = 1e-14 * scal[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = A[i * n + i].x;
      lam[i] = d > cut ? sqrt(d) : 0.0;
    }
    __syncthreads();
    cd* S = side == 0 ? P : Q;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      const int i = idx / n, j = idx - i * n;
      cd acc = {0.0, 0.0};
      for (int k = 0; k < n; ++k)
        if (lam[k] > 0.0) acc = cadd(acc, cscale(cmul(V[i * n + k], cconj(V[j * n + k])), lam[k]));
      S[idx] = acc;
    }
    __syncthreads();
  }
  // 2. Z = Q^T P; A = Z^H Z (Hermitised exactly) = V diag(lambda^2) V^H.
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    cd acc = {0.0, 0.0};
    for (int k = 0; k < n; ++k) acc = cadd(acc, cmul(Q[k * n + i], P[k * n + j]));
    Z[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    cd acc = {0.0, 0.0};
    if (i <= j)
      for (int k = 0; k < n; ++k) acc = cadd(acc, cmul(cconj(Z[k * n + i]), Z[k * n + j]));
    A[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    if (i > j) A[idx] = cconj(A[j * n + i]);
    else if (i == j) A[idx].y = 0.0;
  }
  __syncthreads();
  jacobi_eig(A, V, n, 40, sh, rc, rs, rph);
  sort_eig(A, V, Vs, n, lam, perm);
  if (threadIdx.x == 0) {
    const double l0 = lam[0] > 0.0 ? sqrt(lam[0]) : 0.0;
    double nrm2 = 0.0;
    for (int k = 0; k < n; ++k) {
      const double l = lam[k] > 0.0 ? sqrt(lam[k]) : 0.0;
      lam[k] = (l0 > 0.0 && l > 1e-12 * l0) ? l : 0.0;
      nrm2 += lam[k] * lam[k];
    }
    scal[1] = sqrt(nrm2);
    if (!(scal[1] > 0.0) || !isfinite(scal[1])) atomicOr(flags, 1);
  }
  __syncthreads();
  // 3. U = Z V / lambda (into A); G_u = Q conj(U) / lambda, G_w = P V / lambda.
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i = idx / n, k = idx - i * n;
    cd acc = {0.0, 0.0};
    if (lam[k] > 0.0) {
      for (int j = 0; j < n; ++j) acc = cadd(acc, cmul(Z[i * n + j], Vs[j * n + k]));
      acc = cscale(acc, 1.0 / lam[k]);
    }
    A[idx] = acc;
  }
  __syncthreads();
  float* gu = gout + (int64_t)e * 4 * c2;
  float* gw = gu + 2 * c2;
  for (int idx = threadIdx.x; idx < c2; idx += blockDim.x) {
    const int i = idx / chi, k = idx - i * chi;
    cd au = {0.0, 0.0}, aw = {0.0, 0.0};
    if (lam[k] > 0.0) {
      for (int j = 0; j < n; ++j) {
        au = cadd(au, cmul(Q[i * n + j], cconj(A[j * n + k])));
        aw = cadd(aw, cmul(P[i * n + j], Vs[j * n + k]));
      }
      au = cscale(au, 1.0 / lam[k]);
      aw = cscale(aw, 1.0 / lam[k]);
    }
    gu[idx] = (float)au.x; gu[c2 + idx] = (float)au.y;
    gw[idx] = (float)aw.x; gw[c2 + idx] = (float)aw.y;
  }
  const double nrm = scal[1];
  for (int k = threadIdx.x; k < chi; k += blockDim.x)
    lam_out[(int64_t)e * chi + k] = nrm > 0.0 ? lam[k] / nrm : 0.0;
}

}  // namespace

size_t solve_work_doubles(int chi) { return (size_t)12 * (2 * chi) * (2 * chi); }

cudaError_t launch_solve(const SolveArgs& a, cudaStream_t s) {
  if (a.n_edges <= 0) return cudaSuccess;
  if (2 * a.chi > kMaxN) return cudaErrorInvalidValue;
  solve_kernel<<<a.n_edges, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tnbp

namespace tnbp {

size_t vidal_work_doubles(int chi) {
  const size_t n = (size_t)(chi + (chi & 1));
  return 12 * n * n;
}

cudaError_t launch_vidal_edges(const float* msg, const int32_t* dir, int n_edges, int chi,
                               double* work, float* gout, double* lam_out, int* flags,
                               cudaStream_t s) {
  if (n_edges <= 0) return cudaSuccess;
  if (chi + 1 > kMaxN) return cudaErrorInvalidValue;
  vidal_edge_kernel<<<n_edges, 256, 0, s>>>(msg, dir, chi, work, gout, lam_out, flags);
  return cudaGetLastError();
}

}  // namespace tnbp
