// BP error estimate of one edge (Methods, "Estimating the error of BP for
// general tensor networks", Eq. BPErrorEstimate): the norm network of the
// state in the symmetric gauge, cut along the edge, is contracted exactly down
// to the chi^2 x chi^2 edge environment E; BP takes E as rank one, and the
// error estimate is 1 - sqrt(s_1^2 / sum_i s_i^2) over E's singular values.
//
// Everything runs on the device in FP64.  The symmetric gauge is the Vidal
// gauge with lambda^1/2 on every leg (tn_vidal_gauge); each site's double-layer
// tensor D_v[(l, l'), ..] = sum_p T[p, l, ..] conj(T[p, l', ..]) keeps only
// the support of each lambda_e (a K = 2 product T^T conj(T), then a
// permutation that interleaves ket and bra legs); the cut edge's index is
// split into a u-side and a w-side label; the network is contracted pairwise,
// always the pair with the smallest result (a greedy order chosen on the
// host from the shapes alone), each contraction a permutation of both
// operands followed by a complex FP64 GEMM; a contraction whose result would
// exceed kMaxElems elements is refused.  The eigenvalues of E^H E (E's
// squared singular values) come from a parallel cyclic Jacobi in one CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "tnbp.h"

struct tn_handle;
namespace tnbp {
void set_error(const std::string& m);  // the thread's tn_last_error message
tn_status gamma_view(tn_handle* h, int v, const float** ptr, int64_t* len, cudaStream_t* stream);
}

namespace {

constexpr int64_t kMaxElems = int64_t(1) << 26;
constexpr int kMaxRank = 24;
constexpr int kJacobiMaxN = 1024;
constexpr int kJacobiSweeps = 60;

#define BPE_TRY(x)                                                       \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess) {                                             \
      tnbp::set_error(std::string("CUDA: ") + cudaGetErrorString(e_));   \
      return TN_ECUDA;                                                   \
    }                                                                    \
  } while (0)

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void zfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

struct PermArgs {
  int rank;
  int64_t dim[kMaxRank];      // output dimensions
  int64_t sstride[kMaxRank];  // source stride of each output index
};

// dst[i_0, .., i_{r-1}] = src[sum_j i_j sstride_j] (row-major output)
__global__ void permute_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                               int64_t total, PermArgs p) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, off = 0;
    for (int j = p.rank - 1; j >= 0; --j) {
      const int64_t d = rem % p.dim[j];
      rem /= p.dim[j];
      off += d * p.sstride[j];
    }
    dst[idx] = src[off];
  }
}

// The weighted site tensor on the bond supports: T[p][s] = prod_j
// lambda_j[l_j]^1/2 Gamma[p][l], s = (l_0 .. l_{d-1}) with l_j < r_j, from
// the planar FP32 Vidal tensor (real plane [p][chi^d], then imaginary plane).
struct SiteArgs {
  int d, chi;
  int r[3];
  const double* lam[3];  // lambda of each leg's edge (chi values)
};
__global__ void site_sub_kernel(const float* __restrict__ gamma, int64_t len, SiteArgs a,
                                double2* __restrict__ T, int64_t sub) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < sub;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = s, full = 0, place = 1;
    double w = 1.0;
    for (int j = a.d - 1; j >= 0; --j) {
      const int l = (int)(rem % a.r[j]);
      rem /= a.r[j];
      full += l * place;
      place *= a.chi;
      w *= sqrt(a.lam[j][l]);
    }
    for (int p = 0; p < 2; ++p) {
      const float re = gamma[(int64_t)p * len + full], im = gamma[2 * len + (int64_t)p * len + full];
      T[(int64_t)p * sub + s] = make_double2(w * re, w * im);
    }
  }
}

// C[m][n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m lda + k], or A[k lda + m]
// when trans_a, conjugated when conj_a; B(k, n) = B[k ldb + n], conjugated
// when conj_b.  32 x 32 output tiles over grid.x, K slices over grid.z
// (partials [slice][m][n] summed by the reduce).
struct ZGemm {
  const double2* A;
  const double2* B;
  double2* C;
  double2* part;
  int64_t m, n, k, lda, ldb;
  int64_t tiles_n, k_per_split;
  int trans_a, conj_a, conj_b, splits;
};
__global__ void __launch_bounds__(256) zgemm_kernel(ZGemm g) {
  __shared__ double2 As[16][33];
  __shared__ double2 Bs[16][33];
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / g.tiles_n) * 32, n0 = (tile % g.tiles_n) * 32;
  const int split = blockIdx.z;
  const int64_t kb = split * g.k_per_split, ke = min(g.k, kb + g.k_per_split);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double2 acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int64_t k0 = kb; k0 < ke; k0 += 16) {
    for (int r = 0; r < 2; ++r) {
      const int e = tid + 256 * r;           // 512 elements of each 16 x 32 slab
      const int kk = e >> 5, mm = e & 31;
      const int64_t k = k0 + kk;
      double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
      if (k < ke) {
        const int64_t m = m0 + mm, n = n0 + mm;
        if (m < g.m) {
          va = g.trans_a ? g.A[k * g.lda + m] : g.A[m * g.lda + k];
          if (g.conj_a) va.y = -va.y;
        }
        if (n < g.n) {
          vb = g.B[k * g.ldb + n];
          if (g.conj_b) vb.y = -vb.y;
        }
      }
      As[kk][mm] = va;
      Bs[kk][mm] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      const double2 a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      zfma(acc[0][0], a0, b0);
      zfma(acc[0][1], a0, b1);
      zfma(acc[1][0], a1, b0);
      zfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= g.m || n >= g.n) continue;
      if (g.splits > 1) g.part[(int64_t)split * g.m * g.n + m * g.n + n] = acc[i][j];
      else g.C[m * g.n + n] = acc[i][j];
    }
}

// C = sum over slices of the partials, in slice order
__global__ void zreduce_kernel(const double2* __restrict__ part, double2* __restrict__ C,
                               int64_t mn, int splits) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mn;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < splits; ++q) {
      const double2 v = part[q * mn + i];
      s.x += v.x;
      s.y += v.y;
    }
    C[i] = s;
  }
}

// Eigenvalues of the Hermitian n x n matrix A (row-major, in place) by the
// cyclic Jacobi method in the parallel (round-robin) order: each round pairs
// every index once, the rotations of one round act on disjoint index pairs
// and are applied together (all column rotations A J, then all row rotations
// J^H A).  The rotation of the pair (p, q) zeroes A[p][q]:
//   e^{-i phi} = conj(A_pq) / |A_pq|, tau = (A_qq - A_pp) / (2 |A_pq|),
//   t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c,
//   columns: a_p <- c a_p - s e^{-i phi} a_q, a_q <- s a_p + c e^{-i phi} a_q,
//   rows with e^{+i phi}.
// Sweeps end when the off-diagonal weight is below 1e-30 of the total, after
// at most kJacobiSweeps sweeps.  One CTA of 1024 threads; ev[i] = A[i][i].
__global__ void __launch_bounds__(1024) herm_jacobi_kernel(double2* A, int n, double* ev) {
  __shared__ double cs_s[kJacobiMaxN / 2 + 1], sn_s[kJacobiMaxN / 2 + 1];
  __shared__ double2 ph_s[kJacobiMaxN / 2 + 1];
  __shared__ int p_s[kJacobiMaxN / 2 + 1], q_s[kJacobiMaxN / 2 + 1];
  __shared__ double red[2][32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = n + (n & 1);  // an odd n pairs with a dummy index n
  const int half = np / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t idx = tid; idx < (int64_t)n * n; idx += nt) {
      const double2 v = A[idx];
      const double a2 = v.x * v.x + v.y * v.y;
      tot += a2;
      if (idx / n != idx % n) off += a2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = off; red[1][tid >> 5] = tot; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { a += red[0][w]; b += red[1][w]; }
      red[0][0] = a;
      red[1][0] = b;
    }
    __syncthreads();
    const bool done = !(red[0][0] > 1e-30 * red[1][0]);
    __syncthreads();
    if (done) break;
    for (int r = 0; r < np - 1; ++r) {
      // pairs of this round and their rotations
      for (int k = tid; k < half; k += nt) {
        int p, q;
        if (k == 0) { p = r; q = np - 1; }
        else { p = (r + k) % (np - 1); q = (r - k + (np - 1)) % (np - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        double2 ph = make_double2(1.0, 0.0);
        if (q < n) {
          const double2 apq = A[(int64_t)p * n + q];
          const double rr = sqrt(apq.x * apq.x + apq.y * apq.y);
          if (rr > 1e-300) {
            const double a = A[(int64_t)p * n + p].x, b = A[(int64_t)q * n + q].x;
            ph = make_double2(apq.x / rr, -apq.y / rr);
            const double tau = (b - a) / (2.0 * rr);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        p_s[k] = p;
        q_s[k] = q;
        cs_s[k] = c;
        sn_s[k] = s;
        ph_s[k] = ph;
      }
      __syncthreads();
      // columns p, q of every row
      for (int64_t idx = tid; idx < (int64_t)half * n; idx += nt) {
        const int k = (int)(idx / n), i = (int)(idx % n);
        const int p = p_s[k], q = q_s[k];
        if (q >= n || sn_s[k] == 0.0) continue;
        const double c = cs_s[k], s = sn_s[k];
        const double2 aip = A[(int64_t)i * n + p], aiq = zmul(ph_s[k], A[(int64_t)i * n + q]);
        A[(int64_t)i * n + p] = make_double2(c * aip.x - s * aiq.x, c * aip.y - s * aiq.y);
        A[(int64_t)i * n + q] = make_double2(s * aip.x + c * aiq.x, s * aip.y + c * aiq.y);
      }
      __syncthreads();
      // rows p, q of every column
      for (int64_t idx = tid; idx < (int64_t)half * n; idx += nt) {
        const int k = (int)(idx / n), j = (int)(idx % n);
        const int p = p_s[k], q = q_s[k];
        if (q >= n || sn_s[k] == 0.0) continue;
        const double c = cs_s[k], s = sn_s[k];
        const double2 phc = make_double2(ph_s[k].x, -ph_s[k].y);
        const double2 apj = A[(int64_t)p * n + j], aqj = zmul(phc, A[(int64_t)q * n + j]);
        A[(int64_t)p * n + j] = make_double2(c * apj.x - s * aqj.x, c * apj.y - s * aqj.y);
        A[(int64_t)q * n + j] = make_double2(s * apj.x + c * aqj.x, s * apj.y + c * aqj.y);
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += nt) ev[i] = A[(int64_t)i * n + i].x;
}

// ------------------------------------------------------------------- host
int grid_for(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

// A device tensor: labels, dimensions, row-major FP64 complex data.
struct DTensor {
  std::vector<int> lab;
  std::vector<int64_t> dim;
  double2* a = nullptr;
  int64_t size() const {
    int64_t s = 1;
    for (int64_t d : dim) s *= d;
    return s;
  }
};

// Device buffers of one tn_bp_error call, freed (stream-ordered) at its end.
struct Pool {
  cudaStream_t s;
  std::vector<void*> live;
  explicit Pool(cudaStream_t st) : s(st) {}
  ~Pool() {
    for (void* p : live) cudaFreeAsync(p, s);
  }
  double2* get(int64_t n) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, sizeof(double2) * (size_t)std::max<int64_t>(n, 1), s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    live.push_back(p);
    return (double2*)p;
  }
  void drop(void* p) {
    auto it = std::find(live.begin(), live.end(), p);
    if (it != live.end()) {
      cudaFreeAsync(p, s);
      live.erase(it);
    }
  }
};

tn_status permute(Pool& pool, const DTensor& t, const std::vector<int>& order, DTensor* out) {
  const int r = (int)order.size();
  if (r > kMaxRank) { tnbp::set_error("a tensor of the norm network has too many indices"); return TN_EINVAL; }
  PermArgs pa{};
  pa.rank = r;
  std::vector<int64_t> st(r, 1);
  for (int i = r - 2; i >= 0; --i) st[i] = st[i + 1] * t.dim[i + 1];
  out->lab.resize(r);
  out->dim.resize(r);
  for (int i = 0; i < r; ++i) {
    out->lab[i] = t.lab[order[i]];
    out->dim[i] = t.dim[order[i]];
    pa.dim[i] = t.dim[order[i]];
    pa.sstride[i] = st[order[i]];
  }
  const int64_t n = t.size();
  out->a = pool.get(n);
  if (!out->a) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
  if (r == 0 || n == 0) {
    BPE_TRY(cudaMemcpyAsync(out->a, t.a, sizeof(double2) * std::max<int64_t>(n, 1),
                            cudaMemcpyDeviceToDevice, pool.s));
    return TN_OK;
  }
  permute_kernel<<<grid_for(n), 256, 0, pool.s>>>(t.a, out->a, n, pa);
  BPE_TRY(cudaGetLastError());
  return TN_OK;
}

tn_status zgemm(Pool& pool, const double2* A, const double2* B, double2* C, int64_t m, int64_t n,
                int64_t k, int64_t lda, int64_t ldb, bool trans_a, bool conj_a, bool conj_b) {
  ZGemm g{};
  g.A = A; g.B = B; g.C = C;
  g.m = m; g.n = n; g.k = k; g.lda = lda; g.ldb = ldb;
  g.trans_a = trans_a; g.conj_a = conj_a; g.conj_b = conj_b;
  g.tiles_n = (n + 31) / 32;
  const int64_t tiles = ((m + 31) / 32) * g.tiles_n;
  // a grid under one wave with a long K: slices of at least 1024 K values
  int splits = 1;
  while (splits < 64 && tiles * splits * 2 <= 2 * 152 && k / (2 * splits) >= 1024) splits *= 2;
  g.splits = splits;
  g.k_per_split = ((k + splits - 1) / splits + 15) / 16 * 16;
  if (splits > 1) {
    g.part = pool.get((int64_t)splits * m * n);
    if (!g.part) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
  }
  if (tiles > 0x7fffffffLL) { tnbp::set_error("contraction too large"); return TN_EINVAL; }
  zgemm_kernel<<<dim3((unsigned)tiles, 1, splits), 256, 0, pool.s>>>(g);
  BPE_TRY(cudaGetLastError());
  if (splits > 1) {
    zreduce_kernel<<<grid_for(m * n), 256, 0, pool.s>>>(g.part, C, m * n, splits);
    BPE_TRY(cudaGetLastError());
    pool.drop(g.part);
  }
  return TN_OK;
}

// Contract the labels x and y share: result indices x-only then y-only.
tn_status contract(Pool& pool, const DTensor& x, const DTensor& y, DTensor* out) {
  std::vector<int> xs, xk, ys, yk;
  for (int i = 0; i < (int)x.lab.size(); ++i) {
    const auto it = std::find(y.lab.begin(), y.lab.end(), x.lab[i]);
    (it == y.lab.end() ? xk : xs).push_back(i);
  }
  for (int s : xs) ys.push_back((int)(std::find(y.lab.begin(), y.lab.end(), x.lab[s]) - y.lab.begin()));
  for (int i = 0; i < (int)y.lab.size(); ++i)
    if (std::find(ys.begin(), ys.end(), i) == ys.end()) yk.push_back(i);
  std::vector<int> ox(xk), oy(ys);
  ox.insert(ox.end(), xs.begin(), xs.end());
  oy.insert(oy.end(), yk.begin(), yk.end());
  DTensor px, py;
  tn_status st = permute(pool, x, ox, &px);
  if (st) return st;
  st = permute(pool, y, oy, &py);
  if (st) return st;
  int64_t m = 1, k = 1, n = 1;
  for (int i : xk) m *= x.dim[i];
  for (int i : xs) k *= x.dim[i];
  for (int i : yk) n *= y.dim[i];
  out->lab.clear();
  out->dim.clear();
  for (int i : xk) { out->lab.push_back(x.lab[i]); out->dim.push_back(x.dim[i]); }
  for (int i : yk) { out->lab.push_back(y.lab[i]); out->dim.push_back(y.dim[i]); }
  out->a = pool.get(m * n);
  if (!out->a) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
  st = zgemm(pool, px.a, py.a, out->a, m, n, k, k, n, false, false, false);
  pool.drop(px.a);
  pool.drop(py.a);
  return st;
}

int64_t result_size(const DTensor& x, const DTensor& y) {
  int64_t s = 1;
  for (size_t i = 0; i < x.lab.size(); ++i)
    if (std::find(y.lab.begin(), y.lab.end(), x.lab[i]) == y.lab.end()) s *= x.dim[i];
  for (size_t i = 0; i < y.lab.size(); ++i)
    if (std::find(x.lab.begin(), x.lab.end(), y.lab[i]) == x.lab.end()) s *= y.dim[i];
  return s;
}

bool shares(const DTensor& x, const DTensor& y) {
  for (int l : x.lab)
    if (std::find(y.lab.begin(), y.lab.end(), l) != y.lab.end()) return true;
  return false;
}

tn_status bp_error_impl(tn_handle* h, int32_t e, double* error, double* sv_out, int32_t sv_capacity,
                        int32_t* n_sv) {
  int32_t n = 0, m = 0, chi = 0;
  tn_status st = tn_graph_info(h, &n, &m, &chi, nullptr, 0);
  if (st) return st;
  if (e < 0 || e >= m) { tnbp::set_error("edge out of range"); return TN_EINVAL; }
  std::vector<int32_t> edges(2 * (size_t)m);
  st = tn_graph_info(h, &n, &m, &chi, edges.data(), m);
  if (st) return st;
  std::vector<double> lam((size_t)m * chi);
  st = tn_vidal_gauge(h, lam.data());
  if (st) return st;
  // support of each bond and the legs of each site in increasing edge id
  std::vector<int> rsup(m, 0);
  for (int f = 0; f < m; ++f)
    for (int k = 0; k < chi; ++k)
      if (lam[(size_t)f * chi + k] > 0.0) rsup[f] = k + 1;
  std::vector<std::vector<int>> legs(n);
  for (int f = 0; f < m; ++f) {
    legs[edges[2 * f]].push_back(f);
    legs[edges[2 * f + 1]].push_back(f);
  }
  // the double-layer tensors together stay within 2 x kMaxElems elements
  {
    double total = 0.0;
    for (int v = 0; v < n; ++v) {
      double sz = 1.0;
      for (int f : legs[v]) sz *= (double)rsup[f] * rsup[f];
      total += sz;
    }
    if (total > 2.0 * (double)kMaxElems) {
      tnbp::set_error("the norm network is too large to contract exactly");
      return TN_EINVAL;
    }
  }
  for (int v = 0; v < n; ++v)
    if (legs[v].size() > 3) { tnbp::set_error("vertex degree above 3"); return TN_EINVAL; }
  const float* g0 = nullptr;
  int64_t len0 = 0;
  cudaStream_t stream = nullptr;
  st = tnbp::gamma_view(h, 0, &g0, &len0, &stream);
  if (st) return st;
  Pool pool(stream);
  double* dlam = nullptr;
  {
    void* p = nullptr;
    BPE_TRY(cudaMallocAsync(&p, sizeof(double) * lam.size() + 8 * kJacobiMaxN, stream));
    pool.live.push_back(p);
    dlam = (double*)p;
    BPE_TRY(cudaMemcpyAsync(dlam, lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice,
                            stream));
  }
  std::vector<DTensor> net;
  for (int v = 0; v < n; ++v) {
    const int d = (int)legs[v].size();
    const float* gam = nullptr;
    int64_t len = 0;
    st = tnbp::gamma_view(h, v, &gam, &len, &stream);
    if (st) return st;
    SiteArgs sa{};
    sa.d = d;
    sa.chi = chi;
    int64_t sub = 1;
    for (int j = 0; j < d; ++j) {
      sa.r[j] = rsup[legs[v][j]];
      sa.lam[j] = dlam + (size_t)legs[v][j] * chi;
      sub *= sa.r[j];
    }
    if (sub * sub > kMaxElems) {
      tnbp::set_error("a site's double-layer tensor is too large to contract exactly");
      return TN_EINVAL;
    }
    double2* T = pool.get(2 * sub);
    if (!T) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
    site_sub_kernel<<<grid_for(sub), 256, 0, stream>>>(gam, len, sa, T, sub);
    BPE_TRY(cudaGetLastError());
    // Dm[s1][s2] = sum_p T[p][s1] conj(T[p][s2]), then (l_1..l_d, l_1'..l_d') ->
    // (l_1, l_1', .., l_d, l_d')
    DTensor Dm;
    Dm.a = pool.get(sub * sub);
    if (!Dm.a) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
    st = zgemm(pool, T, T, Dm.a, sub, sub, 2, sub, sub, true, false, true);
    if (st) return st;
    pool.drop(T);
    for (int j = 0; j < d; ++j) { Dm.lab.push_back(j); Dm.dim.push_back(sa.r[j]); }
    for (int j = 0; j < d; ++j) { Dm.lab.push_back(d + j); Dm.dim.push_back(sa.r[j]); }
    std::vector<int> order;
    for (int j = 0; j < d; ++j) { order.push_back(j); order.push_back(d + j); }
    DTensor Dp;
    st = permute(pool, Dm, order, &Dp);
    if (st) return st;
    pool.drop(Dm.a);
    DTensor D;
    D.a = Dp.a;
    for (int j = 0; j < d; ++j) {
      const int f = legs[v][j];
      D.lab.push_back(f == e ? (edges[2 * f] == v ? m : m + 1) : f);
      D.dim.push_back((int64_t)sa.r[j] * sa.r[j]);
    }
    net.push_back(D);
  }
  // greedy pairwise contraction
  while (net.size() > 1) {
    int bi = -1, bj = -1;
    int64_t best = -1;
    for (int i = 0; i < (int)net.size(); ++i)
      for (int j = i + 1; j < (int)net.size(); ++j) {
        if (!shares(net[i], net[j])) continue;
        const int64_t s = result_size(net[i], net[j]);
        if (best < 0 || s < best) { best = s; bi = i; bj = j; }
      }
    if (bi < 0) {  // disconnected: join the two smallest by an outer product
      std::vector<int> o(net.size());
      std::iota(o.begin(), o.end(), 0);
      std::sort(o.begin(), o.end(), [&](int a, int b) { return net[a].size() < net[b].size(); });
      bi = std::min(o[0], o[1]);
      bj = std::max(o[0], o[1]);
      best = net[bi].size() * net[bj].size();
    }
    if (best > kMaxElems) {
      tnbp::set_error("the cut norm network is too large to contract exactly (an intermediate "
                      "above 2^26 elements)");
      return TN_EINVAL;
    }
    DTensor c;
    st = contract(pool, net[bi], net[bj], &c);
    if (st) return st;
    pool.drop(net[bi].a);
    pool.drop(net[bj].a);
    net.erase(net.begin() + bj);
    net[bi] = c;
  }
  // E[(u side), (w side)]
  DTensor E = net[0];
  if (E.lab.size() != 2) { tnbp::set_error("the edge environment lost its cut indices"); return TN_EINVAL; }
  if (E.lab[0] != m) {
    DTensor t;
    st = permute(pool, E, {1, 0}, &t);
    if (st) return st;
    E = t;
  }
  const int64_t ru = E.dim[0], rw = E.dim[1];
  if (rw > kJacobiMaxN) {
    tnbp::set_error("edge environment with more than 1024 columns (the cut bond's index on the "
                    "edge's second endpoint, ket x bra)");
    return TN_EINVAL;
  }
  // H = E^H E (rw x rw), its eigenvalues s_i^2
  double2* H = pool.get(rw * rw);
  if (!H) { tnbp::set_error("device allocation of the norm network failed"); return TN_ENOMEM; }
  st = zgemm(pool, E.a, E.a, H, rw, rw, ru, rw, rw, true, true, false);
  if (st) return st;
  double* dev = dlam + lam.size();
  herm_jacobi_kernel<<<1, 1024, 0, stream>>>(H, (int)rw, dev);
  BPE_TRY(cudaGetLastError());
  std::vector<double> ev(rw);
  BPE_TRY(cudaMemcpyAsync(ev.data(), dev, sizeof(double) * rw, cudaMemcpyDeviceToHost, stream));
  BPE_TRY(cudaStreamSynchronize(stream));
  std::sort(ev.begin(), ev.end(), std::greater<double>());
  double tot = 0.0;
  for (double x : ev) tot += std::max(x, 0.0);
  if (!(tot > 0.0) || !std::isfinite(tot)) {
    tnbp::set_error("the edge environment vanishes or is not finite");
    return TN_ENUMERIC;
  }
  *error = 1.0 - std::sqrt(std::max(ev[0], 0.0) / tot);
  if (n_sv) *n_sv = (int32_t)rw;
  if (sv_out)
    for (int i = 0; i < sv_capacity && i < (int)rw; ++i) sv_out[i] = std::sqrt(std::max(ev[i], 0.0));
  return TN_OK;
}

}  // namespace

extern "C" tn_status tn_bp_error(tn_handle* h, int32_t e, double* error, double* sv_out,
                                 int32_t sv_capacity, int32_t* n_sv) {
  if (!h || !error) { tnbp::set_error("null argument"); return TN_EINVAL; }
  return bp_error_impl(h, e, error, sv_out, sv_capacity, n_sv);
}
