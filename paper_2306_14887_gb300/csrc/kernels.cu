// CUDA-core kernels of the tnbp library: the plain-FP32 batched complex GEMM
// that carries every contraction of the message and gate updates in the
// TN_FP32 mode, the physical-leg gate, message normalisation with the FP64
// residual, the single-site reduced density matrix and a batched block copy.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tnbp.h"

namespace tnbp {

// ---------------------------------------------------------------------------
// Plain FP32 complex GEMM, 64 x 64 output tile per CTA, 16-deep K slices
// staged in shared memory, 4 x 4 complex outputs per thread (planar re/im
// accumulators).  Operand loads pick the thread-to-element map that makes
// consecutive threads read consecutive addresses of whichever index of the
// operand is contiguous.
//
// Summation: each 16-deep slice is summed into fresh registers and the slice
// sums are added to the running total with an error-free two-sum whose
// rounding errors are carried in a compensation term (Knuth's TwoSum).  The
// contractions here run over K up to 2 chi^2 (8192 at chi = 64); a single
// running FP32 sum would carry an error growing with K, while this keeps it
// at the 32-term slice plus a few roundings of the total.
// ---------------------------------------------------------------------------
namespace {
constexpr int BM = 64, BN = 64, BK = 16;

// s + c += b with s the rounded sum and c the accumulated rounding errors.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float b) {
  const float t = __fadd_rn(s, b);
  const float bb = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(b, bb));
  s = t;
  c = __fadd_rn(c, e);
}

__device__ __forceinline__ int64_t koff(int k, int K2, int64_t s1, int64_t s2) {
  int k1 = k / K2;
  int k2 = k - k1 * K2;
  return (int64_t)k1 * s1 + (int64_t)k2 * s2;
}

__global__ void __launch_bounds__(256) cgemm_simt_kernel(GemmDesc d, float* part, int splits,
                                                          int k_per_split) {
  __shared__ float As[2][BK][BM + 1];
  __shared__ float Bs[2][BK][BN + 1];
  int z = blockIdx.z;
  const int split = z % splits;
  z /= splits;
  const int outer = z / d.n_inner;
  const int inner = z - outer * d.n_inner;
  if (outer_frozen(d, outer)) return;  // a converged component of a union
  const float* A = d.A[outer] + inner * d.a_in;
  const float* B = d.B[outer] + inner * d.b_in;
  float* C = d.C[outer] + inner * d.c_in;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int Kall = d.K1 * d.K2;
  // this CTA's K range (all of K without split-K)
  const int kb = split * k_per_split;
  const int K = min(Kall, kb + k_per_split);
  const bool a_kfast = (d.a_k2 == 1) && !(d.M2 > 1 && d.M3 <= 1 && d.a_m2 == 1) &&
                       !(d.M3 > 1 && d.a_m3 == 1);
  const bool b_nfast = (d.b_n == 1);
  const float sa = d.conj_a ? -1.f : 1.f;
  const float sb = d.conj_b ? -1.f : 1.f;

  float accr[4][4], acci[4][4], cmpr[4][4], cmpi[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = cmpr[i][j] = cmpi[i][j] = 0.f;

  for (int k0 = kb; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 256;
      int mm, kk;
      if (a_kfast) { kk = idx & (BK - 1); mm = idx >> 4; }
      else { mm = idx & (BM - 1); kk = idx >> 6; }
      const int m = m0 + mm, k = k0 + kk;
      float re = 0.f, im = 0.f;
      if (m < d.M && k < K) {
        const int64_t off = ROW_A(d, m) + koff(k, d.K2, d.a_k1, d.a_k2);
        re = A[off];
        im = sa * A[off + d.plane_a];
      }
      As[0][kk][mm] = re;
      As[1][kk][mm] = im;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 256;
      int nn, kk;
      if (b_nfast) { nn = idx & (BN - 1); kk = idx >> 6; }
      else { kk = idx & (BK - 1); nn = idx >> 4; }
      const int n = n0 + nn, k = k0 + kk;
      float re = 0.f, im = 0.f;
      if (n < d.N && k < K) {
        const int64_t off = (int64_t)n * d.b_n + koff(k, d.K2, d.b_k1, d.b_k2);
        re = B[off];
        im = sb * B[off + d.plane_b];
      }
      Bs[0][kk][nn] = re;
      Bs[1][kk][nn] = im;
    }
    __syncthreads();
    float pr[4][4], pi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) pr[i][j] = pi[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = As[0][kk][ty + 16 * i];
        ai[i] = As[1][kk][ty + 16 * i];
        br[i] = Bs[0][kk][tx + 16 * i];
        bi[i] = Bs[1][kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          pr[i][j] = fmaf(ar[i], br[j], pr[i][j]);
          pr[i][j] = fmaf(-ai[i], bi[j], pr[i][j]);
          pi[i][j] = fmaf(ar[i], bi[j], pi[i][j]);
          pi[i][j] = fmaf(ai[i], br[j], pi[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        two_sum_acc(accr[i][j], cmpr[i][j], pr[i][j]);
        two_sum_acc(acci[i][j], cmpi[i][j], pi[i][j]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      accr[i][j] = __fadd_rn(accr[i][j], cmpr[i][j]);
      acci[i][j] = __fadd_rn(acci[i][j], cmpi[i][j]);
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= d.N) continue;
      if (splits > 1) {
        // split-K partial [split][outer][inner][re|im][M][N], summed by the reduce
        float* q = part + ((((int64_t)split * d.n_outer + outer) * d.n_inner + inner) * 2) *
                              (int64_t)d.M * d.N;
        q[(int64_t)m * d.N + n] = accr[i][j];
        q[(int64_t)d.M * d.N + (int64_t)m * d.N + n] = acci[i][j];
        continue;
      }
      const int64_t off = ROW_C(d, m) + (int64_t)n * d.c_n;
      if (d.accumulate) {
        C[off] += accr[i][j];
        C[off + d.plane_c] += acci[i][j];
      } else {
        C[off] = accr[i][j];
        C[off + d.plane_c] = acci[i][j];
      }
    }
  }
}
}  // namespace

// Split-K for the CUDA-core GEMM: a launch whose grid is under one wave (152
// CTAs: a few sites with a long contraction, e.g. the closes) is split into at
// most 64 pieces of at least 256 K values, each summed with the compensated
// slices, the pieces then summed in FP64 in a fixed order by the reduce.
int cgemm_plan(const GemmDesc& d, size_t* part_floats, int force_splits) {
  const int64_t K = (int64_t)d.K1 * d.K2;
  const int64_t ctas = (int64_t)((d.N + BN - 1) / BN) * ((d.M + BM - 1) / BM) * d.n_outer * d.n_inner;
  int s = 1;
  if (force_splits > 0)
    s = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)force_splits, 64, (K + BK - 1) / BK}));
  else if (ctas < 152)
    while (s < 64 && ctas * s * 2 <= 2 * 152 && K / (2 * s) >= 256) s *= 2;
  *part_floats = s > 1 ? (size_t)s * d.n_outer * d.n_inner * 2 * d.M * d.N : 0;
  return s;
}

cudaError_t launch_cgemm(const GemmDesc& d, cudaStream_t s, float* part, size_t part_cap,
                         int* n_kernels, int force_splits) {
  if (n_kernels) *n_kernels = 0;
  if (d.M <= 0 || d.N <= 0 || d.n_outer <= 0 || d.n_inner <= 0) return cudaSuccess;
  size_t pf = 0;
  int splits = part ? cgemm_plan(d, &pf, force_splits) : 1;
  if (splits > 1 && pf > part_cap) splits = 1;  // the caller's partial buffer is too small
  const int K = d.K1 * d.K2;
  const int kps = splits > 1 ? ((K + splits - 1) / splits + BK - 1) / BK * BK : K;
  dim3 grid((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, d.n_outer * d.n_inner * splits);
  cgemm_simt_kernel<<<grid, 256, 0, s>>>(d, part, splits, kps);
  if (n_kernels) *n_kernels = splits > 1 ? 2 : 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return launch_tc_reduce(d, part, splits, s);
}

// ---------------------------------------------------------------------------
// 2x2 gate on the physical leg of a list of sites (all of one degree).
// ---------------------------------------------------------------------------
namespace {
__global__ void phys_gate_kernel(float* T, const int64_t* site_off, int64_t len, int64_t plane,
                                 float u00r, float u00i, float u01r, float u01i, float u10r,
                                 float u10i, float u11r, float u11i) {
  const int64_t base = site_off[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    float* t0r = T + base + i;
    float* t1r = T + base + len + i;
    const float ar = t0r[0], ai = t0r[plane];
    const float br = t1r[0], bi = t1r[plane];
    t0r[0] = u00r * ar - u00i * ai + u01r * br - u01i * bi;
    t0r[plane] = u00r * ai + u00i * ar + u01r * bi + u01i * br;
    t1r[0] = u10r * ar - u10i * ai + u11r * br - u11i * bi;
    t1r[plane] = u10r * ai + u10i * ar + u11r * bi + u11i * br;
  }
}
}  // namespace

namespace {
// RX(theta_v) = [[c, -i s], [-i s, c]] with (c, s) = (cos theta_v/2, sin theta_v/2)
// per site: the kicks of many instances batched in one graph.
__global__ void phys_gate_field_kernel(float* T, const int64_t* site_off, const float2* cs,
                                       int64_t len, int64_t plane) {
  const int64_t base = site_off[blockIdx.y];
  const float c = cs[blockIdx.y].x, sn = cs[blockIdx.y].y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    float* t0r = T + base + i;
    float* t1r = T + base + len + i;
    const float ar = t0r[0], ai = t0r[plane];
    const float br = t1r[0], bi = t1r[plane];
    // c a - i s b, -i s a + c b
    t0r[0] = c * ar + sn * bi;
    t0r[plane] = c * ai - sn * br;
    t1r[0] = sn * ai + c * br;
    t1r[plane] = -sn * ar + c * bi;
  }
}
}  // namespace

cudaError_t launch_phys_gate_field(float* T, const int64_t* site_off, const float2* cs,
                                   int n_sites, int64_t len, int64_t plane, cudaStream_t s) {
  if (n_sites <= 0) return cudaSuccess;
  int64_t bx = (len + 255) / 256;
  if (bx > 1024) bx = 1024;
  dim3 grid((unsigned)bx, n_sites);
  phys_gate_field_kernel<<<grid, 256, 0, s>>>(T, site_off, cs, len, plane);
  return cudaGetLastError();
}

cudaError_t launch_phys_gate(float* T, const int64_t* site_off, int n_sites, int64_t len,
                             int64_t plane, float u00r, float u00i, float u01r, float u01i,
                             float u10r, float u10i, float u11r, float u11i, cudaStream_t s) {
  if (n_sites <= 0) return cudaSuccess;
  int64_t bx = (len + 255) / 256;
  if (bx > 1024) bx = 1024;
  dim3 grid((unsigned)bx, n_sites);
  phys_gate_kernel<<<grid, 256, 0, s>>>(T, site_off, len, plane, u00r, u00i, u01r, u01i, u10r,
                                        u10i, u11r, u11i);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Message normalisation: Hermitise, FP64 Frobenius norm, residual vs. the
// current message, overwrite.  One CTA per directed message.
// ---------------------------------------------------------------------------
namespace {
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

// s + c += a^2 without rounding loss: the square split exactly by FMA
// (a a = p + e), the sum kept as an unevaluated pair (s, c) by Knuth's
// two-sum.  About 48 significant bits from FP32 operations, so the per-element
// work avoids the FP64 pipe (1/64 of the FP32 rate on this part).
__device__ __forceinline__ void pair_add_sq(float& s, float& c, float a) {
  const float p = __fmul_rn(a, a);  // not contracted into the sum below
  const float e = fmaf(a, a, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  c += (__fsub_rn(s, __fsub_rn(t, bp)) + __fsub_rn(p, bp)) + e;
  s = t;
}

// Large chi: the transposed entry is read from global memory.
__global__ void normalise_gmem_kernel(const float* raw, float* msg, int chi,
                                      unsigned long long* res_bits, int* flags, BpComp comp) {
  __shared__ double sh[32];
  // a message of a component that has already converged stays as it is
  const int cmp = comp.comp_of_msg ? comp.comp_of_msg[blockIdx.x] : -1;
  if (cmp >= 0 && comp.state[4 * cmp + 3] != 0.0) return;
  const int64_t n2 = (int64_t)chi * chi;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float* r = raw + blockIdx.x * 2 * n2;
  float* m = msg + blockIdx.x * 2 * n2;
  float s0 = 0.f, c0 = 0.f;
  for (int i = warp; i < chi; i += nw)
    for (int j = lane; j < chi; j += 32) {
      const int64_t a = (int64_t)i * chi + j, t = (int64_t)j * chi + i;
      pair_add_sq(s0, c0, 0.5f * (r[a] + r[t]));
      pair_add_sq(s0, c0, 0.5f * (r[n2 + a] - r[n2 + t]));
    }
  const double ss = block_sum((double)s0 + (double)c0, sh);
  const double nrm = sqrt(ss);
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (threadIdx.x == 0) atomicOr(flags, 1);
    return;
  }
  const float inv = (float)(1.0 / nrm);
  // all reads of the raw message precede the writes of the normalised one
  // (different buffers), so the loop may overwrite m as it goes
  float d0 = 0.f, dc = 0.f;
  for (int i = warp; i < chi; i += nw)
    for (int j = lane; j < chi; j += 32) {
      const int64_t a = (int64_t)i * chi + j, t = (int64_t)j * chi + i;
      const float hr = 0.5f * (r[a] + r[t]) * inv;
      const float hi = 0.5f * (r[n2 + a] - r[n2 + t]) * inv;
      pair_add_sq(d0, dc, hr - m[a]);
      pair_add_sq(d0, dc, hi - m[n2 + a]);
      m[a] = hr;
      m[n2 + a] = hi;
    }
  const double dd = block_sum((double)d0 + (double)dc, sh);
  if (threadIdx.x == 0) {
    const double res = sqrt(dd);
    atomicMax(res_bits, (unsigned long long)__double_as_longlong(res));
    if (cmp >= 0) atomicMax(&comp.res[cmp], (unsigned long long)__double_as_longlong(res));
  }
}

// The raw message is staged in shared memory (coalesced loads), so that the
// transposed entry needed by the Hermitisation is a shared-memory read.
__global__ void normalise_kernel(const float* __restrict__ raw, float* __restrict__ msg, int chi,
                                 unsigned long long* res_bits, int* flags,
                                 float* __restrict__ mrt, BpComp comp) {
  __shared__ double sh[32];
  // a message of a component that has already converged stays as it is (and
  // so does its realified copy)
  const int cmp = comp.comp_of_msg ? comp.comp_of_msg[blockIdx.x] : -1;
  if (cmp >= 0 && comp.state[4 * cmp + 3] != 0.0) return;
  // re and im planes of the new message, chi x (chi + 1) each (padded rows for
  // the transposed reads), then the old message's two planes, chi x chi each
  extern __shared__ float sraw[];
  const int ld = chi + 1;
  const int n2 = chi * chi;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* sre = sraw;
  float* sim = sraw + chi * ld;
  float* smr = sim + chi * ld;
  float* smi = smr + n2;
  const float* r = raw + (int64_t)blockIdx.x * 2 * n2;
  float* m = msg + (int64_t)blockIdx.x * 2 * n2;
  // every global read up front (coalesced, all in flight together): rows i over
  // warps, columns j over lanes, no index division
  for (int i = warp; i < chi; i += nw)
    for (int j = lane; j < chi; j += 32) {
      sre[i * ld + j] = r[i * chi + j];
      sim[i * ld + j] = r[n2 + i * chi + j];
      smr[i * chi + j] = m[i * chi + j];
      smi[i * chi + j] = m[n2 + i * chi + j];
    }
  __syncthreads();
  // H = (R + R^H) / 2: element (i, j) with the transposed read from the padded
  // tile (consecutive lanes, consecutive j: distinct banks)
  float s0 = 0.f, c0 = 0.f;
  for (int i = warp; i < chi; i += nw)
    for (int j = lane; j < chi; j += 32) {
      const float hr = 0.5f * (sre[i * ld + j] + sre[j * ld + i]);
      const float hi = 0.5f * (sim[i * ld + j] - sim[j * ld + i]);
      pair_add_sq(s0, c0, hr);
      pair_add_sq(s0, c0, hi);
    }
  double ss = block_sum((double)s0 + (double)c0, sh);
  const double nrm = sqrt(ss);
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (threadIdx.x == 0) atomicOr(flags, 1);
    return;
  }
  const float inv = (float)(1.0 / nrm);
  float d0 = 0.f, dc = 0.f;
  float* q = mrt ? mrt + (int64_t)blockIdx.x * 4 * n2 : nullptr;
  const int w = 2 * chi;
  for (int i = warp; i < chi; i += nw)
    for (int j = lane; j < chi; j += 32) {
      const int idx = i * chi + j;
      const float hr = 0.5f * (sre[i * ld + j] + sre[j * ld + i]) * inv;
      const float hi = 0.5f * (sim[i * ld + j] - sim[j * ld + i]) * inv;
      // the difference of two nearby FP32 values is exact
      pair_add_sq(d0, dc, hr - smr[idx]);
      pair_add_sq(d0, dc, hi - smi[idx]);
      m[idx] = hr;
      m[n2 + idx] = hi;
      if (q) {
        // realified transpose of the message: a [2chi][2chi] matrix with row (t, n)
        // and column (s, k), [[Re, Im], [-Im, Re]] of M[k][n] read transposed.
        // H is Hermitian, so M[k = j][n = i] = conj(H[i][j]): row i, column j is
        // written from this thread's own element (row-contiguous stores).
        q[i * w + j] = hr;
        q[(chi + i) * w + chi + j] = hr;
        q[(chi + i) * w + j] = -hi;
        q[i * w + chi + j] = hi;
      }
    }
  const double dd = block_sum((double)d0 + (double)dc, sh);
  if (threadIdx.x == 0) {
    const double res = sqrt(dd);
    atomicMax(res_bits, (unsigned long long)__double_as_longlong(res));
    if (cmp >= 0) atomicMax(&comp.res[cmp], (unsigned long long)__double_as_longlong(res));
  }
}

// ------------------------------------------------------------------------
// The BP stop rule on the device, per connected component of the handle's
// graph (one instance of a batch union): component c stops after a sweep
// whose residual r_c (the largest ||M_new - M_old||_F of its messages) is
// below tol; or, once r_c is below the precision's residual floor, when r_c is
// under floor / 8 or not below 0.98 of its previous sweep's (FP32 messages
// cannot reach an FP64 tolerance); or at max_iters.  A stopped component's
// messages are frozen (the normalise kernels skip them), so it keeps exactly
// the messages it would have had alone.  state[4c..4c+3]: previous residual,
// final residual, sweeps, done.  out: [0] the largest sweep count, [1] the
// largest final residual (IEEE bits), [2] components stopped at max_iters
// without converging, [3] the flag word, [4] 1 while any component runs.
__global__ void bp_loop_init_kernel(int n_comp, double* state, unsigned long long* res,
                                    unsigned long long* res_bits, double* par, double tol,
                                    double max_iters, double floor_, unsigned long long* out) {
  for (int c = threadIdx.x; c < n_comp; c += blockDim.x) {
    state[4 * c + 0] = INFINITY;
    state[4 * c + 1] = 0.0;
    state[4 * c + 2] = 0.0;
    state[4 * c + 3] = 0.0;
    res[c] = 0ull;
  }
  if (threadIdx.x == 0) {
    res_bits[0] = 0ull;
    res_bits[1] = 0ull;  // the flag word shares this 8-byte slot
    par[0] = tol;
    par[1] = max_iters;
    par[2] = floor_;
    for (int i = 0; i < 5; ++i) out[i] = 0ull;
  }
}

__global__ void bp_stop_kernel(int n_comp, double* state, unsigned long long* res,
                               unsigned long long* res_bits, const double* par,
                               unsigned long long* out, cudaGraphConditionalHandle cond,
                               int set_cond) {
  __shared__ double smax[2];
  __shared__ int cnt[2];
  const int flags = *reinterpret_cast<const int*>(res_bits + 1);
  const double tol = par[0], max_iters = par[1], floor_ = par[2];
  if (threadIdx.x == 0) { smax[0] = 0.0; smax[1] = 0.0; cnt[0] = 0; cnt[1] = 0; }
  __syncthreads();
  int active = 0;
  for (int c = threadIdx.x; c < n_comp; c += blockDim.x) {
    if (state[4 * c + 3] == 0.0) {
      const double r = __longlong_as_double((long long)res[c]);
      const double it = state[4 * c + 2] + 1.0;
      const double prev = state[4 * c + 0];
      const bool conv = r < tol;
      const bool stag = !conv && r < floor_ && (r < floor_ / 8 || (it >= 2.0 && r >= 0.98 * prev));
      const bool cap = it >= max_iters;
      state[4 * c + 2] = it;
      state[4 * c + 0] = r;
      if (conv || stag || cap || flags) {
        state[4 * c + 3] = 1.0;
        state[4 * c + 1] = r;
        if (!conv && !stag) atomicAdd(&cnt[1], 1);
      } else {
        active = 1;
      }
    }
    res[c] = 0ull;  // the next sweep's accumulator
  }
  active = __syncthreads_or(active);
  if (!active) {
    // the loop ends: summary over every component
    double ms = 0.0, mr = 0.0;
    for (int c = threadIdx.x; c < n_comp; c += blockDim.x) {
      ms = fmax(ms, state[4 * c + 2]);
      mr = fmax(mr, state[4 * c + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ms = fmax(ms, __shfl_xor_sync(0xffffffffu, ms, o));
      mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(reinterpret_cast<unsigned long long*>(&smax[0]),
                (unsigned long long)__double_as_longlong(ms));
      atomicMax(reinterpret_cast<unsigned long long*>(&smax[1]),
                (unsigned long long)__double_as_longlong(mr));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!active) {
      out[0] = (unsigned long long)smax[0];
      out[1] = (unsigned long long)__double_as_longlong(smax[1]);
    }
    out[2] += (unsigned long long)cnt[1];
    out[3] = (unsigned long long)(unsigned)flags;
    out[4] = active ? 1ull : 0ull;
    res_bits[0] = 0ull;
    if (set_cond) cudaGraphSetConditional(cond, active ? 1u : 0u);
  }
}

// Region contractions: an up-message scaled to unit Frobenius norm, its log
// norm added to *logacc (one CTA, launches in stream order: a fixed summation
// order); a zero message sets *zero instead.
__global__ void scale_unit_kernel(float* m, int chi, double* logacc, int* zero) {
  __shared__ double sh[32];
  const int n2 = chi * chi;
  float s0 = 0.f, c0 = 0.f;
  for (int i = threadIdx.x; i < 2 * n2; i += blockDim.x) pair_add_sq(s0, c0, m[i]);
  const double ss = block_sum((double)s0 + (double)c0, sh);
  const double nrm = sqrt(ss);
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (threadIdx.x == 0) *zero = 1;
    return;
  }
  const float inv = (float)(1.0 / nrm);
  for (int i = threadIdx.x; i < 2 * n2; i += blockDim.x) m[i] *= inv;
  if (threadIdx.x == 0) *logacc += log(nrm);
}

// out = sum_ij R[i][j] M[i][j] (planar complex chi x chi), FP64.
__global__ void dot_msgs_kernel(const float* R, const float* M, int chi, double* out) {
  __shared__ double sh[32];
  const int n2 = chi * chi;
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    const double ar = R[i], ai = R[n2 + i], br = M[i], bi = M[n2 + i];
    re += ar * br - ai * bi;
    im += ar * bi + ai * br;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) { out[0] = re; out[1] = im; }
}

// Realified transposed copies (see GemmDesc::b_pre).
__global__ void realify_kernel(const float* src, int64_t stride, float* dst, int chi) {
  const int64_t n2 = (int64_t)chi * chi;
  const float* a = src + blockIdx.y * stride;
  float* q = dst + (int64_t)blockIdx.y * 4 * n2;
  const int64_t w = 2 * chi;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / chi), j = (int)(idx - (int64_t)i * chi);  // element [k = i][n = j]
    const float re = a[idx], im = a[n2 + idx];
    q[(int64_t)j * w + i] = re;
    q[(int64_t)(chi + j) * w + chi + i] = re;
    q[(int64_t)(chi + j) * w + i] = im;
    q[(int64_t)j * w + chi + i] = -im;
  }
}

// TA[pl][p][rest][l0] = T[pl][p][l0][rest]: per (site, plane, p) a chi x rest
// matrix transposed through a padded 32 x 33 shared tile, so that both the
// reads (along rest) and the writes (along l0) are row-contiguous.
__global__ void first_leg_last_kernel(const float* T, float* TA, const int64_t* site_off,
                                      int chi, int64_t rest) {
  __shared__ float tile[32][33];
  const int site = blockIdx.z >> 2, pp = blockIdx.z & 3;  // pp = plane * 2 + p
  const int64_t len = rest * chi;  // chi^d
  const float* src = T + site_off[site] + (int64_t)pp * len;  // [l0][rest]
  float* dst = TA + site_off[site] + (int64_t)pp * len;       // [rest][l0]
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int l00 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += 8) {
    const int l0 = l00 + i;
    const int64_t r = r0 + tx;
    if (l0 < chi && r < rest) tile[i][tx] = src[(int64_t)l0 * rest + r];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i;
    const int l0 = l00 + tx;
    if (r < rest && l0 < chi) dst[r * chi + l0] = tile[tx][i];
  }
}

// The same transpose for wide slabs (rest a multiple of 128, chi of 32, site
// offsets 16-byte aligned): a 32 x 128 tile read as 16-byte vectors (four per
// thread in flight), written as 128-byte rows of l0.
__global__ void first_leg_last_wide_kernel(const float* __restrict__ T, float* __restrict__ TA,
                                           const int64_t* site_off, int chi, int64_t rest) {
  __shared__ float tile[32][129];
  const int site = blockIdx.z >> 2, pp = blockIdx.z & 3;
  const int64_t len = rest * chi;
  const float* src = T + site_off[site] + (int64_t)pp * len;  // [l0][rest]
  float* dst = TA + site_off[site] + (int64_t)pp * len;       // [rest][l0]
  const int64_t r0 = (int64_t)blockIdx.x * 128;
  const int l00 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float4 v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    v[k] = *reinterpret_cast<const float4*>(src + (int64_t)(l00 + ty + 8 * k) * rest + r0 + 4 * tx);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float* row = &tile[ty + 8 * k][4 * tx];
    row[0] = v[k].x; row[1] = v[k].y; row[2] = v[k].z; row[3] = v[k].w;
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const int r = ty + 8 * k;
    dst[(r0 + r) * chi + l00 + tx] = tile[tx][r];
  }
}
}  // namespace

cudaError_t launch_scale_unit(float* m, int chi, double* logacc, int* zero, cudaStream_t s) {
  scale_unit_kernel<<<1, 256, 0, s>>>(m, chi, logacc, zero);
  return cudaGetLastError();
}

cudaError_t launch_dot_msgs(const float* R, const float* M, int chi, double* out, cudaStream_t s) {
  dot_msgs_kernel<<<1, 256, 0, s>>>(R, M, chi, out);
  return cudaGetLastError();
}

cudaError_t launch_realify(const float* src, int64_t src_stride, float* dst, int n, int chi,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t n2 = (int64_t)chi * chi;
  int64_t bx = (n2 + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid((unsigned)bx, n);
  realify_kernel<<<grid, 256, 0, s>>>(src, src_stride, dst, chi);
  return cudaGetLastError();
}

cudaError_t launch_first_leg_last(const float* T, float* TA, const int64_t* site_off, int n_sites,
                                  int d, int chi, cudaStream_t s) {
  if (n_sites <= 0 || d < 2) return cudaSuccess;
  int64_t rest = 1;
  for (int i = 1; i < d; ++i) rest *= chi;
  if (4LL * n_sites > 65535) return cudaErrorInvalidValue;
  // site offsets are multiples of 4 floats (whole planes of chi^d values, chi
  // even) when chi % 32 == 0; the base pointers come from 256-byte allocations
  const bool wide = rest % 128 == 0 && chi % 32 == 0 &&
                    ((reinterpret_cast<uintptr_t>(T) | reinterpret_cast<uintptr_t>(TA)) & 15) == 0;
  if (wide) {
    dim3 grid((unsigned)(rest / 128), (unsigned)(chi / 32), (unsigned)(4 * n_sites));
    first_leg_last_wide_kernel<<<grid, dim3(32, 8), 0, s>>>(T, TA, site_off, chi, rest);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((rest + 31) / 32), (unsigned)((chi + 31) / 32), (unsigned)(4 * n_sites));
  first_leg_last_kernel<<<grid, dim3(32, 8), 0, s>>>(T, TA, site_off, chi, rest);
  return cudaGetLastError();
}

// The shared-memory limit of the normalise kernel, raised once to the largest
// tile the kernel takes (chi with 2 chi (chi + 1) floats <= 200 KB); thread-safe.
cudaError_t normalise_prepare(int) {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    result = cudaFuncSetAttribute(normalise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024);
  });
  return result;
}

cudaError_t launch_bp_loop_init(int n_comp, double* state, unsigned long long* res,
                                unsigned long long* res_bits, double* par, double tol,
                                int max_iters, double floor_, unsigned long long* out,
                                cudaStream_t s) {
  bp_loop_init_kernel<<<1, 256, 0, s>>>(n_comp, state, res, res_bits, par, tol, (double)max_iters,
                                        floor_, out);
  return cudaGetLastError();
}

cudaError_t launch_bp_stop(int n_comp, double* state, unsigned long long* res,
                           unsigned long long* res_bits, const double* par, unsigned long long* out,
                           cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s) {
  bp_stop_kernel<<<1, 256, 0, s>>>(n_comp, state, res, res_bits, par, out, cond, set_cond);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const float* raw, float* msg, int n_msgs, int chi,
                             unsigned long long* res_bits, int* flags, cudaStream_t s, float* mrt,
                             const BpComp* comp) {
  if (n_msgs <= 0) return cudaSuccess;
  const BpComp cp = comp ? *comp : BpComp{};
  const size_t sm = sizeof(float) * 2 * (size_t)chi * (chi + 1) + sizeof(float) * 2 * (size_t)chi * chi;
  if (sm > 200 * 1024) {
    normalise_gmem_kernel<<<n_msgs, 256, 0, s>>>(raw, msg, chi, res_bits, flags, cp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !mrt) return e;
    return launch_realify(msg, 2 * (int64_t)chi * chi, mrt, n_msgs, chi, s);
  }
  {
    cudaError_t e = normalise_prepare(chi);
    if (e != cudaSuccess) return e;
  }
  normalise_kernel<<<n_msgs, 256, sm, s>>>(raw, msg, chi, res_bits, flags, mrt, cp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// rho[p][p'] = sum_r X[p][r] conj(T[p'][r]), FP64 accumulation, one CTA per site.
// ---------------------------------------------------------------------------
namespace {
// s + c += a b without rounding loss (exact product split by FMA, two-sum).
__device__ __forceinline__ void pair_add_prod(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  c += (__fsub_rn(s, __fsub_rn(t, bp)) + __fsub_rn(p, bp)) + e;
  s = t;
}

// rho_v[p][q] = sum_i X_v[p][i] conj(T_v[q][i]): grid (blocks per site, sites);
// each thread keeps the 8 real parts as compensated FP32 pairs (about 48 bits,
// off the FP64 pipe), each CTA writes its 8 sums to part[site][block][8]; a
// second kernel adds the blocks in a fixed order in FP64.
__global__ void rho_part_kernel(const float* X, const float* T, const int64_t* x_off,
                                const int64_t* t_off, int64_t len, int64_t plane, double* part) {
  __shared__ double sh[32];
  const float* x = X + x_off[blockIdx.y];
  const float* t = T + t_off[blockIdx.y];
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0}, c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x0r = x[i], x0i = x[plane + i], x1r = x[len + i], x1i = x[plane + len + i];
    const float t0r = t[i], t0i = t[plane + i], t1r = t[len + i], t1i = t[plane + len + i];
    // x_p conj(t_q) = (xr tr + xi ti) + i (xi tr - xr ti)
    pair_add_prod(s[0], c[0], x0r, t0r); pair_add_prod(s[0], c[0], x0i, t0i);
    pair_add_prod(s[1], c[1], x0i, t0r); pair_add_prod(s[1], c[1], -x0r, t0i);
    pair_add_prod(s[2], c[2], x0r, t1r); pair_add_prod(s[2], c[2], x0i, t1i);
    pair_add_prod(s[3], c[3], x0i, t1r); pair_add_prod(s[3], c[3], -x0r, t1i);
    pair_add_prod(s[4], c[4], x1r, t0r); pair_add_prod(s[4], c[4], x1i, t0i);
    pair_add_prod(s[5], c[5], x1i, t0r); pair_add_prod(s[5], c[5], -x1r, t0i);
    pair_add_prod(s[6], c[6], x1r, t1r); pair_add_prod(s[6], c[6], x1i, t1i);
    pair_add_prod(s[7], c[7], x1i, t1r); pair_add_prod(s[7], c[7], -x1r, t1i);
  }
  for (int k = 0; k < 8; ++k) {
    const double v = block_sum((double)s[k] + (double)c[k], sh);
    if (threadIdx.x == 0) part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + k] = v;
  }
}

__global__ void rho_sum_kernel(const double* part, int nblk, int n_sites, double* rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (site, component)
  if (i >= 8 * n_sites) return;
  const int site = i / 8, k = i % 8;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += part[((int64_t)site * nblk + b) * 8 + k];
  rho[i] = v;
}
}  // namespace

int rho_blocks(int n_sites, int64_t len) {
  int nblk = (2 * 152 + n_sites - 1) / n_sites;
  const int64_t most = (len + 255) / 256;
  if (nblk > most) nblk = (int)most;
  if (nblk > 16) nblk = 16;
  return nblk < 1 ? 1 : nblk;
}

cudaError_t launch_rho(const float* X, const float* T, const int64_t* x_off,
                       const int64_t* t_off, int n_sites, int64_t len, int64_t plane,
                       double* rho, double* part, cudaStream_t s) {
  if (n_sites <= 0) return cudaSuccess;
  const int nblk = rho_blocks(n_sites, len);
  rho_part_kernel<<<dim3(nblk, n_sites), 256, 0, s>>>(X, T, x_off, t_off, len, plane, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rho_sum_kernel<<<(8 * n_sites + 255) / 256, 256, 0, s>>>(part, nblk, n_sites, rho);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
namespace {
__global__ void copy_blocks_kernel(float* const* dst, const float* const* src, int64_t n4) {
  float4* d = reinterpret_cast<float4*>(dst[blockIdx.y]);
  const float4* s = reinterpret_cast<const float4*>(src[blockIdx.y]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}
}  // namespace

cudaError_t launch_copy_blocks(float* const* dst, const float* const* src, int n_blocks,
                               int64_t n_floats, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  const int64_t n4 = n_floats / 4;
  int64_t bx = (n4 + 255) / 256;
  if (bx > 512) bx = 512;
  dim3 grid((unsigned)bx, n_blocks);
  copy_blocks_kernel<<<grid, 256, 0, s>>>(dst, src, n4);
  return cudaGetLastError();
}

}  // namespace tnbp
