// Shared definitions of the tnbp CUDA library (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tnbp.h"

namespace tnbp {

// Thread-local error message behind tn_last_error().
void set_error(const std::string& msg);

#define TN_CUDA_TRY(expr)                                                        \
  do {                                                                          \
    cudaError_t err__ = (expr);                                                 \
    if (err__ != cudaSuccess) {                                                 \
      ::tnbp::set_error(std::string(#expr) + ": " + cudaGetErrorString(err__)); \
      return TN_ECUDA;                                                          \
    }                                                                           \
  } while (0)

// ---------------------------------------------------------------------------
// Batched strided complex GEMM on planar complex FP32 data.
//
//   C[m][n] (+)= alpha * sum_k opA(A)[m][k] * opB(B)[k][n]
//
// The contraction index k runs over K1 * K2 values, k = k1 * K2 + k2, so that
// a contraction over two tensor legs with unrelated strides is one GEMM.  The
// row index may likewise be two-level: with M2 > 1, m = m1 * M2 + m2 and row m
// of A (C) starts at m1*a_m + m2*a_m2 (m1*c_m + m2*c_m2); with M2 <= 1 it
// starts at m*a_m (m*c_m).  Element (m, k1, k2) of A is then at
// A + row(m) + k1*a_k1 + k2*a_k2; likewise B (n*b_n + ...) and C.  Each operand is planar: the imaginary plane starts plane_* floats after
// the real plane.  The batch is outer x inner: the outer index selects base
// pointers from device arrays, the inner index adds inner * *_in.
// ---------------------------------------------------------------------------
struct GemmDesc {
  const float* const* A;
  const float* const* B;
  float* const* C;
  int64_t plane_a, plane_b, plane_c;
  int32_t M, N, K1, K2;
  int64_t a_m, a_k1, a_k2;
  int64_t b_k1, b_k2, b_n;
  int64_t c_m, c_n;
  int32_t n_outer, n_inner;
  int64_t a_in, b_in, c_in;
  int32_t conj_a, conj_b;
  int32_t accumulate;
  int32_t prec;  // tn_precision of the contraction
  int32_t M2, M3;
  int64_t a_m2, c_m2, a_m3, c_m3;
  // b_pre: B points to the realified, transposed small operand, a real
  // [2N][2K] row-major matrix Bt[(t,n)][(s,k)] = [[B_re, B_im], [-B_im, B_re]][s][t]
  // (the fields b_n, b_k2, plane_b then describe its complex view).
  int32_t b_pre;
  // BP sweep launches over a disjoint union: the component of each outer
  // entry and the stop rule's per-component state; a CTA whose component has
  // stopped returns at once (null: no skipping).  Honoured by the tile GEMM,
  // the CUDA-core GEMM and the split-K reduce.
  const int* outer_comp;
  const double* comp_state;
};
// true when the outer entry's component has met the BP stop rule
__device__ __forceinline__ bool outer_frozen(const GemmDesc& d, int outer) {
  return d.outer_comp && d.comp_state[4 * d.outer_comp[outer] + 3] != 0.0;
}

// Row offset for the two- or three-level row index: with M3 > 1,
// m = (m1 * M2 + m2) * M3 + m3 and the offset is m1*s1 + m2*s2 + m3*s3; with
// M3 <= 1 and M2 > 1, m = m1 * M2 + m2; otherwise m*s1.
__host__ __device__ __forceinline__ int64_t row_off3(int m, int M2, int M3, int64_t s1,
                                                     int64_t s2, int64_t s3) {
  if (M3 > 1) {
    const int m12 = m / M3;
    const int m3 = m - m12 * M3;
    const int m1 = m12 / M2;
    return (int64_t)m1 * s1 + (int64_t)(m12 - m1 * M2) * s2 + (int64_t)m3 * s3;
  }
  if (M2 <= 1) return (int64_t)m * s1;
  const int m1 = m / M2;
  return (int64_t)m1 * s1 + (int64_t)(m - m1 * M2) * s2;
}
#define ROW_A(d, m) row_off3((m), (d).M2, (d).M3, (d).a_m, (d).a_m2, (d).a_m3)
#define ROW_C(d, m) row_off3((m), (d).M2, (d).M3, (d).c_m, (d).c_m2, (d).c_m3)

// Launch helpers implemented in kernels.cu / solve.cu.  All return a
// cudaError_t from the launch.
// CUDA-core complex GEMM (kernels.cu); with part != nullptr (part_cap floats) a
// launch whose grid is under one wave is split over K into partials (cgemm_plan
// gives the count and the partial floats) and summed by the fixed-order reduce.
// force_splits > 0 replaces the heuristic split count (the autotuner's
// choice); a count whose partials would not fit part_cap falls back to one.
int cgemm_plan(const GemmDesc& d, size_t* part_floats, int force_splits = 0);
cudaError_t launch_cgemm(const GemmDesc& d, cudaStream_t s, float* part = nullptr,
                         size_t part_cap = 0, int* n_kernels = nullptr, int force_splits = 0);
// Tensor-core version (tc_gemm.cu) for TN_TF32 / TN_BF16 descriptors.  part:
// scratch for K-split partial products (tc_plan gives the size, part_cap the
// floats the caller holds: a plan that needs more is refused); err: bit 1 is
// set when a device-side wait gave up.  force_splits as for cgemm_plan.
bool tc_plan(const GemmDesc& d, int* quad, int* splits, size_t* part_floats,
             int force_splits = 0);
cudaError_t launch_cgemm_tc(const GemmDesc& d, float* part, int* err, cudaStream_t s,
                            int* n_kernels = nullptr, int force_splits = 0,
                            size_t part_cap = (size_t)-1);
// Persistent TMA-fed kernel for mode products (tc_stream.cu): one A and one B
// tensor map per batch entry, encoded on the host when a plan is uploaded.
struct TcStreamPlan {
  const void* maps = nullptr;  // device CUtensorMap[2 * n_outer]
  int kind = 0;                // 0: mode product (streaming), 1: close (TMA split-K),
                               // 2: two fused mode products (maps: A, Bt1, Bt2)
  int n_outer = 0, rank = 0, lev0 = 1, lev1 = 1;
  int splits = 1;              // close: K splits per entry
};
cudaError_t launch_tc_reduce(const GemmDesc& d, const float* part, int splits, cudaStream_t s);
// Fills host_maps (tc_stream_map_bytes(n_outer) bytes, 64-byte aligned) and
// the plan's shape fields; false when the descriptor is not eligible.
bool tc_stream_encode(const GemmDesc& d, const float* const* A, const float* const* B, int n_outer,
                      void* host_maps, TcStreamPlan* p);
size_t tc_stream_map_bytes(int n_outer);
cudaError_t tc_stream_prepare();
cudaError_t launch_tc_stream(const GemmDesc& d, const TcStreamPlan& p, int* err, cudaStream_t s);
// Closes (tc_stream.cu): out[m][n] = sum_K A[m][K] op(B[n][K]), M = N = 64, both
// operands K-contiguous, TF32; TMA-fed split-K into partials + the fixed-order
// reduce (a single split writes the output directly).  part_floats bounds the
// partial buffer the caller provides.
bool tc_close_encode(const GemmDesc& d, const float* const* A, const float* const* B, int n_outer,
                     size_t part_floats, void* host_maps, TcStreamPlan* p);
cudaError_t launch_tc_close(const GemmDesc& d, const TcStreamPlan& p, float* part, int* err,
                            cudaStream_t s);
// Two consecutive mode products fused (tc_stream.cu): d1 the first (A, B1 ->
// C1), d2 the second (A2 == C1, B2 -> its C); eligible when the second reads
// exactly what the first writes, contracting the first's innermost row level.
// host_maps: tc_chain_map_bytes(n_outer) bytes, 64-byte aligned.
bool tc_chain_encode(const GemmDesc& d1, const GemmDesc& d2, const float* const* A,
                     const float* const* B1, const float* const* A2, const float* const* B2,
                     float* const* C1, int n_outer, void* host_maps, TcStreamPlan* p);
size_t tc_chain_map_bytes(int n_outer);
cudaError_t launch_tc_chain(const GemmDesc& d1, const GemmDesc& d2, const TcStreamPlan& p,
                            int* err, cudaStream_t s);
// Vidal gauge of every edge from the converged messages (solve.cu): per edge
// e, dir[2e], dir[2e+1] the directed-message ids u->w and w->u; out the leg
// matrices G_u, G_w (FP32 planar, [e][side][re|im][chi][chi]) and the
// normalised bond weights lambda (FP64 [e][chi]).  work: vidal_work_doubles(chi)
// per edge.
size_t vidal_work_doubles(int chi);
cudaError_t launch_vidal_edges(const float* msg, const int32_t* dir, int n_edges, int chi,
                               double* work, float* gout, double* lam_out, int* flags,
                               cudaStream_t s);
// Bounded-wait self-test (tc_stream.cu): a wait nothing completes; sets bit 1
// of *err when it gives up (bit 2 if it returned without giving up).
cudaError_t launch_wait_selftest(int* err, cudaStream_t s);
// Kernel attributes set once, before any launch or stream capture.
cudaError_t tc_prepare();
cudaError_t normalise_prepare(int chi);

// RX-type 2x2 on the physical leg: T[p] <- sum_q U[p][q] T[q] for every site in
// the list.  site_off: float offset of each site's real plane; len: chi^d
// complex entries per physical value; plane: 2*chi^d.
cudaError_t launch_scale_unit(float* m, int chi, double* logacc, int* zero, cudaStream_t s);
cudaError_t launch_dot_msgs(const float* R, const float* M, int chi, double* out, cudaStream_t s);
cudaError_t launch_phys_gate_field(float* T, const int64_t* site_off, const float2* cs,
                                   int n_sites, int64_t len, int64_t plane, cudaStream_t s);
cudaError_t launch_phys_gate(float* T, const int64_t* site_off, int n_sites, int64_t len,
                             int64_t plane, float u00r, float u00i, float u01r, float u01i,
                             float u10r, float u10i, float u11r, float u11i, cudaStream_t s);

// Hermitise, normalise (Frobenius, FP64) and compare raw messages against the
// current ones: msg <- normalise(raw); residual <- max ||new - old||_F.
// res_bits: one unsigned long long holding the max residual as IEEE bits;
// flags: bit 0 set on a non-finite or zero-norm message.
// Per-component state of the device-side BP stop rule (kernels.cu): the
// component of each directed message, the per-component state
// [previous residual, final residual, sweeps, done] and residual accumulator.
struct BpComp {
  const int* comp_of_msg = nullptr;
  const double* state = nullptr;
  unsigned long long* res = nullptr;
};
cudaError_t launch_normalise(const float* raw, float* msg, int n_msgs, int chi,
                             unsigned long long* res_bits, int* flags, cudaStream_t s,
                             float* mrt = nullptr, const BpComp* comp = nullptr);
// The device-side BP loop: reset the per-component state and the loop's
// parameters; after each sweep, apply the stop rule per component and set the
// while-loop condition (set_cond) or only the continue word out[4].
cudaError_t launch_bp_loop_init(int n_comp, double* state, unsigned long long* res,
                                unsigned long long* res_bits, double* par, double tol,
                                int max_iters, double floor_, unsigned long long* out,
                                cudaStream_t s);
cudaError_t launch_bp_stop(int n_comp, double* state, unsigned long long* res,
                           unsigned long long* res_bits, const double* par, unsigned long long* out,
                           cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s);

// Realified transposed copies of n planar complex chi x chi matrices (each at
// src + i*src_stride): dst + i*4chi^2 holds Bt[(t,n)][(s,k)] as in GemmDesc::b_pre.
cudaError_t launch_realify(const float* src, int64_t src_stride, float* dst, int n, int chi,
                           cudaStream_t s);

// TA copies of site tensors with the first leg moved last:
// TA[pl][p][l1..l_{d-1}][l0] = T[pl][p][l0][l1..l_{d-1}] (planar).
cudaError_t launch_first_leg_last(const float* T, float* TA, const int64_t* site_off, int n_sites,
                                  int d, int chi, cudaStream_t s);

// rho[site][p][p'] = sum_r X[p][r] conj(T[p'][r]) in FP64 (complex, 8 doubles
// per site).  x_off / t_off: real-plane offsets; len = chi^d; plane = 2*len.
// rho of n_sites sites; part: scratch of n_sites * 16 * 8 doubles.
cudaError_t launch_rho(const float* X, const float* T, const int64_t* x_off,
                       const int64_t* t_off, int n_sites, int64_t len, int64_t plane,
                       double* rho, double* part, cudaStream_t s);

// Batched copy of equally sized blocks: dst[i][0..n) = src[i][0..n).
cudaError_t launch_copy_blocks(float* const* dst, const float* const* src, int n_blocks,
                               int64_t n_floats, cudaStream_t s);

// FP64 truncation solve for one colour layer (see solve.cu).
struct SolveArgs {
  int n_edges;
  int chi;
  int sign;                 // +1: exp(+i pi/4 ZZ); -1: exp(-i pi/4 ZZ)
  double gram_cut;          // relative eigenvalue cutoff of the v-side Gram
  double svd_cut;           // relative singular-value cutoff
  const float* gram;        // [edge][side][p][plane][chi][chi]
  float* dmat;              // [edge][side][p][plane][chi][chi]
  float* msg;               // message buffer [2E][plane][chi][chi] (may be null)
  const int32_t* msg_vw;    // per edge: directed index of v->w and w->v
  double* s_out;            // per edge: chi normalised singular values (may be null)
  double* work;             // [edge][6][n][n] complex doubles
  double* stats;            // per edge: [discarded weight, kept, sigma_1, min_gap]
  int* flags;
  int max_sweeps;
  float orth_tol = 2e-6f;   // shared solve: pairs with |<x_p, x_q>| below
                            // orth_tol ||x_p|| ||x_q|| count as orthogonal
  int basis = 0;            // shared solve in basis mode (the refined solve's FP32
                            // phase): R_v from the FP64 Cholesky in work, output the
                            // starting eigenbasis to work instead of the leg matrices
};

// Per-edge layout of the refined solve's workspace (offsets in doubles from the
// edge's base work + edge * stride; complex values are pairs of doubles).
struct RefineLayout {
  int64_t L;      // [2][chi][chi] complex: FP64 Cholesky factors of the G_v blocks
  int64_t U;      // [n][n] complex: starting basis, column m at U + 2 n m
  int64_t U1;     // [chi][n] complex: refined kept columns
  int64_t lam0;   // [n]: sigma^2 of the starting basis (decreasing)
  int64_t lam1;   // [chi]: refined eigenvalues of the kept columns
  int64_t misc;   // [4]: sum of all sigma^2 of the start, FP32 sweeps
  int64_t ints;   // int32 [2 chi] perm, [2] rank, [1] active columns
  int64_t S;      // [n][n] float2: FP32 G_w and its Cholesky factor (2 chi > 128 only)
  int64_t stride;
};
__host__ __device__ inline RefineLayout refine_layout(int chi) {
  const int64_t n = 2 * (int64_t)chi;
  RefineLayout l;
  l.L = 0;
  l.U = l.L + 4 * (int64_t)chi * chi;
  l.U1 = l.U + 2 * n * n;
  l.lam0 = l.U1 + 2 * n * chi;
  l.lam1 = l.lam0 + n;
  l.misc = l.lam1 + chi;
  l.ints = l.misc + 4;
  l.S = l.ints + chi + 4;  // after the 2 chi + 3 ints
  l.stride = 12 * n * n;  // solve_work_doubles(chi)
  return l;
}
cudaError_t launch_solve(const SolveArgs& a, cudaStream_t s);
size_t solve_work_doubles(int chi);
// Shared-memory solve with FP32 rotations (solve32.cu), chi <= 64.
bool solve32_supported(int chi);
cudaError_t launch_solve32(const SolveArgs& a, cudaStream_t s);
// The refined solve's FP32 starting basis for 2 chi > 128 (solve32.cu): the
// bond matrix in the global workspace, one CTA per edge, 16 <= chi <= 256.
cudaError_t launch_basis_gmem(const SolveArgs& a, cudaStream_t s);
// Refined solve (solve_refine.cu): FP64 Cholesky, FP32 starting basis, FP64
// Newton refinement and FP64 leg matrices; chi <= 64.  work: solve_work_doubles
// per edge.
bool solve_refined_supported(int chi);
cudaError_t launch_solve_refined(const SolveArgs& a, cudaStream_t s);
// The two halves of launch_solve_refined: the FP64 Cholesky and the FP32
// starting basis; the FP64 Newton step and leg matrices.
cudaError_t launch_solve_refined_basis(const SolveArgs& a, cudaStream_t s);
cudaError_t launch_solve_refined_newton(const SolveArgs& a, cudaStream_t s);

}  // namespace tnbp
