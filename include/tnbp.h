/*
 * tnbp.h — C ABI of the GB300 library for BP-approximated tensor-network
 * simulation of the kicked-Ising Floquet circuit on heavy-hex lattices
 * (Tindall, Fishman, Stoudenmire, Sels, arXiv:2306.14887).
 *
 * The library evolves |psi(theta_h, n)> = U(theta_h)^n |0...0> (Eq. 1 and
 * Eq. "State") as a tensor network with one site tensor T_v[p, l_1..l_d] per
 * qubit (physical index p, one virtual leg of dimension chi per incident edge,
 * Fig. "heavyhexdiagram"), kept in an arbitrary gauge together with the
 * belief-propagation (BP) messages of its norm network (Methods, "Belief
 * propagation on a tensor network state").  One Floquet step is: RX(theta_h)
 * on every qubit (exact), then exp(+i pi/4 Z_v Z_w) on every edge by the
 * BP-gauged simple update with truncation back to chi (Methods, "The simple
 * update procedure"), edge colour layer by layer, then BP regauging.
 * Expectation values are read from the converged messages (Methods,
 * "Measuring expectation values within the Vidal gauge").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns tn_status: TN_OK (0) or a negative error code.
 *   Nothing throws across the ABI and nothing aborts the process.
 *   tn_last_error() returns a message for the calling thread's last error;
 *   the string is owned by the library and valid until the next call on
 *   that thread.
 * - Host arrays passed in are owned by the caller and copied during the call.
 *   Host output arrays are owned by the caller and must have the stated size.
 * - Device memory is obtained through the tn_allocator callbacks given to
 *   tn_create (NULL: the library calls cudaMalloc/cudaFree itself) and all
 *   device work runs on the CUDA stream given to tn_create (NULL: the legacy
 *   default stream).  Calls return after the work they describe has finished
 *   unless stated otherwise.
 * - One handle must not be used by two host threads at the same time.
 * - The device must be an sm_103a GPU (GB300); tn_create fails with
 *   TN_ECUDA otherwise.
 */
#ifndef TNBP_H
#define TNBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tn_status;
#define TN_OK 0
#define TN_EINVAL (-1)         /* bad argument: graph, chi, pointer, size */
#define TN_ENOMEM (-2)         /* allocation failed or footprint over budget */
#define TN_ENOTCONVERGED (-3)  /* BP hit max_iters; results are still written */
#define TN_ENUMERIC (-4)       /* NaN/Inf or a zero-norm message was detected */
#define TN_ETIMEOUT (-5)       /* a device-side wait gave up */
#define TN_ECUDA (-6)          /* a CUDA runtime call failed */
#define TN_EAGAIN (-7)         /* (server) the job is still running */
#define TN_EUNSUPPORTED (-8)   /* valid request the library does not handle */

typedef struct tn_handle tn_handle;

/*
 * Interaction graph.  Vertices are qubits 0..n_vertices-1; edges[2e], edges[2e+1]
 * are the endpoints of edge e.  Every vertex must have degree 1, 2 or 3 and no
 * edge may repeat or be a self-loop (TN_EINVAL otherwise).  The legs of vertex v
 * are its incident edges in increasing edge id; site tensors are indexed
 * T_v[p, leg_0, .., leg_{d-1}] with leg_{d-1} fastest.
 * colour: n_edges proper edge colours (no two edges at one vertex share a
 * colour); the ZZ gates are applied colour layer by colour layer in increasing
 * colour.  NULL lets the library colour the graph (first-fit).
 * periodic: informational flag (1 when the graph is a periodic unit cell whose
 * BP fixed point stands for an infinite lattice).
 */
typedef struct {
  int32_t n_vertices;
  int32_t n_edges;
  const int32_t* edges;
  const uint8_t* colour;
  int32_t periodic;
} tn_graph;

/* Arithmetic of the message and gate contractions (tensor-core modes
 * accumulate in FP32 in tensor memory).  FP64 is used for the BP convergence
 * and normalisation reductions in every mode and for the truncation solve's
 * spectrum.
 *   TN_FP32    plain FP32 on the CUDA cores.
 *   TN_TF32    TF32 operands (10-bit mantissa).
 *   TN_BF16    BF16 operands (7-bit mantissa).
 *   TN_BF16X3, TN_TF32X3  split-precision products: each operand is x = hi + lo
 *              with hi = round(x), lo = round(x - hi) in the operand format, and
 *              the product is accumulated as hi*hi + hi*lo + lo*hi (three
 *              tensor-core products; the dropped lo*lo term is below FP32
 *              rounding for TF32X3, about 2^-16 relative for BF16X3). */
typedef enum {
  TN_FP32 = 0,
  TN_TF32 = 1,
  TN_BF16 = 2,
  TN_BF16X3 = 3,
  TN_TF32X3 = 4
} tn_precision;

typedef struct {
  int32_t chi;          /* maximum bond dimension, 1..256 */
  int32_t prec;         /* tn_precision */
  double bp_tol;        /* BP stops when max_e ||M_new - M_old||_F < bp_tol */
  int32_t bp_max_iters; /* BP sweep cap per regauge */
  double svd_cutoff;    /* singular values below svd_cutoff * sigma_1 are dropped;
                           <= 0 selects the precision's default */
  uint64_t seed;        /* reserved (the method draws no random numbers) */
  int32_t solve;        /* truncation solve: TN_SOLVE_AUTO, _REFINED, _FP64 or _SHARED */
  int32_t kernels;      /* contraction kernels: TN_KERNELS_AUTO or TN_KERNELS_TILE */
  double solve_tol;     /* FP32 Jacobi of the shared and refined solves: it stops when every
                           pair of rows of the bond matrix has |<x_p, x_q>| <= solve_tol
                           ||x_p|| ||x_q||; <= 0 selects the default (refined: 2e-6, the
                           FP32 floor; shared: 2e-6 for TN_FP32, 1e-4 for TN_TF32, 1e-3 for
                           TN_BF16, about the relative rounding of the Gram inputs) */
} tn_config;

/* Contraction kernels of the tensor-core modes.
 * TN_KERNELS_AUTO: with TN_TF32 and chi = 32 or 64, the mode products (one leg
 *   of a site tensor times a chi x chi matrix: the BP sweep's first two
 *   contractions per chain, the gate environments and rebuilds) run in the
 *   persistent TMA-fed streaming kernel; every other contraction, and every
 *   contraction of the other modes, in the generic tile kernel.
 * TN_KERNELS_TILE: the generic tile kernel for every contraction.
 * The two give the same sums in different rounding orders. */
#define TN_KERNELS_AUTO 0
#define TN_KERNELS_TILE 1

/* Truncation solve variants (Methods, "The simple update procedure": the
 * truncated SVD of the 2chi x 2chi bond matrix K = R_v R_w^T, taken as the
 * eigen-decomposition of H = K K^H, from the Gram matrices of both sides).
 * TN_SOLVE_REFINED: FP64 pivoted Cholesky of the v-side Gram blocks; an FP32
 *   one-sided Jacobi of K in shared memory for a starting eigenbasis; one FP64
 *   Newton step (the eigenvector refinement of Ogita and Aishima, 2018) of the
 *   kept chi eigenvectors and eigenvalues of H = R_v conj(G_w) R_v^H; FP64 leg
 *   matrices by triangular solves.  Every quantity the outputs are computed
 *   from is FP64; the FP32 phase only chooses the basis the FP64 step starts
 *   from (chi <= 64; larger chi fall back to TN_SOLVE_FP64).
 * TN_SOLVE_FP64: Hermitian Jacobi eigen-solves of G_v and of H in FP64 on
 *   global-memory workspaces (all arithmetic FP64; slow on GB300, whose FP64
 *   rate is about 1/58 of its FP32 rate).  chi <= 256.
 * TN_SOLVE_SHARED: everything in FP32 in shared memory except the spectrum's
 *   norms (FP64): FP32 pivoted Cholesky of the Gram blocks, one-sided Jacobi of
 *   K with FP32 rotations, FP32 triangular solves for the leg matrices
 *   (chi <= 64; larger chi fall back to TN_SOLVE_FP64).  Singular values to
 *   about 2e-6 relative; end to end about 1e-5 in <Z> against the FP64 oracle.
 * TN_SOLVE_AUTO: TN_SOLVE_REFINED for chi <= 64, TN_SOLVE_FP64 above. */
#define TN_SOLVE_AUTO 0
#define TN_SOLVE_FP64 1
#define TN_SOLVE_SHARED 2
#define TN_SOLVE_REFINED 3

/* Device allocator callbacks.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, size_t bytes, void* ctx, void* stream);
  void* ctx;
} tn_allocator;

/* Counters of the last tn_apply_floquet / tn_bp_converge call. */
typedef struct {
  int32_t steps_done;
  int32_t bp_iters_last;     /* sweeps of the last regauge */
  int32_t bp_iters_total;    /* sweeps summed over the call */
  double bp_residual_last;   /* residual at the end of the last regauge */
  double discarded_max;      /* largest discarded weight sum(sigma^2 dropped)/sum(sigma^2) */
  double discarded_sum;      /* summed over all gates of the call */
  int64_t kernel_launches;   /* device kernels launched by the call */
  int64_t tma_launches;      /* of which launches of the TMA-fed streaming kernel */
  int64_t solve_edges;       /* truncation solves (gate edges) of the call */
  int64_t solve_sweeps;      /* Jacobi rotation sweeps summed over those solves */
  int64_t solve_sweeps_max;  /* the largest count of one solve */
} tn_stats;

/*
 * tn_create — build the state |0...0> (Eq. "State": all spins up) on `graph`
 * with bond dimension cap cfg->chi: T_v[0, 0..0] = 1, every other entry 0, and
 * every message the chi x chi matrix with a single 1 at [0, 0] (the exact BP
 * fixed point of a product state).  *out receives the handle.
 * Errors: TN_EINVAL (graph or config), TN_ENOMEM, TN_ECUDA.
 */
tn_status tn_create(const tn_graph* graph, const tn_config* cfg,
                    const tn_allocator* alloc, void* cuda_stream, tn_handle** out);

/* tn_destroy — release every device and host resource of the handle. */
tn_status tn_destroy(tn_handle* h);

/*
 * tn_apply_floquet — apply U(theta_h) `steps` times (Eq. 1): per step RX(theta_h)
 * = exp(-i theta_h X/2) on every site, then exp(+i pi/4 Z_v Z_w) on every edge
 * by the BP-gauged simple update (Methods, "The simple update procedure": the
 * environment of each tensor is the product of its incoming messages; the
 * two-site bond is truncated to the chi largest singular values by the
 * truncation solve of tn_config; the messages on the gate edge become diag(S)
 * with ||S||_2 = 1), colour
 * layer by colour layer, then BP regauging with the handle's bp_tol and
 * bp_max_iters ("State ansatz": regauge after every Trotter step).
 * theta_h may be any real.  steps >= 0.
 * Errors: TN_EINVAL, TN_ENUMERIC, TN_ENOTCONVERGED (a regauge hit its cap; the
 * evolution still completed), TN_ECUDA.
 */
tn_status tn_apply_floquet(tn_handle* h, double theta_h, int32_t steps);

/*
 * tn_apply_floquet_field — tn_apply_floquet with a kick angle per vertex:
 * RX(theta_v[v]) on site v.  theta_v: n_vertices host doubles (caller-owned,
 * copied at the call).  Used to evolve many independent instances as one
 * graph (their disjoint union): BP and the gates never couple components, so
 * each component evolves as it would alone, while every contraction of every
 * instance runs in the same launches.  Errors: as tn_apply_floquet, plus
 * TN_EINVAL for a null or non-finite theta_v.
 */
tn_status tn_apply_floquet_field(tn_handle* h, const double* theta_v, int32_t steps);

/*
 * tn_apply_clifford_dagger — apply U(pi/2)^dagger `steps` times: the ZZ layers
 * with exp(-i pi/4 Z_v Z_w), then RX(-pi/2), then BP regauging.  This is the
 * "extended time evolution" used to measure the Pauli string
 * U^n'(pi/2) Z_i U^n'(pi/2)^dagger as <Z_i> ("Measuring expectation values").
 */
tn_status tn_apply_clifford_dagger(tn_handle* h, int32_t steps);

/*
 * tn_bp_converge — iterate the BP equations (Eq. "MessageTensorSelfConsistency")
 * with a synchronous schedule from the current messages: every directed message
 * M_{v->w}[e, e'] = sum T_v[p, .., e, ..] conj(T_v[p, .., e', ..]) prod_{x != w}
 * M_{x->v}, then Hermitised and scaled to unit Frobenius norm.  Stops when
 * max_e ||M_new - M_old||_F < tol (FP64 reduction) or after max_iters sweeps.
 * iters_out / residual_out may be NULL.
 * Errors: TN_ENOTCONVERGED (cap reached), TN_ENUMERIC, TN_EINVAL, TN_ECUDA.
 */
tn_status tn_bp_converge(tn_handle* h, double tol, int32_t max_iters,
                         int32_t* iters_out, double* residual_out);

/*
 * tn_bp_components — the connected components of the handle's graph (the
 * instances of a disjoint union, see tn_apply_floquet_field) and what the last
 * BP iteration did on each.  The stop rule of tn_bp_converge and of the
 * regauging in tn_apply_floquet acts on every component separately: a
 * component stops at its own tolerance (or FP32 residual floor, or max_iters)
 * and its messages stay as they are while the others continue, so each
 * instance receives the sweeps it would receive alone.
 *   comp_of_vertex  n_vertices host int32 (may be NULL): component of each vertex,
 *                   numbered in order of their smallest vertex.
 *   sweeps_out      cap host int32 (may be NULL): sweeps of each component in
 *                   the last BP iteration.
 *   residual_out    cap host doubles (may be NULL): its final residual.
 *   n_comp_out      number of components (may be NULL).
 * Arrays are caller-owned; entries past min(cap, n_comp) are not written.
 * Before the first BP iteration sweeps and residuals are 0.
 * Errors: TN_EINVAL (null handle, cap < 0), TN_ECUDA.
 */
tn_status tn_bp_components(tn_handle* h, int32_t* comp_of_vertex, int32_t* sweeps_out,
                           double* residual_out, int32_t cap, int32_t* n_comp_out);

/*
 * tn_autotune — choose the split-K count of every BP-sweep launch that has one
 * (the TMA split-K closes, the tensor-core tile GEMMs, the CUDA-core GEMMs;
 * not the fused chain kernels, whose tiles are fixed) by timing each valid
 * power-of-two count from 1 to 64 on the handle's own state and buffers:
 * one warm-up launch, then `reps` launches timed with CUDA events on the
 * handle's stream.  A count replaces the current one only when it is at least
 * 3% faster.  The launches the captured sweep runs on its side stream keep a
 * single split.  The sweep launches read the state and write only scratch
 * and the raw messages, so the state is unchanged; the next BP iteration
 * captures its loop again with the new counts, and its results may differ
 * from the untuned ones in the last FP32 bits (the order of the partial
 * sums).  Per (chi, degree, precision) the launch shapes fix the key of a
 * table row, so a table tuned on one handle applies to any handle of the same
 * chi, precision and graph shape.
 *   reps       timed launches per candidate, >= 1
 *   table_out  optional (may be NULL): the table as text, one row per tuned
 *              launch: "kind M N K outer inner prec splits us_per_launch\n"
 *              (kind: close, tile or simt), truncated to table_cap - 1 bytes
 *              and NUL-terminated;
 *   table_len  optional: the table's full length in bytes.
 * Errors: TN_EINVAL (null handle, reps < 1), TN_ECUDA.
 */
tn_status tn_autotune(tn_handle* h, int32_t reps, char* table_out, size_t table_cap,
                      size_t* table_len);

/*
 * tn_autotune_apply — set the split counts of a table written by tn_autotune
 * (on this or another handle): every sweep launch whose key (kind, M, N, K,
 * outer, inner, prec) has a row takes that row's count if it is valid for
 * this handle (its partials fit); other launches keep theirs.  table: a
 * NUL-terminated text, caller-owned.  n_applied (may be NULL): rows applied.
 * Errors: TN_EINVAL (null argument).
 */
tn_status tn_autotune_apply(tn_handle* h, const char* table, int32_t* n_applied);

/* A Pauli string sign * prod_j P_{sites[j]}, P in {'X','Y','Z'}; sites distinct. */
typedef struct {
  int32_t weight;
  const int32_t* sites;
  const char* paulis;
  int8_t sign;
} tn_pauli;

/*
 * tn_expect — expectation values of n_ops Pauli strings from the current
 * state and messages (Methods, "Measuring expectation values within the Vidal
 * gauge": the environment of a region is the product of its incoming BP
 * messages).  Weight-1 strings use rho_v[p, p'] = sum T_v[p, ..] conj(T_v[p', ..])
 * prod_x M_{x->v} and <P> = Tr(rho P) / Tr(rho).
 * method 0: strings of weight > 1 are contracted exactly over a tree T_S
 *           spanning their support, every edge leaving T_S closed by its
 *           converged message, and divided by the same contraction without the
 *           operators.  T_S: breadth-first search from the smallest support site
 *           (neighbours in increasing edge id), the union of the search-tree
 *           paths from the other support sites.  Errors: TN_ENUMERIC when the
 *           region's norm contraction vanishes.
 * method 1: "extended time evolution": the library finds (i, n') with
 *           string = +-U^n'(pi/2) Z_i U^n'(pi/2)^dagger by Pauli propagation, evolves
 *           a copy of the state by U(pi/2)^dagger n' times and measures Z_i;
 *           TN_EUNSUPPORTED if no n' <= 32 reduces the string to one Z.
 * out: n_ops doubles (real parts; Pauli strings are Hermitian).
 */
tn_status tn_expect(tn_handle* h, const tn_pauli* ops, int32_t n_ops, int32_t method,
                    double* out);

/*
 * tn_clifford_reduce — host-only: find n' <= max_steps and a site i with
 * op = sign * U^n'(pi/2) Z_i U^n'(pi/2)^dagger ("Measuring expectation values":
 * any such string is one Z conjugated by the Clifford circuit U(pi/2)), by
 * propagating op through U(pi/2)^dagger.  sign_out includes op->sign.
 * Errors: TN_EINVAL (graph or string), TN_EUNSUPPORTED (no such n').
 */
tn_status tn_clifford_reduce(const tn_graph* graph, const tn_pauli* op, int32_t max_steps,
                             int32_t* site_out, int32_t* nprime_out, int32_t* sign_out);

/* tn_expect_z_all — <Z_v> for every vertex v (out: n_vertices doubles). */
tn_status tn_expect_z_all(tn_handle* h, double* out);

/*
 * tn_truncation_solve — the FP64 truncation solve of the simple update (Methods,
 * "The simple update procedure") as a standalone batched call on caller-owned
 * device buffers, on `cuda_stream` (NULL: legacy default stream); returns after
 * the stream has finished it.  For each of n_edges gate edges (v, w):
 *   gram  [edge][side v|w][p][re|im][chi][chi] FP32 (input): the open-p
 *         environments N_p[e, e'] = sum T[p, .., e, ..] conj(T[p, .., e', ..]) prod M
 *         of both sides (the BP message contraction with p left open);
 *   dmat  same shape (output): per side and p the chi x chi matrix D_p with
 *         T'[p, .., n, ..] = sum_e T[p, .., e, ..] D_p[e][n] giving the truncated
 *         two-site update of exp(sign i pi/4 Z Z);
 *   s_out [edge][chi] FP64 (output): the kept singular values with ||S||_2 = 1
 *         (zeros past the rank or below svd_cutoff * sigma_1).
 * The FP64 workspace (12 (2 chi)^2 doubles per edge) is allocated with
 * cudaMallocAsync on the stream and freed before return.
 * Errors: TN_EINVAL, TN_ENUMERIC (zero or non-finite spectrum), TN_ECUDA.
 */
tn_status tn_truncation_solve(const float* gram, float* dmat, double* s_out, int32_t n_edges,
                              int32_t chi, int32_t sign, double svd_cutoff, void* cuda_stream);

/* tn_truncation_solve_ex — tn_truncation_solve with the solve variant chosen:
 * TN_SOLVE_FP64 (what tn_truncation_solve runs), TN_SOLVE_REFINED or
 * TN_SOLVE_SHARED (both chi <= 64, TN_EUNSUPPORTED otherwise), or
 * TN_SOLVE_AUTO (TN_SOLVE_REFINED for chi <= 64, TN_SOLVE_FP64 above). */
tn_status tn_truncation_solve_ex(const float* gram, float* dmat, double* s_out, int32_t n_edges,
                                 int32_t chi, int32_t sign, double svd_cutoff, int32_t solve,
                                 void* cuda_stream);

/*
 * tn_truncation_solve_noalloc — tn_truncation_solve for callers that cannot
 * allocate device memory (a host application or serving runtime that owns the
 * whole device pool, or a latency-bound loop that cannot afford the
 * synchronisation cudaMalloc/cudaFree may imply).  The paper has no
 * counterpart: this is a deployment variant.  Same arguments, layouts, results
 * and errors as tn_truncation_solve; the caller still passes gram, dmat and
 * s_out.  The FP64 workspace is one fixed 16 MiB device array inside the
 * library (held by every GPU that loads it until the process exits), so a call
 * needs n_edges * (12 (2 chi)^2 + 4) + 1 <= 2^21 doubles (for example up to 10
 * edges at chi = 64, 42 at chi = 32); larger requests fail with TN_EINVAL and a
 * message giving the limit.  No cudaMalloc, cudaFree or other allocating call
 * is made.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life of
 * the process; a cudaDeviceReset in the application destroys the context that
 * address belongs to, so do not call this function on that device afterwards.
 * Like tn_truncation_solve it returns only after its stream has finished the
 * work (it reads the error flag back).  Every call shares the one array, which
 * keeps the last call's contents: calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.
 */
tn_status tn_truncation_solve_noalloc(const float* gram, float* dmat, double* s_out,
                                      int32_t n_edges, int32_t chi, int32_t sign,
                                      double svd_cutoff, void* cuda_stream);

/*
 * tn_bond_spectrum — the chi normalised singular values (descending, zero
 * padded, sum of squares 1) that the truncation solve kept on edge e at the
 * edge's last gate (Methods, "The simple update procedure"); the product
 * state's (1, 0, .., 0) before any gate.  out: chi host doubles.
 * tn_entanglement_entropy — s = -sum_i lambda_i^2 log2 lambda_i^2 over that
 * spectrum: the entanglement entropy across the edge in the BP-gauged state
 * (Eq. EntanglementEntropy of "Dynamics of the infinite heavy-hex lattice",
 * read with the minus sign the printed formula lacks).  Errors: TN_EINVAL.
 */
tn_status tn_bond_spectrum(tn_handle* h, int32_t e, double* out);
tn_status tn_entanglement_entropy(tn_handle* h, int32_t e, double* out);

/*
 * Checkpoint / resume of a job's state: the site tensors, the messages and
 * the bond spectra (everything later steps and expectation values read).
 * tn_state_size gives the bytes of the host image; tn_save_state writes it
 * into caller-owned host memory; tn_load_state restores it into a handle
 * created with the same graph (same edges and colour layers) and chi, after
 * which evolution continues exactly as from the saved point.  The precision
 * and solve of the loading handle may differ.  Errors: TN_EINVAL (buffer too
 * small, not a checkpoint, or another graph or chi), TN_ECUDA.
 */
tn_status tn_state_size(const tn_handle* h, size_t* bytes);
tn_status tn_save_state(tn_handle* h, void* host, size_t bytes);
tn_status tn_load_state(tn_handle* h, const void* host, size_t bytes);

/*
 * tn_vidal_gauge — the Vidal gauge (Gamma_v, lambda_e) of the state from its
 * current BP messages (Methods, "The Vidal gauge" and "Belief propagation on
 * a tensor network state": at the BP fixed point the messages define the
 * gauge transformation to the Vidal form, exact on trees).  Per edge e =
 * (u, w): P = sqrt(M_{u->w}), Q = sqrt(M_{w->u}) (Hermitian square roots of
 * the messages u and w send across e), the SVD Q^T P = U diag(lambda) V^H
 * (FP64 on the device), and the leg matrices Q conj(U) lambda^-1 (u's leg) and
 * P V lambda^-1 (w's leg), which every site contracts into each of its legs
 * (FP32) to give Gamma_v: T_v is Gamma_v with lambda_e^1/2 on every leg, and
 * sum over the other indices of Gamma_v conj(Gamma_v) prod_{x != e} lambda_x^2
 * is proportional to the identity on leg e at the fixed point.
 *   lambda_out  n_edges x chi doubles (host, caller-owned): lambda_e in
 *               decreasing order, unit 2-norm, zero past the messages'
 *               support (below 1e-12 lambda_1).
 * Call it on converged messages (tn_apply_floquet and tn_bp_converge end
 * there).  Gamma is kept in the handle (one more state-sized buffer, allocated
 * on the first call) until the next call; tn_get_gamma reads it.  The state
 * and the messages are unchanged.  Errors: TN_EINVAL, TN_ENOMEM, TN_ECUDA,
 * TN_ENUMERIC (a message with no support).
 */
tn_status tn_vidal_gauge(tn_handle* h, double* lambda_out);
/* tn_get_gamma — Gamma_v of the last tn_vidal_gauge call, in the layout of
 * tn_get_site (interleaved complex64, shape (2, chi, .., chi), 4 chi^d floats).
 * Errors: TN_EINVAL (no tn_vidal_gauge yet, vertex out of range, buffer size). */
tn_status tn_get_gamma(tn_handle* h, int32_t v, float* host_out, size_t n_floats);

/*
 * tn_bp_error — the BP error estimate of edge e (Methods, "Estimating the
 * error of BP for general tensor networks", Eq. BPErrorEstimate): the norm
 * network of the state in the symmetric gauge (the Vidal gauge of
 * tn_vidal_gauge with lambda^1/2 on every leg) is cut along e and contracted
 * exactly to the chi^2 x chi^2 edge environment E (rows: the cut index on
 * e's first endpoint, ket x bra; columns: on its second); BP takes E as rank
 * one, and *error = 1 - sqrt(s_1^2 / sum_i s_i^2) over E's singular values s.
 * Exact contraction is exponential in the loops' size: meant for small
 * patches (a few heavy hexagons at small chi).  FP64 on the device after the
 * device gauge (double-layer tensors, pairwise contractions as complex GEMMs
 * in a greedy order planned on the host from the shapes, and the eigenvalues
 * of E^H E by a parallel Jacobi); each bond keeps only the support of its
 * lambda.  Device memory of the contraction is allocated stream-ordered on
 * the handle's stream and released before the call returns.
 *   sv_out       optional (may be NULL): the singular values of E in
 *                decreasing order, up to sv_capacity of them;
 *   n_sv         optional: their number (the squared support of lambda_e).
 * Errors: TN_EINVAL (edge out of range, an intermediate tensor above 2^26
 * elements: the network is too large to contract exactly, or an edge
 * environment above 1024 x 1024, i.e. a support above 32 on the cut edge),
 * TN_ENUMERIC, and those of tn_vidal_gauge.  Leaves the Vidal-gauge tensors
 * of the handle set.
 */
tn_status tn_bp_error(tn_handle* h, int32_t e, double* error, double* sv_out,
                      int32_t sv_capacity, int32_t* n_sv);
/* tn_graph_info — the handle's vertex and edge counts and chi; edges_out
 * (2 * capacity ints, may be NULL) receives the edges (u, w) in edge-id
 * order.  Errors: TN_EINVAL (NULL counts, capacity below the edge count). */
tn_status tn_graph_info(const tn_handle* h, int32_t* n_vertices, int32_t* n_edges, int32_t* chi,
                        int32_t* edges_out, int32_t capacity);

/* tn_get_stats — counters of the last evolution call. */
tn_status tn_get_stats(const tn_handle* h, tn_stats* out);

/*
 * State transfer (tests, checkpoint/resume).  Site tensors cross the ABI as
 * interleaved complex64 (re, im) with shape (2, chi, .., chi) in leg order
 * (2 * chi^d complex values); messages as chi x chi complex64 row-major
 * [ket, bra].  The message from `src` across edge e is selected by (e, src).
 */
tn_status tn_get_site(tn_handle* h, int32_t v, float* host_out, size_t n_floats);
tn_status tn_set_site(tn_handle* h, int32_t v, const float* host_in, size_t n_floats);
tn_status tn_get_message(tn_handle* h, int32_t e, int32_t src, float* host_out,
                         size_t n_floats);
tn_status tn_set_message(tn_handle* h, int32_t e, int32_t src, const float* host_in,
                         size_t n_floats);
/* Bytes of device memory the handle holds (state, messages, workspaces). */
tn_status tn_footprint(const tn_handle* h, size_t* bytes_out);
/* Footprint tn_create would need for this graph and config (admission). */
tn_status tn_footprint_estimate(const tn_graph* graph, const tn_config* cfg,
                                size_t* bytes_out);

/*
 * Serving (continuous batching).  A server runs (graph, chi, theta_h, steps)
 * jobs as they arrive: max_slots host threads, each driving one job at a time
 * on its own CUDA stream, so that concurrent jobs' kernels overlap on the
 * device.  A queued job is admitted (oldest first) once the sum of the
 * resident jobs' footprints (tn_footprint_estimate: state, messages,
 * workspaces) plus its own fits the HBM budget.  A job's device memory is
 * allocated stream-ordered on its slot's stream and released when it ends.
 * Its result, <Z_v> for every vertex after the last step, does not depend on
 * what else runs (no shared buffers; deterministic kernels).
 */
typedef struct tn_server tn_server;

typedef struct {
  size_t hbm_budget;   /* bytes the resident jobs may hold; 0: 90% of free device memory */
  int32_t max_slots;   /* jobs resident and running at once, 1..64 */
  int32_t device;      /* CUDA device ordinal */
  int32_t policy;      /* which queued job a free slot takes (TN_SERVE_*); 0: oldest first */
} tn_server_config;

/* Admission order of a server.  TN_SERVE_FIFO: the oldest queued job, once it
 * fits the HBM budget (later jobs wait behind it).  TN_SERVE_SHORTEST: among
 * the queued jobs that fit, the one with the least estimated work
 * steps x (sum_v d_v chi^(d_v + 1) + 8 n_edges chi^3) (the BP message updates
 * and the truncation solves), the oldest among equals. */
#define TN_SERVE_FIFO 0
#define TN_SERVE_SHORTEST 1

typedef struct {
  tn_graph graph;      /* copied at submit */
  tn_config cfg;       /* chi, precision, tolerances as for tn_create */
  double theta_h;
  int32_t steps;
  const tn_pauli* ops; /* weight-k strings evaluated after the steps, as tn_expect
                          evaluates them (copied at submit; may be NULL) */
  int32_t n_ops;       /* number of strings (0: <Z_v> only) */
  int32_t ops_method;  /* tn_expect's method: 0 BP region, 1 extended evolution */
} tn_job;

typedef struct {
  int32_t status;      /* the job's status: TN_OK, TN_ENOTCONVERGED, or an error */
  int32_t n_vertices;
  int32_t steps_done;
  double queue_s;      /* submit to admission, seconds */
  double latency_s;    /* submit to result, seconds */
} tn_result;

typedef struct {
  int64_t submitted, completed, failed;
  int32_t resident, peak_resident, queued;
  size_t used_bytes, peak_bytes, budget_bytes;
} tn_server_stats;

/* tn_server_create — start the slots.  Errors: TN_EINVAL (max_slots outside
 * 1..64, negative device), TN_ECUDA (no such device). */
tn_status tn_server_create(const tn_server_config* cfg, tn_server** out);
/* tn_server_submit — queue a job; *ticket identifies it.  Errors: TN_EINVAL
 * (graph or config), TN_ENOMEM (its footprint alone exceeds the budget). */
tn_status tn_server_submit(tn_server* s, const tn_job* job, uint64_t* ticket);
/* tn_server_poll — TN_EAGAIN while the job is queued or running; otherwise the
 * job's status, with z (caller-owned, n_vertices doubles, may be NULL) and info
 * (may be NULL) filled; the ticket is then released.  TN_EINVAL: unknown ticket. */
tn_status tn_server_poll(tn_server* s, uint64_t ticket, double* z, tn_result* info);
/* tn_server_wait — tn_server_poll after waiting up to timeout_s seconds
 * (timeout_s <= 0: do not wait; values above 1e9 count as 1e9). */
tn_status tn_server_wait(tn_server* s, uint64_t ticket, double timeout_s, double* z,
                         tn_result* info);
/* tn_server_poll_ex / tn_server_wait_ex — as tn_server_poll / tn_server_wait,
 * and ops_out (caller-owned, the job's n_ops doubles, may be NULL) receives the
 * values of the job's strings (Main text, "Measuring expectation values"), in
 * the order submitted. */
tn_status tn_server_poll_ex(tn_server* s, uint64_t ticket, double* z, double* ops_out,
                            tn_result* info);
tn_status tn_server_wait_ex(tn_server* s, uint64_t ticket, double timeout_s, double* z,
                            double* ops_out, tn_result* info);
tn_status tn_server_get_stats(tn_server* s, tn_server_stats* out);
/* tn_server_destroy — drop queued jobs, wait for the resident ones, join the slots. */
tn_status tn_server_destroy(tn_server* s);

/*
 * tn_chi_extrapolate — linear extrapolation in 1/chi to infinite bond
 * dimension (Main text, the n = 20 results and Fig. F2c, where a fit linear in
 * 1/chi carries the BP-approximated TNS values to chi -> infinity).  For each
 * of n_obs observables k, a least-squares fit of values[i * n_obs + k] =
 * A_k + B_k / chi[i] over the n_chi bond dimensions:
 *   chi       n_chi bond dimensions (host, caller-owned, each > 0, at least two
 *             distinct);
 *   values    n_chi x n_obs row-major (host), e.g. <Z_v> of a chi-ladder run
 *             through the server;
 *   intercept A_k, the chi -> infinity estimate (n_obs doubles, caller-owned);
 *   slope     B_k (n_obs doubles, may be NULL);
 *   rms       root-mean-square fit residual per observable (may be NULL).
 * Host arithmetic only (FP64; no device call).  Errors: TN_EINVAL (NULL
 * arguments, n_chi < 2, n_obs < 1, chi <= 0, all chi equal, non-finite
 * values).
 */
tn_status tn_chi_extrapolate(const double* chi, const double* values, int32_t n_chi,
                             int32_t n_obs, double* intercept, double* slope, double* rms);

/*
 * tn_heavy_hex — the heavy-hex patch with `rows` rows (odd) of `cols` columns
 * (cols = 3 mod 4): row 0 has no last column, the last row no first column;
 * between rows r and r+1 a bridge qubit sits at columns = 0 mod 4 (r even) or
 * 2 mod 4 (r odd); numbering row-major with each bridge row after the row above
 * (Fig. "heavyhexdiagram"; (7, 15) is the 127-qubit Eagle layout with the
 * dangling qubits 13 and 113).  Edges are sorted by (min, max) endpoint.
 * Colours: row edge (r,c)-(r,c+1) gets [0,1,2,1][c%4] on even r and
 * [1,0,1,2][c%4] on odd r; a bridge's upper edge 2 and its lower edge 0.
 * edges_out holds 2*capacity ints, colours_out capacity bytes (either may be
 * NULL to query sizes).  TN_EINVAL if the shape is invalid or capacity short.
 */
tn_status tn_heavy_hex(int32_t rows, int32_t cols, int32_t* n_vertices, int32_t* n_edges,
                       int32_t* edges_out, uint8_t* colours_out, int32_t capacity);

/*
 * Per-kernel-class timing.  While enabled, every kernel the handle launches is
 * bracketed by CUDA events on the handle's stream and its algorithmic work is
 * added to its class: flops = 8 per complex multiply-add of the contraction
 * (40 (2 chi)^3 per edge for the FP64 truncation solve), bytes = every operand
 * element read once and every result written once.  Classes (index: name):
 * 0 bp_contract, 1 bp_normalise, 2 gate_env, 3 trunc_solve, 4 gate_rebuild,
 * 5 copyback, 6 phys_gate, 7 rho.
 */
typedef struct {
  int32_t n_classes;
  int64_t launches[16];
  double ms[16];
  double flops[16];
  double bytes[16];
} tn_profile;
/* tn_profile_enable — switch timing on (1) or off (0); resets the counters. */
tn_status tn_profile_enable(tn_handle* h, int32_t on);
/* tn_profile_read — synchronise the handle's stream and copy the counters. */
tn_status tn_profile_read(tn_handle* h, tn_profile* out);
/* tn_profile_class_name — name of class cls ("" when out of range), static storage. */
const char* tn_profile_class_name(int32_t cls);

/* tn_last_error — message of the calling thread's last failed call ("" if none). */
const char* tn_last_error(void);

/*
 * tn_selftest_bounded_wait — exercises the timeout path of the device-side
 * waits (the paper has no counterpart; it is a check of this library's
 * failure handling).  One thread waits, through the same bounded mbarrier wait
 * the tensor-core kernels use, on a barrier nothing completes; after about one
 * second the wait gives up and sets the timeout bit.  *flags_out receives the
 * flag word: 2 (timeout) when the path works, 4 if the wait returned without
 * giving up.  The call allocates 4 bytes of device memory and synchronises
 * the stream (cuda_stream, may be NULL for the legacy default stream); the
 * context stays usable afterwards.  Errors: TN_EINVAL, TN_ECUDA.
 */
tn_status tn_selftest_bounded_wait(void* cuda_stream, int32_t* flags_out);

/* tn_version — library version string, static storage. */
const char* tn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TNBP_H */
