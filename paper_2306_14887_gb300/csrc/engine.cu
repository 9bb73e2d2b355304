// Engine and C ABI of the tnbp library (declarations in include/tnbp.h).
//
// Device state of a handle, all planar complex FP32 unless noted:
//   T       site tensors, site v at t_off[v]: [re|im][p][leg_0]..[leg_{d-1}]
//           (each plane 2*chi^d floats, legs padded to chi, increasing edge id)
//   Ts      rebuild target of the gate layers (same layout as T)
//   Y1, Y2  intermediates of the leg-by-leg contractions (same layout as T)
//   msg     canonical BP messages [2E][re|im][chi][chi], index [ket][bra];
//           directed id 2e + 0: from eu[e] to ew[e]; 2e + 1: from ew[e] to eu[e]
//   raw     un-normalised messages of the sweep in flight (same layout)
//   gram    open-p environments of a gate layer [slot][side][p][re|im][chi][chi]
//   dmat    per-p gate-leg matrices from the FP64 solve (same layout)
//   work    FP64 solve workspace
//
// One Floquet step (Eq. 1): RX on every site, then per colour layer the gate
// environments (the message contraction with p left open, both sides of every
// edge of the layer), the FP64 truncation solve, the rebuild of both site
// tensors, then BP regauging (synchronous sweeps until the FP64 residual is
// below tol).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <string>
#include <vector>

#include "common.cuh"
#include "graph.h"
#include "tnbp.h"

namespace tnbp {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

namespace {

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

struct HostLaunch {
  GemmDesc d{};
  std::vector<const float*> A, B;
  std::vector<float*> C;
  TcStreamPlan sp;         // maps set: the launch runs in a TMA kernel
  bool fuse_next = false;  // the next launch contracts this one's output (chain stages)
  bool skip = false;       // carried out by the previous launch's fused kernel
  int tuned = 0;           // split-K count chosen by tn_autotune (0: the heuristic)
  std::vector<int> outer_site;  // sweep launches: the site of each outer entry
};

struct Plan {
  std::vector<HostLaunch> L;
};

struct CopyLaunch {
  std::vector<float*> dst;
  std::vector<const float*> src;
  int64_t n_floats = 0;
  float* const* d_dst = nullptr;
  const float* const* d_src = nullptr;
};

struct RhoLaunch {
  int deg = 0;
  std::vector<int64_t> x_off, t_off;
  std::vector<int> sites;
  const int64_t* d_x = nullptr;
  const int64_t* d_t = nullptr;
};

}  // namespace
}  // namespace tnbp

struct tn_handle {
  tnbp::HostGraph g;
  tn_config cfg{};
  int chi = 0;
  cudaStream_t stream = nullptr;
  tn_allocator alloc{};
  bool own_alloc = true;
  std::vector<std::pair<void*, size_t>> allocations;
  size_t bytes = 0;

  std::vector<int64_t> t_off;      // per site (floats)
  std::vector<int64_t> t_len;      // chi^d per site
  int64_t t_floats = 0;
  float *T = nullptr, *Ts = nullptr, *Y1 = nullptr, *Y2 = nullptr;
  float *msg = nullptr, *raw = nullptr, *gram = nullptr, *dmat = nullptr;
  float* part = nullptr;          // K-split partials of tensor-core closes
  float* TA = nullptr;            // site tensors with the first leg moved last
  float* mrt = nullptr;           // realified transposed messages [2E][2chi][2chi]
  float* drt = nullptr;           // realified transposed leg matrices [slot][side][p][2chi][2chi]
  bool ta_valid = false, mrt_valid = false;
  double* work = nullptr;
  double* solve_stats = nullptr;
  double* spectra = nullptr;          // [edges in layer order][chi] last kept bond spectra
  std::vector<int64_t> spec_off;      // per layer: first row of its edges in spectra
  std::vector<int> spec_row;          // per edge: its row in spectra
  int32_t* msg_vw = nullptr;      // per layer slot: directed ids of v->w and w->v
  std::vector<std::vector<int32_t>> layer_msg_vw;  // host copy per layer
  std::vector<int32_t*> d_layer_msg_vw;
  int max_layer = 0;
  unsigned long long* res_bits = nullptr;
  int* flags = nullptr;
  double* rho = nullptr;
  double* rho_part = nullptr;  // [site][block][8] partial sums of rho
  int64_t* site_offs_by_deg[4] = {nullptr, nullptr, nullptr, nullptr};
  float2* rx_cs = nullptr;   // per-site (cos, sin) of theta_v / 2, by degree blocks
  int rx_base[4] = {0, 0, 0, 0};
  int n_by_deg[4] = {0, 0, 0, 0};
  std::vector<int> sites_by_deg[4];

  tnbp::Plan sweep;
  std::vector<tnbp::Plan> gate_env, rebuild;
  std::vector<std::vector<tnbp::CopyLaunch>> copyback;
  tnbp::Plan rho_prep;
  std::vector<tnbp::RhoLaunch> rho_l;
  void* arena = nullptr;

  // backup for the extended-evolution expectation
  float *T_bak = nullptr, *msg_bak = nullptr;
  // Vidal-gauge site tensors of the last tn_vidal_gauge call (same layout as T)
  float* gamma = nullptr;
  // The captured sweep forks onto a second stream: sweep.L[sweep_split..] (the
  // degree-2 chains and degree-1 closes, which share no scratch with the
  // degree-3 chains) runs beside sweep.L[..sweep_split].
  size_t sweep_split = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  tn_stats stats{};
  double* h_stats = nullptr;  // host copy of solve stats
  // one BP sweep captured as a CUDA graph (memset of the status words, the
  // contraction launches, normalisation, read-back of the status words)
  // The BP iteration runs on the device: a graph whose while-loop node repeats
  // the sweep (contractions, normalisation, the stop-rule kernel) until every
  // connected component of the graph has met the stop rule; the host waits
  // once per regauge.
  cudaGraphExec_t loop_exec = nullptr;
  bool loop_unavailable = false;  // the driver refused the conditional node
  double sweep_flops = 0.0, sweep_bytes = 0.0;
  int64_t sweep_kernels = 0, sweep_tma = 0;  // launches inside the captured sweep
  size_t part_floats = 0;                     // size of the split-K partial buffer
  unsigned long long* h_status = nullptr;  // pinned: the stop rule's 5 output words
  // connected components (the instances of a disjoint union)
  int n_comp = 0;
  std::vector<int> comp_of_vertex;
  int* comp_of_msg = nullptr;        // [2E] component of each directed message
  double* comp_state = nullptr;      // [n_comp][4] prev residual, final residual, sweeps, done
  unsigned long long* comp_res = nullptr;  // [n_comp] residual accumulator of a sweep
  double* loop_par = nullptr;              // tol, max_iters, floor
  unsigned long long* loop_out = nullptr;  // the stop rule's output words

  // per-kernel-class timing with CUDA events on the handle's stream
  bool prof_on = false;
  struct ProfEv { int cls; cudaEvent_t a, b; double flops, bytes; };
  std::vector<ProfEv> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  tn_profile prof{};
};

namespace tnbp {
namespace {

void* dev_alloc(tn_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->own_alloc) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  } else {
    p = h->alloc.alloc(bytes, h->alloc.ctx, (void*)h->stream);
    if (!p) return nullptr;
  }
  h->allocations.push_back({p, bytes});
  h->bytes += bytes;
  return p;
}

void dev_free(tn_handle* h, void* p) {
  for (size_t i = 0; i < h->allocations.size(); ++i) {
    if (h->allocations[i].first != p) continue;
    if (h->own_alloc) cudaFree(p);
    else h->alloc.free(p, h->allocations[i].second, h->alloc.ctx, (void*)h->stream);
    h->bytes -= h->allocations[i].second;
    h->allocations.erase(h->allocations.begin() + i);
    return;
  }
}

void dev_free_all(tn_handle* h) {
  for (auto& a : h->allocations) {
    if (h->own_alloc) cudaFree(a.first);
    else h->alloc.free(a.first, a.second, h->alloc.ctx, (void*)h->stream);
  }
  h->allocations.clear();
  h->bytes = 0;
}

int dir_id(const HostGraph& g, int src, int e) { return 2 * e + (g.eu[e] == src ? 0 : 1); }

// ----------------------------------------------------------------- builders
GemmDesc blank_desc(int prec) {
  GemmDesc d;
  memset(&d, 0, sizeof(d));
  d.n_outer = 0;
  d.n_inner = 1;
  d.K1 = 1;
  d.prec = prec;
  d.M2 = 1;
  return d;
}

// Y = X x_j M on degree-d tensors (leg j contracted with M's row index, the
// result keeps M's column index in place of leg j).  Rows are the other
// indices (o, i): o = (p, legs before j), i = legs after j, a two-level row
// index, so that every launch has 2 chi^(d-1) rows per site and the small
// chi x chi matrix is the B operand.  entries: (X, M, Y).
void add_mode_product(Plan& P, int d, int j, int chi, int prec,
                      const std::vector<std::array<const float*, 3>>& ent, bool with_p = true) {
  if (ent.empty()) return;
  HostLaunch L;
  L.d = blank_desc(prec);
  const int64_t inner = ipow(chi, d - 1 - j);
  const int64_t outer = (with_p ? 2 : 1) * ipow(chi, j);
  const int64_t plane = 2 * ipow(chi, d);
  const int64_t c2 = (int64_t)chi * chi;
  L.d.M = (int)(outer * inner);
  L.d.N = chi;
  L.d.K2 = chi;
  L.d.M2 = (int)inner;
  L.d.a_m = chi * inner; L.d.a_m2 = 1; L.d.a_k2 = inner;
  L.d.b_k2 = chi; L.d.b_n = 1;
  L.d.c_m = chi * inner; L.d.c_m2 = 1; L.d.c_n = inner;
  if (inner == 1) { L.d.M2 = 1; L.d.a_m = chi; L.d.c_m = chi; }
  L.d.plane_a = plane; L.d.plane_b = c2; L.d.plane_c = plane;
  for (auto& e : ent) { L.A.push_back(e[0]); L.B.push_back(e[1]); L.C.push_back((float*)e[2]); }
  L.d.n_outer = (int)ent.size();
  P.L.push_back(std::move(L));
}

// out[e][e'] = sum_{all but leg j} Y[.., e, ..] conj(T[.., e', ..]); with open_p
// the sum excludes p and two matrices (p = 0, 1) are written 2*chi^2 apart.
// entries: (Y, T, out).
void add_close(Plan& P, int d, int j, int chi, bool open_p, int prec,
               const std::vector<std::array<const float*, 3>>& ent) {
  if (ent.empty()) return;
  HostLaunch L;
  L.d = blank_desc(prec);
  const int64_t inner = ipow(chi, d - 1 - j);
  const int64_t outer_legs = ipow(chi, j);
  const int64_t plane = 2 * ipow(chi, d);
  const int64_t c2 = (int64_t)chi * chi;
  L.d.M = chi;
  L.d.N = chi;
  L.d.K1 = (int)(open_p ? outer_legs : 2 * outer_legs);
  L.d.K2 = (int)inner;
  L.d.a_m = inner; L.d.a_k1 = chi * inner; L.d.a_k2 = 1;
  L.d.b_k1 = chi * inner; L.d.b_k2 = 1; L.d.b_n = inner;
  L.d.c_m = chi; L.d.c_n = 1;
  L.d.conj_b = 1;
  L.d.plane_a = plane; L.d.plane_b = plane; L.d.plane_c = c2;
  if (open_p) {
    L.d.n_inner = 2;
    L.d.a_in = ipow(chi, d); L.d.b_in = ipow(chi, d); L.d.c_in = 2 * c2;
  }
  for (auto& e : ent) { L.A.push_back(e[0]); L.B.push_back(e[1]); L.C.push_back((float*)e[2]); }
  L.d.n_outer = (int)ent.size();
  P.L.push_back(std::move(L));
}

tn_status upload_plans(tn_handle* h) {
  // gather every pointer array into one arena
  std::vector<const void*> all;
  std::vector<Plan*> plans = {&h->sweep, &h->rho_prep};
  for (auto& p : h->gate_env) plans.push_back(&p);
  for (auto& p : h->rebuild) plans.push_back(&p);
  size_t count = 0;
  for (Plan* p : plans)
    for (auto& L : p->L) count += L.A.size() * 3;
  for (auto& v : h->copyback)
    for (auto& c : v) count += c.dst.size() * 2;
  size_t n64 = 0;
  for (auto& r : h->rho_l) n64 += r.x_off.size() * 2;
  const size_t bytes = count * sizeof(void*) + n64 * sizeof(int64_t);
  void* arena = dev_alloc(h, bytes);
  if (!arena) {
    set_error("device allocation of the plan arena failed");
    return TN_ENOMEM;
  }
  h->arena = arena;
  std::vector<unsigned char> host(bytes);
  size_t pos = 0;
  auto put_ptrs = [&](const void* const* src, size_t n) -> void* {
    void* dev = (unsigned char*)arena + pos;
    memcpy(host.data() + pos, src, n * sizeof(void*));
    pos += n * sizeof(void*);
    return dev;
  };
  for (Plan* p : plans)
    for (auto& L : p->L) {
      L.d.A = (const float* const*)put_ptrs((const void* const*)L.A.data(), L.A.size());
      L.d.B = (const float* const*)put_ptrs((const void* const*)L.B.data(), L.B.size());
      L.d.C = (float* const*)put_ptrs((const void* const*)L.C.data(), L.C.size());
    }
  for (auto& v : h->copyback)
    for (auto& c : v) {
      c.d_dst = (float* const*)put_ptrs((const void* const*)c.dst.data(), c.dst.size());
      c.d_src = (const float* const*)put_ptrs((const void* const*)c.src.data(), c.src.size());
    }
  for (auto& r : h->rho_l) {
    void* dx = (unsigned char*)arena + pos;
    memcpy(host.data() + pos, r.x_off.data(), r.x_off.size() * 8);
    pos += r.x_off.size() * 8;
    void* dt = (unsigned char*)arena + pos;
    memcpy(host.data() + pos, r.t_off.data(), r.t_off.size() * 8);
    pos += r.t_off.size() * 8;
    r.d_x = (const int64_t*)dx;
    r.d_t = (const int64_t*)dt;
  }
  TN_CUDA_TRY(cudaMemcpyAsync(arena, host.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  // tensor maps of the mode products that the streaming kernel takes
  if (h->cfg.prec == TN_TF32 && h->cfg.kernels == TN_KERNELS_AUTO) {
    size_t mbytes = 0;
    for (Plan* p : plans)
      for (auto& L : p->L) mbytes += tc_chain_map_bytes((int)L.A.size() * L.d.n_inner);
    std::vector<unsigned char> hm(mbytes + 64);
    unsigned char* base =
        (unsigned char*)(((uintptr_t)hm.data() + 63) & ~uintptr_t(63));
    std::vector<HostLaunch*> users;
    std::vector<size_t> offs;
    size_t mpos = 0;
    for (Plan* p : plans)
      for (size_t li = 0; li < p->L.size(); ++li) {
        HostLaunch& L = p->L[li];
        TcStreamPlan sp;
        if (L.skip) continue;
        // two chain stages in one pass: the intermediate never reaches HBM
        if (L.fuse_next && li + 1 < p->L.size()) {
          HostLaunch& L2 = p->L[li + 1];
          if ((int)L2.A.size() == (int)L.A.size() &&
              tc_chain_encode(L.d, L2.d, L.A.data(), L.B.data(), L2.A.data(), L2.B.data(),
                              L.C.data(), (int)L.A.size(), base + mpos, &sp)) {
            L.sp = sp;
            L2.skip = true;
            users.push_back(&L);
            offs.push_back(mpos);
            mpos += tc_chain_map_bytes(sp.n_outer);
            continue;
          }
        }
        if (tc_stream_encode(L.d, L.A.data(), L.B.data(), (int)L.A.size(), base + mpos, &sp) ||
            tc_close_encode(L.d, L.A.data(), L.B.data(), (int)L.A.size(), h->part_floats,
                            base + mpos, &sp)) {
          L.sp = sp;
          users.push_back(&L);
          offs.push_back(mpos);
          mpos += tc_stream_map_bytes(sp.n_outer);
        }
      }
    if (mpos > 0) {
      void* dm = dev_alloc(h, mpos);
      if (!dm) {
        set_error("device allocation of the tensor maps failed");
        return TN_ENOMEM;
      }
      TN_CUDA_TRY(cudaMemcpyAsync(dm, base, mpos, cudaMemcpyHostToDevice, h->stream));
      TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
      for (size_t i = 0; i < users.size(); ++i) users[i]->sp.maps = (unsigned char*)dm + offs[i];
      TN_CUDA_TRY(tc_stream_prepare());
    }
  }
  return TN_OK;
}

// ------------------------------------------------------------- profiling
enum { P_BP = 0, P_NORM, P_ENV, P_SOLVE, P_REBUILD, P_COPY, P_PHYS, P_RHO, P_REFINE, P_NCLS };
const char* kProfNames[P_NCLS] = {"bp_contract", "bp_normalise", "gate_env", "trunc_solve",
                                  "gate_rebuild", "copyback", "phys_gate", "rho", "trunc_refine"};

cudaEvent_t next_event(tn_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

tn_status prof_flush(tn_handle* h) {
  if (h->prof_pending.empty()) return TN_OK;
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (auto& p : h->prof_pending) {
    float ms = 0.f;
    TN_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
    h->prof.launches[p.cls] += 1;
    h->prof.ms[p.cls] += ms;
    h->prof.flops[p.cls] += p.flops;
    h->prof.bytes[p.cls] += p.bytes;
  }
  h->prof_pending.clear();
  h->ev_used = 0;
  return TN_OK;
}

// Record an event before a launch (returns the pending index or -1).
int prof_begin(tn_handle* h, int cls) {
  if (!h->prof_on) return -1;
  if (h->ev_used + 2 > 8192) prof_flush(h);
  tn_handle::ProfEv p;
  p.cls = cls;
  p.a = next_event(h);
  p.b = next_event(h);
  p.flops = p.bytes = 0;
  if (!p.a || !p.b) return -1;
  cudaEventRecord(p.a, h->stream);
  h->prof_pending.push_back(p);
  return (int)h->prof_pending.size() - 1;
}

void prof_end(tn_handle* h, int idx, double flops, double bytes) {
  if (idx < 0) return;
  auto& p = h->prof_pending[idx];
  p.flops = flops;
  p.bytes = bytes;
  cudaEventRecord(p.b, h->stream);
}

// Algorithmic work of a GEMM launch: 8 real flops per complex MAC; bytes of
// each operand element read once and each output written once (complex64).
void gemm_work(const GemmDesc& d, double* flops, double* bytes) {
  const double M = d.M, N = d.N, K = (double)d.K1 * d.K2;
  const double bo = d.n_outer, bi = d.n_inner;
  *flops = 8.0 * M * N * K * bo * bi;
  const double a = M * K * bo * (d.a_in ? bi : 1.0);
  const double b = K * N * bo * (d.b_in ? bi : 1.0);
  const double c = M * N * bo * bi;
  *bytes = 8.0 * (a + b + c);
}

bool use_tensor_cores(const tn_handle* h) {
  return h->cfg.prec != TN_FP32;
}

tn_status run_plan(tn_handle* h, const Plan& P, int cls, size_t begin = 0,
                   size_t end = (size_t)-1, bool on_side = false) {
  const cudaStream_t stream = on_side ? h->side : h->stream;
  for (size_t li = begin; li < P.L.size() && li < end; ++li) {
    const HostLaunch& L = P.L[li];
    if (L.skip) continue;
    const int pi = prof_begin(h, cls);
    int nk = 1;
    if (L.sp.maps && L.sp.kind == 2) {
      // two chain stages fused: the second stage's descriptor gives the output
      const GemmDesc& d2 = P.L[li + 1].d;
      TN_CUDA_TRY(launch_tc_chain(L.d, d2, L.sp, h->flags, stream));
      h->stats.tma_launches++;
      if (pi >= 0) {
        double f1, b1, f2, b2;
        gemm_work(L.d, &f1, &b1);
        gemm_work(d2, &f2, &b2);
        // the intermediate is neither written nor read back
        const double y = 8.0 * L.d.M * L.d.N * L.d.n_outer;
        prof_end(h, pi, f1 + f2, b1 + b2 - 2.0 * y);
      }
      h->stats.kernel_launches += 1;
      continue;
    }
    // contractions too small to fill a tensor-core tile pipeline (the
    // degree-1 closes: chi^2 outputs over K = 2) run on the CUDA cores in FP32
    const double macs = (double)L.d.n_outer * L.d.n_inner * L.d.M * L.d.N * L.d.K1 * L.d.K2;
    const bool tiny = macs < 262144.0;
    if (L.sp.maps && L.sp.kind == 1) {
      TN_CUDA_TRY(launch_tc_close(L.d, L.sp, h->part, h->flags, stream));
      h->stats.tma_launches++;
      nk = L.sp.splits > 1 ? 2 : 1;  // the split-K reduce runs only for several splits
    } else if (L.sp.maps) {
      TN_CUDA_TRY(launch_tc_stream(L.d, L.sp, h->flags, stream));
      h->stats.tma_launches++;
    } else if (use_tensor_cores(h) && !tiny) {
      TN_CUDA_TRY(launch_cgemm_tc(L.d, h->part, h->flags, stream, &nk, L.tuned, h->part_floats));
    } else {
      // a tiny-grid launch on the main stream may split K into the partial buffer
      TN_CUDA_TRY(launch_cgemm(L.d, stream, on_side ? nullptr : h->part, h->part_floats, &nk,
                               L.tuned));
    }
    if (pi >= 0) {
      double f, b;
      gemm_work(L.d, &f, &b);
      prof_end(h, pi, f, b);
    }
    h->stats.kernel_launches += nk;
  }
  return TN_OK;
}

// A launch may run on the side stream only if it does not use the shared
// split-K partial buffer.
bool side_safe(const tn_handle* h, const Plan& P, size_t begin) {
  for (size_t li = begin; li < P.L.size(); ++li) {
    const HostLaunch& L = P.L[li];
    if (L.skip) continue;
    if (L.sp.maps) {
      if (L.sp.kind == 2 || (L.sp.kind == 1 && L.sp.splits > 1)) return false;
      continue;
    }
    const double macs = (double)L.d.n_outer * L.d.n_inner * L.d.M * L.d.N * L.d.K1 * L.d.K2;
    if (use_tensor_cores(h) && !(macs < 262144.0)) {
      int q = 0, sp = 1;
      size_t pf = 0;
      tc_plan(L.d, &q, &sp, &pf, L.tuned);
      if (sp > 1) return false;
    } else {
      size_t pf = 0;
      if (cgemm_plan(L.d, &pf, L.tuned) > 1) return false;
    }
  }
  return true;
}

const float* site_ptr(const tn_handle* h, const float* base, int v) { return base + h->t_off[v]; }
const float* msg_ptr(const tn_handle* h, const float* base, int did) {
  return base + (int64_t)did * 2 * h->chi * h->chi;
}
// incoming message into v along edge e
const float* in_msg(const tn_handle* h, int v, int e) {
  return msg_ptr(h, h->msg, dir_id(h->g, h->g.other(e, v), e));
}

using Ent = std::array<const float*, 3>;

// A contraction spec: every stride of a GemmDesc, filled by the builders below.
struct Spec {
  int M, N, K1 = 1, K2, M2 = 1, M3 = 1;
  int64_t a_m, a_m2 = 0, a_m3 = 0, a_k1 = 0, a_k2;
  int64_t b_n, b_k1 = 0, b_k2;
  int64_t c_m, c_m2 = 0, c_m3 = 0, c_n;
  int64_t plane_a, plane_b, plane_c;
  int n_inner = 1;
  int64_t a_in = 0, b_in = 0, c_in = 0;
  int conj_b = 0, b_pre = 0;
};

void add_spec(Plan& P, const Spec& sp, int prec, const std::vector<Ent>& ent) {
  if (ent.empty()) return;
  HostLaunch L;
  L.d = blank_desc(prec);
  GemmDesc& d = L.d;
  d.M = sp.M; d.N = sp.N; d.K1 = sp.K1; d.K2 = sp.K2; d.M2 = sp.M2; d.M3 = sp.M3;
  d.a_m = sp.a_m; d.a_m2 = sp.a_m2; d.a_m3 = sp.a_m3; d.a_k1 = sp.a_k1; d.a_k2 = sp.a_k2;
  d.b_n = sp.b_n; d.b_k1 = sp.b_k1; d.b_k2 = sp.b_k2;
  d.c_m = sp.c_m; d.c_m2 = sp.c_m2; d.c_m3 = sp.c_m3; d.c_n = sp.c_n;
  d.plane_a = sp.plane_a; d.plane_b = sp.plane_b; d.plane_c = sp.plane_c;
  d.n_inner = sp.n_inner; d.a_in = sp.a_in; d.b_in = sp.b_in; d.c_in = sp.c_in;
  d.conj_b = sp.conj_b; d.b_pre = sp.b_pre;
  for (auto& e : ent) { L.A.push_back(e[0]); L.B.push_back(e[1]); L.C.push_back((float*)e[2]); }
  d.n_outer = (int)ent.size();
  P.L.push_back(std::move(L));
}

// Mode product Y = X x_leg Mt with the contracted leg fastest in X's rows (each
// row of X holds chi contiguous values of the contracted leg) and the small
// operand given realified and transposed (b_pre).  rows: number of rows per
// entry; the row levels and output strides come from the caller.
Spec mode_spec(int chi, int64_t plane, int M, int M2, int M3, int64_t a_m, int64_t a_m2,
               int64_t a_m3, int64_t c_m, int64_t c_m2, int64_t c_m3, int64_t c_n) {
  Spec sp;
  sp.M = M; sp.N = chi; sp.K1 = 1; sp.K2 = chi; sp.M2 = M2; sp.M3 = M3;
  sp.a_m = a_m; sp.a_m2 = a_m2; sp.a_m3 = a_m3; sp.a_k2 = 1;
  sp.b_pre = 1; sp.b_n = 2 * chi; sp.b_k1 = chi; sp.b_k2 = 1; sp.plane_b = 2LL * chi * chi;
  sp.c_m = c_m; sp.c_m2 = c_m2; sp.c_m3 = c_m3; sp.c_n = c_n;
  sp.plane_a = plane; sp.plane_c = plane;
  return sp;
}

// Close out[e][e'] = sum_K Y[e][K] conj(X[e'][K]) with both operands K-contiguous.
Spec close_spec(int chi, int64_t plane, int K1, int K2, int64_t a_m, int64_t a_k1, int64_t b_n,
                int64_t b_k1) {
  Spec sp;
  sp.M = chi; sp.N = chi; sp.K1 = K1; sp.K2 = K2;
  sp.a_m = a_m; sp.a_k1 = a_k1; sp.a_k2 = 1;
  sp.b_n = b_n; sp.b_k1 = b_k1; sp.b_k2 = 1;
  sp.c_m = chi; sp.c_n = 1;
  sp.plane_a = plane; sp.plane_b = plane; sp.plane_c = (int64_t)chi * chi;
  sp.conj_b = 1;
  return sp;
}

const float* mrt_ptr(const tn_handle* h, int did) {
  return h->mrt + (int64_t)did * 4 * h->chi * h->chi;
}
// realified transposed incoming message into v along edge e
const float* in_mrt(const tn_handle* h, int v, int e) {
  return mrt_ptr(h, dir_id(h->g, h->g.other(e, v), e));
}

// Degree-3 chains (legs a, b, c of T[p][a][b][c]; TA[p][b][c][a]):
//   A1  Y1[(p,a,c')][b]   = T  x_c Mc        A2  Y2[a][p][b'][c'] = Y1 x_b Mb
//   B1  Y1[(p,b,c')][a]   = T  x_c Mc        B2  Y2[b][p][a'][c'] = Y1 x_a Ma
//   C1  Y1[(p,c,a')][b]   = TA x_a Ma        C2  Y2[c][p][b'][a'] = Y1 x_b Mb
// each followed by the close on the open leg against T (chains A, B) or TA (C).
// Operands of one site's chain: ket tensor and its first-leg-last copy, the
// bra (the same tensor, or the tensor with an operator applied on p) and its
// copy, the site's intermediate slots, the realified transposed incoming
// message per leg position, and the output.
struct ChainSite {
  const float *T, *TA, *bra, *braA, *Y1, *Y2;
  const float* m[3];
  float* out;
};

ChainSite handle_site(const tn_handle* h, int v, float* out) {
  const auto& lg = h->g.legs[v];
  ChainSite c;
  c.T = c.bra = site_ptr(h, h->T, v);
  c.TA = c.braA = site_ptr(h, h->TA, v);
  c.Y1 = site_ptr(h, h->Y1, v);
  c.Y2 = site_ptr(h, h->Y2, v);
  for (int j = 0; j < 3; ++j) c.m[j] = j < (int)lg.size() ? in_mrt(h, v, lg[j]) : nullptr;
  c.out = out;
  return c;
}

void deg3_chain_sites(tn_handle* h, Plan& P, int which, const std::vector<ChainSite>& cs,
                      bool open_p) {
  const int x = h->chi, prec = h->cfg.prec;
  const int64_t x2 = (int64_t)x * x, x3 = x2 * x, plane = 2 * x3;
  std::vector<Ent> e1, e2, ec;
  for (const ChainSite& c : cs) {
    if (which == 0) {
      e1.push_back({c.T, c.m[2], c.Y1});
      e2.push_back({c.Y1, c.m[1], c.Y2});
      ec.push_back({c.Y2, c.bra, c.out});
    } else if (which == 1) {
      e1.push_back({c.T, c.m[2], c.Y1});
      e2.push_back({c.Y1, c.m[0], c.Y2});
      ec.push_back({c.Y2, c.bra, c.out});
    } else {
      e1.push_back({c.TA, c.m[0], c.Y1});
      e2.push_back({c.Y1, c.m[1], c.Y2});
      ec.push_back({c.Y2, c.braA, c.out});
    }
  }
  const int M = (int)(2 * x2);
  Spec s1, s2, sc;
  if (which == 0) {
    // rows (p,a,b) of T -> Y1 at (pa) x^2 + c' x + b
    s1 = mode_spec(x, plane, M, x, 1, x2, x, 0, x2, 1, 0, x);
    // rows (p,a,c') of Y1 -> Y2 at a 2x^2 + p x^2 + b' x + c'
    s2 = mode_spec(x, plane, M, x, x, x3, x2, x, x2, 2 * x2, 1, x);
    sc = close_spec(x, plane, 2, (int)x2, 2 * x2, x2, x2, x3);
    if (open_p) { sc.K1 = 1; sc.n_inner = 2; sc.a_in = x2; sc.b_in = x3; sc.c_in = 2 * x2; }
  } else if (which == 1) {
    // rows enumerated (p,b,a) so that a, contiguous in the output, is the fastest
    // row index: T row at p x^3 + a x^2 + b x -> Y1 at p x^3 + b x^2 + c' x + a
    s1 = mode_spec(x, plane, M, x, x, x3, x, x2, x3, x2, 1, x);
    // rows (p,b,c') of Y1 -> Y2 at b 2x^2 + p x^2 + a' x + c'
    s2 = mode_spec(x, plane, M, x, x, x3, x2, x, x2, 2 * x2, 1, x);
    sc = close_spec(x, plane, 2 * x, x, 2 * x2, x, x, x2);
    if (open_p) { sc.K1 = x; sc.n_inner = 2; sc.a_in = x2; sc.b_in = x3; sc.c_in = 2 * x2; }
  } else {
    // rows enumerated (p,c,b): TA row at p x^3 + b x^2 + c x -> Y1 at
    // p x^3 + c x^2 + a' x + b (b, the fastest row index, contiguous)
    s1 = mode_spec(x, plane, M, x, x, x3, x, x2, x3, x2, 1, x);
    // rows (p,c,a') of Y1 -> Y2 at c 2x^2 + p x^2 + b' x + a'
    s2 = mode_spec(x, plane, M, x, x, x3, x2, x, x2, 2 * x2, 1, x);
    sc = close_spec(x, plane, 2 * x, x, 2 * x2, x, x, x2);
    if (open_p) { sc.K1 = x; sc.n_inner = 2; sc.a_in = x2; sc.b_in = x3; sc.c_in = 2 * x2; }
  }
  add_spec(P, s1, prec, e1);
  if (!e1.empty()) P.L.back().fuse_next = true;  // Y1 feeds only the second product
  add_spec(P, s2, prec, e2);
  add_spec(P, sc, prec, ec);
}

void deg3_chain(tn_handle* h, Plan& P, int which, const std::vector<int>& sites, bool open_p,
                const std::vector<float*>& outs) {
  std::vector<ChainSite> cs;
  for (size_t i = 0; i < sites.size(); ++i) cs.push_back(handle_site(h, sites[i], outs[i]));
  deg3_chain_sites(h, P, which, cs, open_p);
}

// Degree-2 chains (T[p][a][b], TA[p][b][a]):
//   which 0: Y1[a][p][b'] = T x_b Mb, close on a against T
//   which 1: Y1[b][p][a'] = TA x_a Ma, close on b against TA
void deg2_chain_sites(tn_handle* h, Plan& P, int which, const std::vector<ChainSite>& cs,
                      bool open_p) {
  const int x = h->chi, prec = h->cfg.prec;
  const int64_t x2 = (int64_t)x * x, plane = 2 * x2;
  std::vector<Ent> e1, ec;
  for (const ChainSite& c : cs) {
    const float* src = which == 0 ? c.T : c.TA;
    const float* bra = which == 0 ? c.bra : c.braA;
    const float* Y1 = which == 0 ? c.Y1 : c.Y2;
    e1.push_back({src, c.m[which == 0 ? 1 : 0], Y1});
    ec.push_back({Y1, bra, c.out});
  }
  // rows (p, l) of the source -> Y1 at l 2x + p x + n
  Spec s1 = mode_spec(x, plane, (int)(2 * x), x, 1, x2, x, 0, x, 2 * x, 0, 1);
  Spec sc = close_spec(x, plane, 2, x, 2 * x, x, x, x2);
  if (open_p) { sc.K1 = 1; sc.n_inner = 2; sc.a_in = x; sc.b_in = x2; sc.c_in = 2 * x2; }
  add_spec(P, s1, prec, e1);
  add_spec(P, sc, prec, ec);
}


void deg2_chain(tn_handle* h, Plan& P, int which, const std::vector<int>& sites, bool open_p,
                const std::vector<float*>& outs) {
  std::vector<ChainSite> cs;
  for (size_t i = 0; i < sites.size(); ++i) cs.push_back(handle_site(h, sites[i], outs[i]));
  deg2_chain_sites(h, P, which, cs, open_p);
}

void build_sweep_plan(tn_handle* h) {
  const HostGraph& g = h->g;
  Plan& P = h->sweep;
  // All sites of a degree in one launch per chain stage: grouping the sites so
  // that a group's intermediates stay in L2 costs more in lost parallelism
  // than it saves in traffic (measured at chi = 64 on 127 qubits).
  // every launch's outer entries are the sites of one degree, in list order
  auto tag = [&](size_t from, const std::vector<int>& sites) {
    for (size_t i = from; i < P.L.size(); ++i) P.L[i].outer_site = sites;
  };
  const std::vector<int>& s3 = h->sites_by_deg[3];
  for (int which = 0; which < 3; ++which) {
    std::vector<float*> outs;
    for (int v : s3) outs.push_back((float*)msg_ptr(h, h->raw, dir_id(g, v, g.legs[v][which])));
    const size_t from = P.L.size();
    deg3_chain(h, P, which, s3, false, outs);
    tag(from, s3);
  }
  h->sweep_split = P.L.size();
  const std::vector<int>& s2 = h->sites_by_deg[2];
  for (int which = 0; which < 2; ++which) {
    std::vector<float*> outs;
    for (int v : s2) outs.push_back((float*)msg_ptr(h, h->raw, dir_id(g, v, g.legs[v][which])));
    const size_t from = P.L.size();
    deg2_chain(h, P, which, s2, false, outs);
    tag(from, s2);
  }
  std::vector<Ent> d1;
  for (int v : h->sites_by_deg[1]) {
    const float* T = site_ptr(h, h->T, v);
    d1.push_back({T, T, msg_ptr(h, h->raw, dir_id(g, v, g.legs[v][0]))});
  }
  const size_t from = P.L.size();
  add_close(P, 1, 0, h->chi, false, h->cfg.prec, d1);
  tag(from, h->sites_by_deg[1]);
}

// A union of several components: every sweep launch gets the component of
// each of its outer entries, so that the kernels that honour it skip the
// components that have met the stop rule.
tn_status attach_components(tn_handle* h) {
  if (h->n_comp <= 1) return TN_OK;
  for (auto& L : h->sweep.L) {
    if (L.outer_site.empty() || (int)L.outer_site.size() != L.d.n_outer) continue;
    std::vector<int> comp(L.outer_site.size());
    for (size_t i = 0; i < comp.size(); ++i) comp[i] = h->comp_of_vertex[L.outer_site[i]];
    int* dc = (int*)dev_alloc(h, sizeof(int) * comp.size());
    if (!dc) { set_error("device allocation of the component tables failed"); return TN_ENOMEM; }
    if (cudaMemcpy(dc, comp.data(), sizeof(int) * comp.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      set_error("upload of the component tables failed");
      return TN_ECUDA;
    }
    L.d.outer_comp = dc;
    L.d.comp_state = h->comp_state;
  }
  return TN_OK;
}

// Environments of both sides of every edge in layer `li`, open p, into gram;
// rebuild of both site tensors from the solve's leg matrices, into Ts.
void build_gate_plans(tn_handle* h, int li) {
  const int x = h->chi, prec = h->cfg.prec;
  const HostGraph& g = h->g;
  const auto& layer = g.layers[li];
  const int64_t c2 = (int64_t)x * x;
  Plan env, reb;
  std::vector<std::array<int, 3>> sides[4][3];  // (v, slot, side) by (degree, leg position)
  for (int s = 0; s < (int)layer.size(); ++s) {
    const int e = layer[s];
    const int ends[2] = {g.eu[e], g.ew[e]};
    for (int side = 0; side < 2; ++side) {
      const int v = ends[side];
      sides[g.degree(v)][g.leg_pos(v, e)].push_back({v, s, side});
    }
  }
  auto gram_ptr = [&](int slot, int side) { return h->gram + ((int64_t)slot * 2 + side) * 4 * c2; };
  auto drt_ptr = [&](int slot, int side, int p) {
    return h->drt + (((int64_t)slot * 2 + side) * 2 + p) * 4 * c2;
  };
  for (int j = 0; j < 3; ++j) {
    std::vector<int> vs;
    std::vector<float*> outs;
    for (auto& sd : sides[3][j]) { vs.push_back(sd[0]); outs.push_back(gram_ptr(sd[1], sd[2])); }
    if (!vs.empty()) deg3_chain(h, env, j, vs, true, outs);
  }
  for (int j = 0; j < 2; ++j) {
    std::vector<int> vs;
    std::vector<float*> outs;
    for (auto& sd : sides[2][j]) { vs.push_back(sd[0]); outs.push_back(gram_ptr(sd[1], sd[2])); }
    if (!vs.empty()) deg2_chain(h, env, j, vs, true, outs);
  }
  {
    std::vector<Ent> c;
    for (auto& sd : sides[1][0]) {
      const float* T = site_ptr(h, h->T, sd[0]);
      c.push_back({T, T, gram_ptr(sd[1], sd[2])});
    }
    add_close(env, 1, 0, x, true, prec, c);
  }
  // rebuild T'_p = T_p x_leg D_p for each (site, p), the contracted leg read
  // where it is fastest (T for the last leg, TA for the first leg)
  const int64_t x2 = c2;
  std::vector<CopyLaunch> cps(4);
  for (int d = 1; d <= 3; ++d)
    for (int j = 0; j < d; ++j) {
      if (sides[d][j].empty()) continue;
      const int64_t plane = 2 * ipow(x, d);
      const bool first = (j == 0 && d >= 2);
      std::vector<Ent> ent;
      for (auto& sd : sides[d][j]) {
        const int v = sd[0];
        const int64_t len = h->t_len[v];
        for (int p = 0; p < 2; ++p)
          ent.push_back({site_ptr(h, first ? h->TA : h->T, v) + p * len, drt_ptr(sd[1], sd[2], p),
                         site_ptr(h, h->Ts, v) + p * len});
        cps[d].dst.push_back(h->T + h->t_off[v]);
        cps[d].src.push_back(h->Ts + h->t_off[v]);
        cps[d].n_floats = 4 * len;
      }
      Spec sp;
      if (d == 3 && j == 2) sp = mode_spec(x, plane, (int)x2, 1, 1, x, 0, 0, x, 0, 0, 1);
      else if (d == 3 && j == 0) sp = mode_spec(x, plane, (int)x2, 1, 1, x, 0, 0, 1, 0, 0, x2);
      else if (d == 3 && j == 1) {
        // rows (a, c), the contracted leg b at stride chi
        sp = mode_spec(x, plane, (int)x2, x, 1, x2, 1, 0, x2, 1, 0, x);
        sp.a_k2 = x;
      } else if (d == 2 && j == 1) sp = mode_spec(x, plane, x, 1, 1, x, 0, 0, x, 0, 0, 1);
      else if (d == 2 && j == 0) sp = mode_spec(x, plane, x, 1, 1, x, 0, 0, 1, 0, 0, x);
      else sp = mode_spec(x, plane, 1, 1, 1, x, 0, 0, x, 0, 0, 1);  // degree 1
      add_spec(reb, sp, prec, ent);
    }
  h->gate_env[li] = std::move(env);
  h->rebuild[li] = std::move(reb);
  std::vector<CopyLaunch> keep;
  for (int d = 1; d <= 3; ++d)
    if (!cps[d].dst.empty()) keep.push_back(std::move(cps[d]));
  h->copyback[li] = std::move(keep);
}

void build_rho_plan(tn_handle* h) {
  const int chi = h->chi, prec = h->cfg.prec;
  const HostGraph& g = h->g;
  Plan& P = h->rho_prep;
  std::vector<Ent> a, b, c;
  // degree 3: Y1 = T x_2 M2 ; Y2 = Y1 x_1 M1 ; Y1 = Y2 x_0 M0
  for (int v : h->sites_by_deg[3]) {
    const auto& lg = g.legs[v];
    a.push_back({site_ptr(h, h->T, v), in_msg(h, v, lg[2]), site_ptr(h, h->Y1, v)});
    b.push_back({site_ptr(h, h->Y1, v), in_msg(h, v, lg[1]), site_ptr(h, h->Y2, v)});
    c.push_back({site_ptr(h, h->Y2, v), in_msg(h, v, lg[0]), site_ptr(h, h->Y1, v)});
  }
  add_mode_product(P, 3, 2, chi, prec, a);
  add_mode_product(P, 3, 1, chi, prec, b);
  add_mode_product(P, 3, 0, chi, prec, c);
  a.clear(); b.clear();
  // degree 2: Y1 = T x_0 M0 ; Y2 = Y1 x_1 M1 -> result in Y2, copy pointer for rho
  for (int v : h->sites_by_deg[2]) {
    const auto& lg = g.legs[v];
    a.push_back({site_ptr(h, h->T, v), in_msg(h, v, lg[0]), site_ptr(h, h->Y2, v)});
    b.push_back({site_ptr(h, h->Y2, v), in_msg(h, v, lg[1]), site_ptr(h, h->Y1, v)});
  }
  add_mode_product(P, 2, 0, chi, prec, a);
  add_mode_product(P, 2, 1, chi, prec, b);
  a.clear();
  for (int v : h->sites_by_deg[1])
    a.push_back({site_ptr(h, h->T, v), in_msg(h, v, g.legs[v][0]), site_ptr(h, h->Y1, v)});
  add_mode_product(P, 1, 0, chi, prec, a);
  // every degree ends with X in Y1
  for (int d = 1; d <= 3; ++d) {
    if (h->sites_by_deg[d].empty()) continue;
    RhoLaunch r;
    r.deg = d;
    for (int v : h->sites_by_deg[d]) {
      r.sites.push_back(v);
      r.x_off.push_back(h->t_off[v]);
      r.t_off.push_back(h->t_off[v]);
    }
    h->rho_l.push_back(std::move(r));
  }
}

// --------------------------------------------------------------- execution
tn_status check_flags(tn_handle* h, const char* where) {
  int f = 0;
  TN_CUDA_TRY(cudaMemcpyAsync(&f, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (f) {
    TN_CUDA_TRY(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
    if (f & 2) {
      set_error(std::string("a device-side wait gave up in ") + where);
      return TN_ETIMEOUT;
    }
    set_error(std::string("non-finite or zero-norm values detected in ") + where);
    return TN_ENUMERIC;
  }
  return TN_OK;
}

// TA (first leg last) must match T before any plan that reads it.
tn_status ensure_ta(tn_handle* h) {
  if (h->ta_valid) return TN_OK;
  for (int d = 2; d <= 3; ++d) {
    if (!h->n_by_deg[d]) continue;
    TN_CUDA_TRY(launch_first_leg_last(h->T, h->TA, h->site_offs_by_deg[d], h->n_by_deg[d], d,
                                      h->chi, h->stream));
    h->stats.kernel_launches++;
  }
  h->ta_valid = true;
  return TN_OK;
}

// The realified transposed messages must match msg before any mode product.
tn_status ensure_mrt(tn_handle* h) {
  if (h->mrt_valid) return TN_OK;
  const int nmsg = 2 * (int)h->g.eu.size();
  TN_CUDA_TRY(launch_realify(h->msg, 2LL * h->chi * h->chi, h->mrt, nmsg, h->chi, h->stream));
  h->stats.kernel_launches++;
  h->mrt_valid = true;
  return TN_OK;
}

tn_status phys_gate(tn_handle* h, const double u[8]) {
  h->ta_valid = false;
  for (int d = 1; d <= 3; ++d) {
    if (!h->n_by_deg[d]) continue;
    const int64_t len = ipow(h->chi, d);
    const int pi = prof_begin(h, P_PHYS);
    TN_CUDA_TRY(launch_phys_gate(h->T, h->site_offs_by_deg[d], h->n_by_deg[d], len, 2 * len,
                                 (float)u[0], (float)u[1], (float)u[2], (float)u[3], (float)u[4],
                                 (float)u[5], (float)u[6], (float)u[7], h->stream));
    prof_end(h, pi, 28.0 * len * h->n_by_deg[d], 2.0 * 16.0 * len * h->n_by_deg[d]);
    h->stats.kernel_launches++;
  }
  return TN_OK;
}

// RX(theta_v) with a per-site angle: (cos, sin) of theta_v / 2 uploaded once
// per call, then one launch per degree each step.
tn_status upload_rx_field(tn_handle* h, const double* theta_v) {
  std::vector<float2> cs(h->g.n);
  for (int d = 1; d <= 3; ++d)
    for (int i = 0; i < h->n_by_deg[d]; ++i) {
      const double th = theta_v[h->sites_by_deg[d][i]];
      cs[h->rx_base[d] + i] = make_float2((float)cos(th / 2), (float)sin(th / 2));
    }
  TN_CUDA_TRY(cudaMemcpyAsync(h->rx_cs, cs.data(), sizeof(float2) * cs.size(),
                              cudaMemcpyHostToDevice, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return TN_OK;
}

tn_status phys_gate_field(tn_handle* h) {
  h->ta_valid = false;
  for (int d = 1; d <= 3; ++d) {
    if (!h->n_by_deg[d]) continue;
    const int64_t len = ipow(h->chi, d);
    const int pi = prof_begin(h, P_PHYS);
    TN_CUDA_TRY(launch_phys_gate_field(h->T, h->site_offs_by_deg[d], h->rx_cs + h->rx_base[d],
                                       h->n_by_deg[d], len, 2 * len, h->stream));
    prof_end(h, pi, 16.0 * len * h->n_by_deg[d], 2.0 * 16.0 * len * h->n_by_deg[d]);
    h->stats.kernel_launches++;
  }
  return TN_OK;
}

void rx_matrix(double theta, double u[8]) {
  const double c = cos(theta / 2), s = sin(theta / 2);
  // [[c, -i s], [-i s, c]]
  u[0] = c; u[1] = 0; u[2] = 0; u[3] = -s;
  u[4] = 0; u[5] = -s; u[6] = c; u[7] = 0;
}

// Orthogonality tolerance of the shared solve's Jacobi: about the relative
// rounding of its Gram inputs, which the contraction precision sets.
double solve_tol(const tn_handle* h) {
  if (h->cfg.solve_tol > 0) return h->cfg.solve_tol;
  if (h->cfg.prec == TN_TF32) return 1e-4;
  if (h->cfg.prec == TN_BF16) return 1e-3;
  if (h->cfg.prec == TN_BF16X3) return 1e-5;
  return 2e-6;
}

double default_svd_cut(const tn_handle* h) {
  if (h->cfg.svd_cutoff > 0) return h->cfg.svd_cutoff;
  return h->cfg.prec == TN_FP32 || h->cfg.prec == TN_TF32X3 || h->cfg.prec == TN_BF16X3 ? 1e-6
                                                                                       : 1e-4;
}

// The solve a handle runs: TN_SOLVE_REFINED, TN_SOLVE_SHARED or TN_SOLVE_FP64.
int solve_kind(int solve, int chi) {
  if (solve == TN_SOLVE_AUTO) solve = TN_SOLVE_REFINED;
  if (solve == TN_SOLVE_REFINED && !solve_refined_supported(chi)) return TN_SOLVE_FP64;
  if (solve == TN_SOLVE_SHARED && !solve32_supported(chi)) return TN_SOLVE_FP64;
  return solve;
}

// Residual below which FP32-stored messages can no longer improve.
double precision_floor(const tn_handle* h) {
  switch (h->cfg.prec) {
    case TN_TF32: return 2e-3;
    case TN_BF16: return 2e-2;
    case TN_BF16X3: return 2e-5;  // split BF16: about 16 significant bits per operand
    default: return 2e-6;         // FP32 and split TF32 (about 21 bits)
  }
}

tn_status gate_layer(tn_handle* h, int li, int sign) {
  tn_status st = ensure_ta(h);
  if (st) return st;
  st = ensure_mrt(h);
  if (st) return st;
  st = run_plan(h, h->gate_env[li], P_ENV);
  if (st) return st;
  SolveArgs a;
  a.n_edges = (int)h->g.layers[li].size();
  a.chi = h->chi;
  a.sign = sign;
  a.gram_cut = 1e-13;
  a.svd_cut = default_svd_cut(h);
  a.gram = h->gram;
  a.dmat = h->dmat;
  a.msg = h->msg;
  a.msg_vw = h->d_layer_msg_vw[li];
  a.work = h->work;
  a.stats = h->solve_stats;
  a.flags = h->flags;
  a.max_sweeps = 30;
  a.s_out = h->spectra + h->spec_off[li] * h->chi;
  {
    const int pi = prof_begin(h, P_SOLVE);
    const int kind = solve_kind(h->cfg.solve, h->chi);
    if (kind == TN_SOLVE_REFINED) {
      a.max_sweeps = 20;
      a.orth_tol = h->cfg.solve_tol > 0 ? (float)h->cfg.solve_tol : 2e-6f;
      TN_CUDA_TRY(launch_solve_refined_basis(a, h->stream));
      const double n = 2.0 * h->chi, x = h->chi;
      // FP32 phase (Jacobi sweeps: about 7 of n^2/2 pairs x 16 n real flops)
      prof_end(h, pi, 7.0 * n * n / 2 * 16.0 * n * a.n_edges, 0.0);
      // FP64 phase: Newton step (Y, P: chi^3 each; Z through the two open-q
      // environments: n^2 chi / 2; S, R and the update: n^2 chi each) and the
      // leg matrices (2 chi^3), 8 real flops per cMAC
      const int pr = prof_begin(h, P_REFINE);
      TN_CUDA_TRY(launch_solve_refined_newton(a, h->stream));
      prof_end(h, pr, 8.0 * (4.0 * x * x * x + 3.5 * n * n * x) * a.n_edges,
               (16.0 * (2.0 * n * n + n * x) + 4.0 * n * n) * a.n_edges);
      h->stats.kernel_launches += 3;
    } else if (kind == TN_SOLVE_SHARED) {
      a.max_sweeps = 20;
      a.orth_tol = (float)solve_tol(h);
      TN_CUDA_TRY(launch_solve32(a, h->stream));
    } else {
      TN_CUDA_TRY(launch_solve(a, h->stream));
    }
    if (kind != TN_SOLVE_REFINED) {
      const double n = 2.0 * h->chi;
      prof_end(h, pi, 40.0 * n * n * n * a.n_edges, 4.0 * 16.0 * h->chi * h->chi * a.n_edges);
    }
  }
  h->stats.kernel_launches++;
  h->mrt_valid = false;  // the solve rewrote the gate-edge messages
  TN_CUDA_TRY(launch_realify(h->dmat, 2LL * h->chi * h->chi, h->drt, 4 * a.n_edges, h->chi,
                             h->stream));
  h->stats.kernel_launches++;
  st = run_plan(h, h->rebuild[li], P_REBUILD);
  if (st) return st;
  h->ta_valid = false;
  for (auto& c : h->copyback[li]) {
    const int pi = prof_begin(h, P_COPY);
    TN_CUDA_TRY(launch_copy_blocks(c.d_dst, c.d_src, (int)c.dst.size(), c.n_floats, h->stream));
    prof_end(h, pi, 0.0, 8.0 * c.n_floats * c.dst.size());
    h->stats.kernel_launches++;
  }
  // discarded weights of this layer
  const int ne = a.n_edges;
  TN_CUDA_TRY(cudaMemcpyAsync(h->h_stats, h->solve_stats, sizeof(double) * 4 * ne,
                              cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < ne; ++i) {
    const double dw = h->h_stats[4 * i];
    h->stats.solve_edges++;
    h->stats.solve_sweeps += (int64_t)h->h_stats[4 * i + 3];
    h->stats.solve_sweeps_max = std::max(h->stats.solve_sweeps_max, (int64_t)h->h_stats[4 * i + 3]);
    h->stats.discarded_sum += dw;
    h->stats.discarded_max = std::max(h->stats.discarded_max, dw);
  }
  return check_flags(h, "the truncation solve");
}

// Enqueue one sweep: contract, normalise (the residual of every component
// and the flags accumulate on the device), then the stop-rule kernel.  Inside
// the device loop (`in_loop`) the stop kernel sets the while-loop condition;
// otherwise its output words are copied to pinned host memory.
tn_status enqueue_sweep(tn_handle* h, bool fork, bool in_loop, cudaGraphConditionalHandle cond = 0) {
  const int nmsg = 2 * (int)h->g.eu.size();
  tn_status st;
  if (fork) {
    // degree-2 and degree-1 launches on the side stream, beside the degree-3 chains
    TN_CUDA_TRY(cudaEventRecord(h->ev_fork, h->stream));
    TN_CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    st = run_plan(h, h->sweep, P_BP, h->sweep_split, (size_t)-1, true);
    if (st) return st;
    TN_CUDA_TRY(cudaEventRecord(h->ev_join, h->side));
    st = run_plan(h, h->sweep, P_BP, 0, h->sweep_split, false);
    if (st) return st;
    TN_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  } else {
    st = run_plan(h, h->sweep, P_BP);
    if (st) return st;
  }
  const int pi = prof_begin(h, P_NORM);
  BpComp comp;
  comp.comp_of_msg = h->comp_of_msg;
  comp.state = h->comp_state;
  comp.res = h->comp_res;
  TN_CUDA_TRY(launch_normalise(h->raw, h->msg, nmsg, h->chi, h->res_bits, h->flags, h->stream,
                               h->mrt, &comp));
  prof_end(h, pi, 0.0, 3.0 * 8.0 * h->chi * h->chi * nmsg);
  TN_CUDA_TRY(launch_bp_stop(h->n_comp, h->comp_state, h->comp_res, h->res_bits, h->loop_par,
                             h->loop_out, cond, in_loop ? 1 : 0, h->stream));
  h->stats.kernel_launches += 2;
  if (!in_loop)
    TN_CUDA_TRY(cudaMemcpyAsync(h->h_status, h->loop_out, 5 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, h->stream));
  return TN_OK;
}

// Build (once, on a non-default stream) the device-side BP loop: a graph
// holding one while-loop node whose body is the captured sweep.  The loop
// condition starts at 1 and the stop-rule kernel at the end of each sweep
// sets it; every component stops at max_iters at the latest, so the loop
// ends after at most max_iters sweeps.
tn_status loop_graph(tn_handle* h, bool* use) {
  *use = false;
  if (!h->loop_exec) {
    if (!h->stream || h->loop_unavailable) return TN_OK;  // the legacy default stream cannot be captured
    const bool prof = h->prof_on;
    h->prof_on = false;
    bool fork = h->sweep_split > 0 && h->sweep_split < h->sweep.L.size() &&
                side_safe(h, h->sweep, h->sweep_split);
    if (fork && !h->side) {
      if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        fork = false;
      }
    }
    fork = fork && h->side && h->ev_fork && h->ev_join;
    cudaGraph_t graph = nullptr;
    TN_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNode_t node = nullptr;
    cudaGraphNodeParams cp = {};
    cudaError_t ce = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (ce != cudaSuccess) {
      // a driver without conditional nodes: the host drives the loop
      cudaGetLastError();
      cudaGraphDestroy(graph);
      h->loop_unavailable = true;
      h->prof_on = prof;
      return TN_OK;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ce = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      h->prof_on = prof;
      TN_CUDA_TRY(ce);
    }
    const int64_t launches = h->stats.kernel_launches, tma = h->stats.tma_launches;
    tn_status st = enqueue_sweep(h, fork, true, cond);
    // the captured sweep's launch counts, charged once per sweep
    h->sweep_kernels = h->stats.kernel_launches - launches;
    h->sweep_tma = h->stats.tma_launches - tma;
    h->stats.kernel_launches = launches;
    h->stats.tma_launches = tma;
    h->prof_on = prof;
    cudaGraph_t captured = nullptr;
    ce = cudaStreamEndCapture(h->stream, &captured);
    if (st || ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      if (st) return st;
      TN_CUDA_TRY(ce);
    }
    ce = cudaGraphInstantiate(&h->loop_exec, graph, 0);
    cudaGraphDestroy(graph);
    TN_CUDA_TRY(ce);
  }
  *use = true;
  return TN_OK;
}

void sweep_work(tn_handle* h) {
  if (h->sweep_flops > 0.0 || h->sweep_bytes > 0.0) return;
  for (auto& L : h->sweep.L) {
    double f, b;
    gemm_work(L.d, &f, &b);
    h->sweep_flops += f;
    h->sweep_bytes += b;
    // a fused pair neither writes nor reads back its intermediate
    if (L.sp.maps && L.sp.kind == 2) h->sweep_bytes -= 16.0 * L.d.M * L.d.N * L.d.n_outer;
  }
}

// ---------------------------------------------------------------- autotuner
// The split-K count of each sweep launch that has one: the TMA closes (kind 1),
// the tensor-core tile GEMM and the CUDA-core GEMM.  Key of a launch: its
// kind, M, N, K, entries (outer x inner) and precision.
enum TuneKind { TUNE_NONE = 0, TUNE_CLOSE = 1, TUNE_TILE = 2, TUNE_SIMT = 3 };
const char* kTuneNames[] = {"none", "close", "tile", "simt"};

int tune_kind(const tn_handle* h, const HostLaunch& L) {
  if (L.skip) return TUNE_NONE;
  if (L.sp.maps) return L.sp.kind == 1 ? TUNE_CLOSE : TUNE_NONE;
  const double macs = (double)L.d.n_outer * L.d.n_inner * L.d.M * L.d.N * L.d.K1 * L.d.K2;
  return (use_tensor_cores(h) && !(macs < 262144.0)) ? TUNE_TILE : TUNE_SIMT;
}

// The split count a launch runs with now, and whether `s` is a valid count
// for it (its partials fit the handle's buffer, every split holds K work).
int current_splits(const tn_handle* h, const HostLaunch& L, int kind) {
  size_t pf = 0;
  if (kind == TUNE_CLOSE) return L.sp.splits;
  if (kind == TUNE_TILE) {
    int q, sp;
    tc_plan(L.d, &q, &sp, &pf, L.tuned);
    return sp;
  }
  return cgemm_plan(L.d, &pf, L.tuned);
}

bool splits_valid(const tn_handle* h, const HostLaunch& L, int kind, int s) {
  const size_t entries = (size_t)L.d.n_outer * L.d.n_inner;
  const size_t pf = s > 1 ? (size_t)s * entries * 2 * L.d.M * L.d.N : 0;
  if (pf > h->part_floats) return false;
  if (kind == TUNE_CLOSE) {
    const int chunks = L.d.K1 * L.d.K2 / 32;
    const int per = (chunks + s - 1) / s;
    return s >= 1 && s <= 64 && (chunks + per - 1) / per == s;  // no empty split
  }
  if (kind == TUNE_TILE) {
    int q, sp;
    size_t p2;
    tc_plan(L.d, &q, &sp, &p2, s);
    return sp == s;
  }
  size_t p2;
  return cgemm_plan(L.d, &p2, s) == s;
}

void set_splits(HostLaunch& L, int kind, int s) {
  if (kind == TUNE_CLOSE) L.sp.splits = s;
  else L.tuned = s;
}

std::string tune_key(const HostLaunch& L, int kind) {
  char buf[160];
  snprintf(buf, sizeof(buf), "%s %d %d %lld %d %d %d", kTuneNames[kind], L.d.M, L.d.N,
           (long long)L.d.K1 * L.d.K2, L.d.n_outer, L.d.n_inner, L.d.prec);
  return buf;
}

tn_status launch_one(tn_handle* h, const HostLaunch& L, int kind) {
  int nk = 0;
  if (kind == TUNE_CLOSE) {
    TN_CUDA_TRY(launch_tc_close(L.d, L.sp, h->part, h->flags, h->stream));
  } else if (kind == TUNE_TILE) {
    TN_CUDA_TRY(launch_cgemm_tc(L.d, h->part, h->flags, h->stream, &nk, L.tuned, h->part_floats));
  } else {
    TN_CUDA_TRY(launch_cgemm(L.d, h->stream, h->part, h->part_floats, &nk, L.tuned));
  }
  return TN_OK;
}

tn_status bp_converge_impl(tn_handle* h, double tol, int max_iters, int* iters, double* res) {
  // Messages are stored in FP32: once the residual is down at the rounding
  // floor of the arithmetic it stops decreasing and only fluctuates.  Below
  // `floor`, a sweep whose residual is not below 0.98 of the previous one
  // (the floor's signature; slow but steady convergence keeps going), or a
  // residual under floor / 8, ends the iteration as converged: the FP64
  // tolerance cannot be met by FP32 messages.  The rule acts on every
  // connected component separately (bp_stop_kernel), and a component that has
  // stopped keeps its messages, so an instance of a disjoint union receives
  // exactly the sweeps it would receive alone.
  const double floor = precision_floor(h);
  {
    tn_status st0 = ensure_ta(h);
    if (st0) return st0;
    st0 = ensure_mrt(h);
    if (st0) return st0;
  }
  sweep_work(h);
  bool use_loop = false;
  {
    tn_status st0 = loop_graph(h, &use_loop);
    if (st0) return st0;
  }
  if (max_iters < 1) max_iters = 1;
  TN_CUDA_TRY(launch_bp_loop_init(h->n_comp, h->comp_state, h->comp_res, h->res_bits, h->loop_par,
                                  tol, max_iters, floor, h->loop_out, h->stream));
  h->stats.kernel_launches++;
  int64_t sweeps = 0;
  if (use_loop) {
    const int pi = prof_begin(h, P_BP);
    TN_CUDA_TRY(cudaGraphLaunch(h->loop_exec, h->stream));
    prof_end(h, pi, 0.0, 0.0);
    TN_CUDA_TRY(cudaMemcpyAsync(h->h_status, h->loop_out, 5 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    sweeps = (int64_t)h->h_status[0];
    if (pi >= 0) {
      h->prof_pending[pi].flops = h->sweep_flops * sweeps;
      h->prof_pending[pi].bytes = h->sweep_bytes * sweeps;
    }
    h->stats.kernel_launches += h->sweep_kernels * sweeps;
    h->stats.tma_launches += h->sweep_tma * sweeps;
  } else {
    for (int it = 1; it <= max_iters; ++it) {
      tn_status st = enqueue_sweep(h, false, false);
      if (st) return st;
      TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
      if (h->h_status[4] == 0) break;
    }
    sweeps = (int64_t)h->h_status[0];
  }
  const int flags = (int)h->h_status[3];
  double r;
  const unsigned long long bits = h->h_status[1];
  memcpy(&r, &bits, sizeof(r));
  if (flags) {
    TN_CUDA_TRY(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
    set_error(flags & 2 ? "a device-side wait gave up in a BP sweep"
                        : "non-finite or zero-norm values detected in a BP sweep");
    return flags & 2 ? TN_ETIMEOUT : TN_ENUMERIC;
  }
  const int it = (int)sweeps;
  h->stats.bp_iters_last = it;
  h->stats.bp_iters_total += it;
  h->stats.bp_residual_last = r;
  if (iters) *iters = it;
  if (res) *res = r;
  if (h->h_status[2] > 0) {
    set_error("BP did not reach the tolerance within max_iters");
    return TN_ENOTCONVERGED;
  }
  return TN_OK;
}

tn_status compute_rho(tn_handle* h, std::vector<double>* rho_out) {
  tn_status st = run_plan(h, h->rho_prep, P_RHO);
  if (st) return st;
  const int n = h->g.n;
  int base = 0;
  std::vector<int> order;
  for (auto& r : h->rho_l) {
    const int64_t len = ipow(h->chi, r.deg);
    const int pi = prof_begin(h, P_RHO);
    TN_CUDA_TRY(launch_rho(h->Y1, h->T, r.d_x, r.d_t, (int)r.sites.size(), len, 2 * len,
                           h->rho + 8 * base, h->rho_part, h->stream));
    prof_end(h, pi, 32.0 * len * r.sites.size(), 2.0 * 16.0 * len * r.sites.size());
    h->stats.kernel_launches += 2;
    for (int v : r.sites) order.push_back(v);
    base += (int)r.sites.size();
  }
  std::vector<double> tmp(8 * n);
  TN_CUDA_TRY(cudaMemcpyAsync(tmp.data(), h->rho, sizeof(double) * 8 * n,
                              cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  rho_out->assign(8 * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 8; ++c) (*rho_out)[8 * order[i] + c] = tmp[8 * i + c];
  return TN_OK;
}

double pauli_from_rho(const double* r, char p) {
  // r: [(00) re im, (01) re im, (10) re im, (11) re im]; <P> = Tr(rho P)/Tr(rho)
  const double tr = r[0] + r[6];
  switch (p) {
    case 'X': return (r[2] + r[4]) / tr;
    case 'Y': return (-r[3] + r[5]) / tr;  // Tr(rho Y) = i rho01 - i rho10 (real part)
    case 'Z': return (r[0] - r[6]) / tr;
    default: return NAN;
  }
}

tn_status init_state(tn_handle* h) {
  TN_CUDA_TRY(cudaMemsetAsync(h->T, 0, sizeof(float) * h->t_floats, h->stream));
  const int64_t c2 = (int64_t)h->chi * h->chi;
  const int nmsg = 2 * (int)h->g.eu.size();
  TN_CUDA_TRY(cudaMemsetAsync(h->msg, 0, sizeof(float) * nmsg * 2 * c2, h->stream));
  const float one = 1.f;
  for (int v = 0; v < h->g.n; ++v)
    TN_CUDA_TRY(cudaMemcpyAsync(h->T + h->t_off[v], &one, sizeof(float), cudaMemcpyHostToDevice,
                                h->stream));
  for (int m = 0; m < nmsg; ++m)
    TN_CUDA_TRY(cudaMemcpyAsync(h->msg + (int64_t)m * 2 * c2, &one, sizeof(float),
                                cudaMemcpyHostToDevice, h->stream));
  {
    // bond spectra of the product state: (1, 0, .., 0) on every edge
    std::vector<double> sp(h->g.eu.size() * (size_t)h->chi, 0.0);
    for (size_t e = 0; e < h->g.eu.size(); ++e) sp[e * h->chi] = 1.0;
    if (!sp.empty())
      TN_CUDA_TRY(cudaMemcpyAsync(h->spectra, sp.data(), sizeof(double) * sp.size(),
                                  cudaMemcpyHostToDevice, h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  h->ta_valid = false;
  h->mrt_valid = false;
  return TN_OK;
}

size_t footprint_of(const HostGraph& g, int chi) {
  int64_t tf = 0;
  for (int v = 0; v < g.n; ++v) tf += 4 * ipow(chi, g.degree(v));
  const int64_t c2 = (int64_t)chi * chi;
  size_t maxl = 0;
  for (auto& l : g.layers) maxl = std::max(maxl, l.size());
  size_t b = 0;
  b += 5 * sizeof(float) * (size_t)tf;                      // T, Ts, TA, Y1, Y2
  b += sizeof(float) * (size_t)(2 * g.eu.size()) * 4 * c2;  // realified messages
  b += sizeof(float) * maxl * 16 * c2;                     // realified leg matrices
  b += 2 * sizeof(float) * (size_t)(2 * g.eu.size()) * 2 * c2;  // msg, raw
  b += 2 * sizeof(float) * maxl * 8 * c2;                  // gram, dmat
  b += sizeof(double) * maxl * solve_work_doubles(chi);    // work
  b += sizeof(double) * g.eu.size() * (size_t)chi;        // bond spectra
  return b;
}

}  // namespace
}  // namespace tnbp

using namespace tnbp;

extern "C" {

const char* tn_last_error(void) { return g_err.c_str(); }
const char* tn_version(void) { return "tnbp 0.1 (sm_103a)"; }

tn_status tn_heavy_hex(int32_t rows, int32_t cols, int32_t* n_vertices, int32_t* n_edges,
                       int32_t* edges_out, uint8_t* colours_out, int32_t capacity) {
  HostGraph g;
  std::string why;
  if (!heavy_hex(rows, cols, &g, &why)) {
    set_error(why);
    return TN_EINVAL;
  }
  const int m = (int)g.eu.size();
  if (n_vertices) *n_vertices = g.n;
  if (n_edges) *n_edges = m;
  if (edges_out || colours_out) {
    if (capacity < m) {
      set_error("capacity smaller than the number of edges");
      return TN_EINVAL;
    }
    for (int e = 0; e < m; ++e) {
      if (edges_out) { edges_out[2 * e] = g.eu[e]; edges_out[2 * e + 1] = g.ew[e]; }
      if (colours_out) colours_out[e] = (uint8_t)g.colour[e];
    }
  }
  return TN_OK;
}

tn_status tn_footprint_estimate(const tn_graph* graph, const tn_config* cfg, size_t* out) {
  if (!graph || !cfg || !out) { set_error("null argument"); return TN_EINVAL; }
  HostGraph g;
  std::string why;
  if (!build_graph(graph->n_vertices, graph->n_edges, graph->edges, graph->colour, &g, &why)) {
    set_error(why);
    return TN_EINVAL;
  }
  *out = footprint_of(g, cfg->chi);
  return TN_OK;
}

tn_status tn_create(const tn_graph* graph, const tn_config* cfg, const tn_allocator* alloc,
                    void* cuda_stream, tn_handle** out) {
  if (!graph || !cfg || !out) { set_error("null argument"); return TN_EINVAL; }
  *out = nullptr;
  if (cfg->chi < 1 || cfg->chi > 256) { set_error("chi must be in 1..256"); return TN_EINVAL; }
  if (cfg->prec < TN_FP32 || cfg->prec > TN_TF32X3) { set_error("unknown precision"); return TN_EINVAL; }

  if (cfg->solve != TN_SOLVE_AUTO && cfg->solve != TN_SOLVE_SHARED && cfg->solve != TN_SOLVE_FP64 &&
      cfg->solve != TN_SOLVE_REFINED) {
    set_error("unknown truncation solve");
    return TN_EINVAL;
  }
  if (!(cfg->solve_tol < 0.1)) {
    set_error("solve_tol must be below 0.1");
    return TN_EINVAL;
  }
  if (cfg->kernels != TN_KERNELS_AUTO && cfg->kernels != TN_KERNELS_TILE) {
    set_error("unknown kernel selection");
    return TN_EINVAL;
  }
  if (!(cfg->bp_tol > 0) || cfg->bp_max_iters < 1) {
    set_error("bp_tol must be > 0 and bp_max_iters >= 1");
    return TN_EINVAL;
  }
  if (alloc && (!alloc->alloc || !alloc->free)) { set_error("allocator callbacks missing"); return TN_EINVAL; }
  tn_handle* h = new tn_handle();
  std::string why;
  if (!build_graph(graph->n_vertices, graph->n_edges, graph->edges, graph->colour, &h->g, &why)) {
    set_error(why);
    delete h;
    return TN_EINVAL;
  }
  {
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaGetDeviceProperties(&prop, dev);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
      delete h;
      return TN_ECUDA;
    }
    if (prop.major * 10 + prop.minor != 103) {
      set_error("device is sm_" + std::to_string(prop.major * 10 + prop.minor) +
                "; this library is built for sm_103a");
      delete h;
      return TN_ECUDA;
    }
  }
  h->cfg = *cfg;
  h->chi = cfg->chi;
  h->stream = (cudaStream_t)cuda_stream;
  if (alloc) { h->alloc = *alloc; h->own_alloc = false; }
  const HostGraph& g = h->g;
  const int chi = h->chi;
  const int64_t c2 = (int64_t)chi * chi;
  h->t_off.resize(g.n);
  h->t_len.resize(g.n);
  int64_t off = 0;
  for (int v = 0; v < g.n; ++v) {
    h->t_off[v] = off;
    h->t_len[v] = ipow(chi, g.degree(v));
    off += 4 * h->t_len[v];
    h->sites_by_deg[g.degree(v)].push_back(v);
  }
  h->t_floats = off;
  const int nmsg = 2 * (int)g.eu.size();
  for (auto& l : g.layers) h->max_layer = std::max(h->max_layer, (int)l.size());
  auto fail = [&](tn_status s) { dev_free_all(h); delete h; return s; };
  h->T = (float*)dev_alloc(h, sizeof(float) * off);
  h->Ts = (float*)dev_alloc(h, sizeof(float) * off);
  h->Y1 = (float*)dev_alloc(h, sizeof(float) * off);
  h->Y2 = (float*)dev_alloc(h, sizeof(float) * off);
  h->TA = (float*)dev_alloc(h, sizeof(float) * off);
  h->mrt = (float*)dev_alloc(h, sizeof(float) * nmsg * 4 * c2);
  h->msg = (float*)dev_alloc(h, sizeof(float) * nmsg * 2 * c2);
  h->raw = (float*)dev_alloc(h, sizeof(float) * nmsg * 2 * c2);
  h->gram = (float*)dev_alloc(h, sizeof(float) * h->max_layer * 8 * c2);
  h->dmat = (float*)dev_alloc(h, sizeof(float) * h->max_layer * 8 * c2);
  h->drt = (float*)dev_alloc(h, sizeof(float) * h->max_layer * 16 * c2);
  h->work = (double*)dev_alloc(h, sizeof(double) * h->max_layer * solve_work_doubles(chi));
  h->solve_stats = (double*)dev_alloc(h, sizeof(double) * 4 * h->max_layer);
  h->spectra = (double*)dev_alloc(h, sizeof(double) * std::max<size_t>(1, g.eu.size()) * chi);
  {
    h->spec_row.assign(g.eu.size(), 0);
    int64_t row = 0;
    for (const auto& layer : g.layers) {
      h->spec_off.push_back(row);
      for (int e : layer) h->spec_row[e] = (int)row++;
    }
  }
  h->res_bits = (unsigned long long*)dev_alloc(h, 64);
  h->flags = h->res_bits ? reinterpret_cast<int*>(h->res_bits + 1) : nullptr;
  {
    // connected components by union-find over the edges
    std::vector<int> root(g.n);
    for (int v = 0; v < g.n; ++v) root[v] = v;
    auto find = [&](int v) {
      while (root[v] != v) v = root[v] = root[root[v]];
      return v;
    };
    for (size_t e = 0; e < g.eu.size(); ++e) {
      const int a = find(g.eu[e]), b = find(g.ew[e]);
      if (a != b) root[std::max(a, b)] = std::min(a, b);
    }
    h->comp_of_vertex.assign(g.n, -1);
    std::vector<int> id(g.n, -1);
    h->n_comp = 0;
    for (int v = 0; v < g.n; ++v) {
      const int r = find(v);
      if (id[r] < 0) id[r] = h->n_comp++;
      h->comp_of_vertex[v] = id[r];
    }
  }
  h->comp_of_msg = (int*)dev_alloc(h, sizeof(int) * std::max<size_t>(1, 2 * g.eu.size()));
  h->comp_state = (double*)dev_alloc(h, sizeof(double) * 4 * std::max(1, h->n_comp));
  h->comp_res = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * std::max(1, h->n_comp));
  h->loop_par = (double*)dev_alloc(h, sizeof(double) * 4);
  h->loop_out = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * 8);
  h->rho = (double*)dev_alloc(h, sizeof(double) * 8 * g.n);
  h->rho_part = (double*)dev_alloc(h, sizeof(double) * 16 * 8 * std::max(1, g.n));
  for (int d = 1, base = 0; d <= 3; ++d) {
    h->n_by_deg[d] = (int)h->sites_by_deg[d].size();
    h->site_offs_by_deg[d] = (int64_t*)dev_alloc(h, sizeof(int64_t) * (h->n_by_deg[d] + 1));
    h->rx_base[d] = base;
    base += h->n_by_deg[d];
  }
  h->rx_cs = (float2*)dev_alloc(h, sizeof(float2) * std::max(1, g.n));
  const int nl = (int)g.layers.size();
  h->d_layer_msg_vw.resize(nl);
  h->layer_msg_vw.resize(nl);
  for (int li = 0; li < nl; ++li) {
    h->d_layer_msg_vw[li] = (int32_t*)dev_alloc(h, sizeof(int32_t) * 2 * g.layers[li].size());
    if (!h->d_layer_msg_vw[li]) {
      set_error("device allocation of layer tables failed");
      return fail(TN_ENOMEM);
    }
  }
  if (!h->T || !h->Ts || !h->Y1 || !h->Y2 || !h->TA || !h->mrt || !h->drt || !h->msg ||
      !h->raw || !h->gram || !h->dmat ||
      !h->work || !h->solve_stats || !h->res_bits || !h->flags || !h->rho || !h->rho_part ||
      !h->comp_of_msg || !h->comp_state || !h->comp_res || !h->loop_par || !h->loop_out ||
      !h->rx_cs ||
      !h->spectra) {
    set_error("device allocation failed (footprint " + std::to_string(footprint_of(g, chi)) +
              " bytes)");
    return fail(TN_ENOMEM);
  }
  for (int d = 1; d <= 3; ++d) {
    std::vector<int64_t> offs;
    for (int v : h->sites_by_deg[d]) offs.push_back(h->t_off[v]);
    if (!offs.empty() &&
        cudaMemcpy(h->site_offs_by_deg[d], offs.data(), sizeof(int64_t) * offs.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("upload of site offsets failed");
      return fail(TN_ECUDA);
    }
  }
  for (int li = 0; li < nl; ++li) {
    auto& v = h->layer_msg_vw[li];
    for (int e : g.layers[li]) {
      v.push_back(dir_id(g, g.eu[e], e));
      v.push_back(dir_id(g, g.ew[e], e));
    }
    if (cudaMemcpy(h->d_layer_msg_vw[li], v.data(), sizeof(int32_t) * v.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("upload of layer tables failed");
      return fail(TN_ECUDA);
    }
  }
  {
    std::vector<int> cm(2 * g.eu.size());
    for (size_t e = 0; e < g.eu.size(); ++e) cm[2 * e] = cm[2 * e + 1] = h->comp_of_vertex[g.eu[e]];
    if (!cm.empty() && cudaMemcpy(h->comp_of_msg, cm.data(), sizeof(int) * cm.size(),
                                  cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("upload of the component table failed");
      return fail(TN_ECUDA);
    }
  }
  cudaMemset(h->res_bits, 0, 64);
  cudaMemset(h->comp_state, 0, sizeof(double) * 4 * std::max(1, h->n_comp));
  if (cudaMallocHost(&h->h_status, 8 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned host allocation failed");
    delete[] h->h_stats;
    return fail(TN_ENOMEM);
  }
  h->h_stats = new double[4 * std::max(1, h->max_layer)];
  if ((use_tensor_cores(h) && tc_prepare() != cudaSuccess) || normalise_prepare(chi) != cudaSuccess) {
    cudaGetLastError();
    set_error("setting kernel attributes failed");
    delete[] h->h_stats;
    return fail(TN_ECUDA);
  }
  build_sweep_plan(h);
  h->gate_env.resize(nl);
  h->rebuild.resize(nl);
  h->copyback.resize(nl);
  for (int li = 0; li < nl; ++li) build_gate_plans(h, li);
  build_rho_plan(h);
  {
    size_t need = 0;
    std::vector<Plan*> plans = {&h->sweep, &h->rho_prep};
    for (auto& p : h->gate_env) plans.push_back(&p);
    for (auto& p : h->rebuild) plans.push_back(&p);
    for (Plan* p : plans)
      for (auto& L : p->L) {
        size_t pf = 0;
        if (use_tensor_cores(h)) {
          int q, sp;
          tc_plan(L.d, &q, &sp, &pf);
          need = std::max(need, pf);
        }
        cgemm_plan(L.d, &pf);  // the CUDA-core launches of every precision
        need = std::max(need, pf);
      }
    // the TMA closes take at most 2 x 152 CTAs of partials over the entries
    if (use_tensor_cores(h)) need = std::max<size_t>(need, (size_t)2 * 2 * 152 * 2 * 4096);
    h->part_floats = std::max<size_t>(need, 16);
    h->part = (float*)dev_alloc(h, sizeof(float) * h->part_floats);
    if (!h->part) { delete[] h->h_stats; set_error("device allocation failed"); return fail(TN_ENOMEM); }
  }
  tn_status st = upload_plans(h);
  if (st) { delete[] h->h_stats; return fail(st); }
  st = attach_components(h);
  if (st) { delete[] h->h_stats; return fail(st); }
  st = init_state(h);
  if (st) { delete[] h->h_stats; return fail(st); }
  *out = h;
  return TN_OK;
}

tn_status tn_destroy(tn_handle* h) {
  if (!h) return TN_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->h_status) cudaFreeHost(h->h_status);
  dev_free_all(h);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  delete[] h->h_stats;
  delete h;
  return TN_OK;
}

tn_status tn_profile_enable(tn_handle* h, int32_t on) {
  if (!h) { set_error("null handle"); return TN_EINVAL; }
  tn_status st = prof_flush(h);
  if (st) return st;
  h->prof = tn_profile{};
  h->prof.n_classes = P_NCLS;
  h->prof_on = on != 0;
  return TN_OK;
}

tn_status tn_profile_read(tn_handle* h, tn_profile* out) {
  if (!h || !out) { set_error("null argument"); return TN_EINVAL; }
  tn_status st = prof_flush(h);
  if (st) return st;
  h->prof.n_classes = P_NCLS;
  *out = h->prof;
  return TN_OK;
}

const char* tn_profile_class_name(int32_t cls) {
  if (cls < 0 || cls >= P_NCLS) return "";
  return kProfNames[cls];
}

static tn_status evolve(tn_handle* h, double theta, int steps, bool clifford_dagger,
                        const double* theta_v = nullptr) {
  if (!h) { set_error("null handle"); return TN_EINVAL; }
  if (steps < 0) { set_error("steps must be >= 0"); return TN_EINVAL; }
  h->stats = tn_stats{};
  tn_status worst = TN_OK;
  double u[8];
  rx_matrix(clifford_dagger ? -M_PI / 2 : theta, u);
  if (theta_v) {
    tn_status st = upload_rx_field(h, theta_v);
    if (st) return st;
  }
  for (int s = 0; s < steps; ++s) {
    tn_status st;
    if (!clifford_dagger) {
      st = theta_v ? phys_gate_field(h) : phys_gate(h, u);
      if (st) return st;
    }
    for (int li = 0; li < (int)h->g.layers.size(); ++li) {
      st = gate_layer(h, li, clifford_dagger ? -1 : +1);
      if (st) return st;
    }
    if (clifford_dagger) {
      st = phys_gate(h, u);
      if (st) return st;
    }
    st = bp_converge_impl(h, h->cfg.bp_tol, h->cfg.bp_max_iters, nullptr, nullptr);
    if (st == TN_ENOTCONVERGED) worst = st;
    else if (st) return st;
    h->stats.steps_done = s + 1;
  }
  if (worst) set_error("a BP regauge hit bp_max_iters");
  return worst;
}

tn_status tn_apply_floquet(tn_handle* h, double theta_h, int32_t steps) {
  return evolve(h, theta_h, steps, false);
}

tn_status tn_apply_floquet_field(tn_handle* h, const double* theta_v, int32_t steps) {
  if (!h) { set_error("null handle"); return TN_EINVAL; }
  if (!theta_v) { set_error("theta_v is null"); return TN_EINVAL; }
  for (int v = 0; v < h->g.n; ++v)
    if (!std::isfinite(theta_v[v])) { set_error("theta_v holds a non-finite angle"); return TN_EINVAL; }
  return evolve(h, 0.0, steps, false, theta_v);
}

tn_status tn_apply_clifford_dagger(tn_handle* h, int32_t steps) {
  return evolve(h, 0.0, steps, true);
}

tn_status tn_bp_converge(tn_handle* h, double tol, int32_t max_iters, int32_t* iters_out,
                         double* residual_out) {
  if (!h) { set_error("null handle"); return TN_EINVAL; }
  if (!(tol > 0) || max_iters < 1) { set_error("tol must be > 0, max_iters >= 1"); return TN_EINVAL; }
  h->stats = tn_stats{};
  int it = 0;
  double r = 0;
  tn_status st = bp_converge_impl(h, tol, max_iters, &it, &r);
  if (iters_out) *iters_out = it;
  if (residual_out) *residual_out = r;
  return st;
}

tn_status tn_autotune(tn_handle* h, int32_t reps, char* table_out, size_t table_cap,
                      size_t* table_len) {
  if (!h || reps < 1) { set_error("null handle or reps < 1"); return TN_EINVAL; }
  tn_status st = ensure_ta(h);
  if (st) return st;
  st = ensure_mrt(h);
  if (st) return st;
  // the launches skip components the last BP iteration marked stopped: clear
  // the marks while timing, and put the state back afterwards
  std::vector<double> comp_saved(4 * (size_t)std::max(1, h->n_comp));
  TN_CUDA_TRY(cudaMemcpyAsync(comp_saved.data(), h->comp_state, sizeof(double) * comp_saved.size(),
                              cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(launch_bp_loop_init(h->n_comp, h->comp_state, h->comp_res, h->res_bits, h->loop_par,
                                  1e-10, 1, 1.0, h->loop_out, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  const bool prof = h->prof_on;
  h->prof_on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    h->prof_on = prof;
    set_error("cudaEventCreate failed");
    return TN_ECUDA;
  }
  std::string table;
  // the sweep's launches read the state and write only the sweep's scratch and
  // raw messages, which the next sweep recomputes from the state
  for (size_t li = 0; li < h->sweep.L.size(); ++li) {
    HostLaunch& L = h->sweep.L[li];
    const int kind = tune_kind(h, L);
    // the launches the captured sweep may run on its side stream keep one
    // split (partials live in the one buffer of the main stream)
    if (kind == TUNE_NONE || (h->sweep_split > 0 && li >= h->sweep_split)) continue;
    const int now = current_splits(h, L, kind);
    // every valid power-of-two count, timed over `reps` launches after one
    // warm-up launch; the fastest replaces the current count only when it is
    // at least 3% faster (timing noise keeps the heuristic's choice)
    int best = now, fastest = 0;
    float now_ms = -1.f, fastest_ms = 0.f;
    for (int sc = 1; sc <= 64 && !st; sc *= 2) {
      if (!splits_valid(h, L, kind, sc)) continue;
      set_splits(L, kind, sc);
      st = launch_one(h, L, kind);
      if (!st && cudaEventRecord(e0, h->stream) != cudaSuccess) st = TN_ECUDA;
      for (int r = 0; r < reps && !st; ++r) st = launch_one(h, L, kind);
      if (!st && cudaEventRecord(e1, h->stream) != cudaSuccess) st = TN_ECUDA;
      if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = TN_ECUDA;
      float ms = 0.f;
      if (!st && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = TN_ECUDA;
      if (st) break;
      if (sc == now) now_ms = ms;
      if (fastest == 0 || ms < fastest_ms) { fastest = sc; fastest_ms = ms; }
    }
    if (st) { set_splits(L, kind, now); break; }
    float best_ms = now_ms;
    if (fastest > 0 && (now_ms < 0.f || fastest_ms < 0.97f * now_ms)) {
      best = fastest;
      best_ms = fastest_ms;
    }
    set_splits(L, kind, best);
    char line[64];
    snprintf(line, sizeof(line), " %d %.3f\n", best, 1e3 * best_ms / reps);
    table += tune_key(L, kind) + line;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->prof_on = prof;
  cudaGetLastError();
  TN_CUDA_TRY(cudaMemcpyAsync(h->comp_state, comp_saved.data(), sizeof(double) * comp_saved.size(),
                              cudaMemcpyHostToDevice, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (st) return st;
  // the loop graph is captured again with the new counts
  if (h->loop_exec) { cudaGraphExecDestroy(h->loop_exec); h->loop_exec = nullptr; }
  if (table_len) *table_len = table.size();
  if (table_out && table_cap > 0) {
    const size_t n = std::min(table.size(), table_cap - 1);
    memcpy(table_out, table.data(), n);
    table_out[n] = 0;
  }
  return TN_OK;
}

tn_status tn_autotune_apply(tn_handle* h, const char* table, int32_t* n_applied) {
  if (!h || !table) { set_error("null argument"); return TN_EINVAL; }
  std::vector<std::pair<std::string, int>> rows;
  const char* p = table;
  while (*p) {
    const char* q = strchr(p, '\n');
    std::string line = q ? std::string(p, q) : std::string(p);
    p = q ? q + 1 : p + line.size();
    char kind[16];
    int m, n, outer, inner, prec, splits;
    long long k;
    double us;
    if (sscanf(line.c_str(), "%15s %d %d %lld %d %d %d %d %lf", kind, &m, &n, &k, &outer, &inner,
               &prec, &splits, &us) < 8)
      continue;
    char key[160];
    snprintf(key, sizeof(key), "%s %d %d %lld %d %d %d", kind, m, n, k, outer, inner, prec);
    rows.push_back({key, splits});
  }
  int applied = 0;
  for (size_t li = 0; li < h->sweep.L.size(); ++li) {
    HostLaunch& L = h->sweep.L[li];
    const int kind = tune_kind(h, L);
    if (kind == TUNE_NONE || (h->sweep_split > 0 && li >= h->sweep_split)) continue;
    const std::string key = tune_key(L, kind);
    for (auto& r : rows)
      if (r.first == key && splits_valid(h, L, kind, r.second)) {
        set_splits(L, kind, r.second);
        ++applied;
        break;
      }
  }
  if (h->loop_exec) { cudaGraphExecDestroy(h->loop_exec); h->loop_exec = nullptr; }
  if (n_applied) *n_applied = applied;
  return TN_OK;
}

tn_status tn_bp_components(tn_handle* h, int32_t* comp_of_vertex, int32_t* sweeps_out,
                           double* residual_out, int32_t cap, int32_t* n_comp_out) {
  if (!h || cap < 0) { set_error("null handle or cap < 0"); return TN_EINVAL; }
  if (n_comp_out) *n_comp_out = h->n_comp;
  if (comp_of_vertex)
    for (int v = 0; v < h->g.n; ++v) comp_of_vertex[v] = h->comp_of_vertex[v];
  const int m = std::min(cap, h->n_comp);
  if ((sweeps_out || residual_out) && m > 0) {
    std::vector<double> st(4 * (size_t)h->n_comp);
    TN_CUDA_TRY(cudaMemcpyAsync(st.data(), h->comp_state, sizeof(double) * st.size(),
                                cudaMemcpyDeviceToHost, h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < m; ++c) {
      if (sweeps_out) sweeps_out[c] = (int32_t)st[4 * c + 2];
      if (residual_out) residual_out[c] = st[4 * c + 1];
    }
  }
  return TN_OK;
}

tn_status tn_expect_z_all(tn_handle* h, double* out) {
  if (!h || !out) { set_error("null argument"); return TN_EINVAL; }
  std::vector<double> rho;
  tn_status st = compute_rho(h, &rho);
  if (st) return st;
  for (int v = 0; v < h->g.n; ++v) out[v] = pauli_from_rho(&rho[8 * v], 'Z');
  return TN_OK;
}

// ----------------------------------------------------------- checkpoints
// Host image of a job's state: a header, the site tensors, the messages and
// the bond spectra, all as the device holds them.
struct CkptHeader {
  uint64_t magic;        // "TNBPCKP1"
  uint64_t graph_hash;   // FNV-1a over n, the edge list and the colour layers
  int64_t n_vertices, n_edges, chi, t_floats, msg_floats, spec_doubles;
};
constexpr uint64_t kCkptMagic = 0x31504b4350424e54ull;

uint64_t graph_hash(const HostGraph& g) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  mix(g.n);
  for (size_t e = 0; e < g.eu.size(); ++e) { mix(g.eu[e]); mix(g.ew[e]); }
  for (const auto& layer : g.layers) {
    mix(-1);
    for (int e : layer) mix(e);
  }
  return h;
}

CkptHeader ckpt_header(const tn_handle* h) {
  CkptHeader c;
  c.magic = kCkptMagic;
  c.graph_hash = graph_hash(h->g);
  c.n_vertices = h->g.n;
  c.n_edges = (int64_t)h->g.eu.size();
  c.chi = h->chi;
  c.t_floats = h->t_floats;
  c.msg_floats = 2 * c.n_edges * 2 * (int64_t)h->chi * h->chi;
  c.spec_doubles = c.n_edges * h->chi;
  return c;
}

size_t ckpt_bytes(const CkptHeader& c) {
  return sizeof(CkptHeader) + sizeof(float) * (size_t)(c.t_floats + c.msg_floats) +
         sizeof(double) * (size_t)c.spec_doubles;
}

static tn_status backup_state(tn_handle* h, bool restore) {
  const int64_t c2 = (int64_t)h->chi * h->chi;
  const size_t mb = sizeof(float) * 2 * h->g.eu.size() * 2 * c2;
  if (!h->T_bak) {
    h->T_bak = (float*)dev_alloc(h, sizeof(float) * h->t_floats);
    h->msg_bak = (float*)dev_alloc(h, mb);
    if (!h->T_bak || !h->msg_bak) { set_error("no memory for the state copy"); return TN_ENOMEM; }
  }
  float* dst_t = restore ? h->T : h->T_bak;
  float* src_t = restore ? h->T_bak : h->T;
  float* dst_m = restore ? h->msg : h->msg_bak;
  float* src_m = restore ? h->msg_bak : h->msg;
  TN_CUDA_TRY(cudaMemcpyAsync(dst_t, src_t, sizeof(float) * h->t_floats, cudaMemcpyDeviceToDevice,
                              h->stream));
  TN_CUDA_TRY(cudaMemcpyAsync(dst_m, src_m, mb, cudaMemcpyDeviceToDevice, h->stream));
  if (restore) {
    h->ta_valid = false;
    h->mrt_valid = false;
  }
  return TN_OK;
}


// ------------------------------------------------------------ region strings
// A Pauli string of weight k > 1 by the BP-region reading of the expectation
// rule (Methods, "Measuring expectation values within the Vidal gauge"; the
// environment of a region is the product of the converged messages entering
// it): exact contraction of the norm network over a tree T_S spanning the
// string's support, every edge leaving the tree closed by its converged
// message, divided by the same contraction without the operators.
//
// Tree rule: breadth-first search from the smallest support site, neighbours
// in increasing edge id; T_S is the union of the search-tree paths from the
// other support sites back to it.  Contraction: sites in post-order from the
// root (the smallest vertex of T_S); each non-root site sends its parent the
// BP message update of its norm tensor with the operator inserted on the bra's
// physical index (bra = conj(P T) for Hermitian P), taking the children's
// messages on tree legs and the converged messages elsewhere; each such
// message is scaled to unit norm with its log norm kept in FP64; the root
// closes its last leg against the incoming message.
std::vector<int> steiner_edges(const HostGraph& g, std::vector<int> terms) {
  std::sort(terms.begin(), terms.end());
  std::vector<int> par(g.n, -2);
  std::vector<int> q{terms[0]};
  par[terms[0]] = -1;
  for (size_t h0 = 0; h0 < q.size(); ++h0) {
    const int v = q[h0];
    for (int e : g.legs[v]) {
      const int w = g.other(e, v);
      if (par[w] == -2) { par[w] = e; q.push_back(w); }
    }
  }
  std::vector<char> used(g.eu.size(), 0);
  for (size_t i = 1; i < terms.size(); ++i)
    for (int v = terms[i]; par[v] >= 0; v = g.other(par[v], v)) used[par[v]] = 1;
  std::vector<int> out;
  for (int e = 0; e < (int)used.size(); ++e)
    if (used[e]) out.push_back(e);
  return out;
}

// Run a plan built at call time; its pointer arrays go to `arena` first.
tn_status run_adhoc(tn_handle* h, Plan& P, void* arena) {
  std::vector<const void*> host;
  for (auto& L : P.L) {
    for (auto q : L.A) host.push_back(q);
    for (auto q : L.B) host.push_back(q);
    for (auto q : L.C) host.push_back(q);
  }
  TN_CUDA_TRY(cudaMemcpyAsync(arena, host.data(), host.size() * sizeof(void*),
                              cudaMemcpyHostToDevice, h->stream));
  const void** base = (const void**)arena;
  size_t pos = 0;
  for (auto& L : P.L) {
    L.d.A = (const float* const*)(base + pos); pos += L.A.size();
    L.d.B = (const float* const*)(base + pos); pos += L.B.size();
    L.d.C = (float* const*)(base + pos); pos += L.C.size();
  }
  return run_plan(h, P, P_RHO);
}

// <value> = (scalar, log scale) of the tree contraction with operator letters
// op[v] ('X', 'Y', 'Z', or 0 for the identity) on the tree's sites.
tn_status region_contract(tn_handle* h, const std::vector<int>& tree, const std::vector<char>& op,
                          double* re, double* im, double* logscale, bool* zero) {
  const HostGraph& g = h->g;
  const int x = h->chi;
  const int64_t c2 = (int64_t)x * x;
  std::vector<int> eidx(g.eu.size(), -1);
  for (size_t i = 0; i < tree.size(); ++i) eidx[tree[i]] = (int)i;
  int root = g.n;
  for (int e : tree) root = std::min(root, std::min(g.eu[e], g.ew[e]));
  // depth-first order from the root along tree edges; parent edge per site
  std::vector<int> order, parent(g.n, -2);
  {
    std::vector<int> stack{root};
    parent[root] = -1;
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      order.push_back(v);
      for (int e : g.legs[v]) {
        if (eidx[e] < 0) continue;
        const int w = g.other(e, v);
        if (parent[w] == -2) { parent[w] = e; stack.push_back(w); }
      }
    }
  }
  // operator sites: bra copies P T and their first-leg-last copies
  std::vector<int> opsites;
  std::vector<int64_t> op_off;
  int64_t bra_floats = 0;
  for (int v : order)
    if (op[v]) { opsites.push_back(v); op_off.push_back(bra_floats); bra_floats += 4 * h->t_len[v]; }
  const size_t n_te = tree.size();
  const size_t n_ptr = 9 * order.size() + 16;
  const size_t bytes = sizeof(float) * (n_te * 6 * c2 + 2 * c2 + 2 * bra_floats) +
                       sizeof(int64_t) * (op_off.size() + 1) + sizeof(void*) * n_ptr + 64;
  unsigned char* buf = (unsigned char*)dev_alloc(h, bytes);
  if (!buf) { set_error("device allocation for the region contraction failed"); return TN_ENOMEM; }
  float* up = (float*)buf;                        // [n_te][2 c2] messages child -> parent
  float* upr = up + n_te * 2 * c2;                // [n_te][4 c2] realified transposed
  float* root_out = upr + n_te * 4 * c2;          // [2 c2]
  float* bra = root_out + 2 * c2;                 // operator copies
  float* braA = bra + bra_floats;
  int64_t* d_off = (int64_t*)(braA + bra_floats);
  void* arena = (void*)(((uintptr_t)(d_off + op_off.size() + 1) + 15) & ~uintptr_t(15));
  double* scal = (double*)((unsigned char*)arena + sizeof(void*) * n_ptr);  // re, im, log
  int* zflag = (int*)(scal + 3);
  tn_status st = TN_OK;
  auto fail_free = [&](tn_status code) { cudaStreamSynchronize(h->stream); dev_free(h, buf); return code; };
  if (!op_off.empty())
    if (cudaMemcpyAsync(d_off, op_off.data(), sizeof(int64_t) * op_off.size(),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return fail_free(TN_ECUDA);
  for (size_t k = 0; k < opsites.size(); ++k) {
    const int v = opsites[k];
    const int64_t len = h->t_len[v];
    if (cudaMemcpyAsync(bra + op_off[k], site_ptr(h, h->T, v), sizeof(float) * 4 * len,
                        cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return fail_free(TN_ECUDA);
    // Pauli on p: u = [[u00, u01], [u10, u11]] as (re, im) pairs
    float u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (op[v] == 'X') { u[2] = 1; u[4] = 1; }
    else if (op[v] == 'Y') { u[3] = -1; u[5] = 1; }
    else { u[0] = 1; u[6] = -1; }
    if (launch_phys_gate(bra, d_off + k, 1, len, 2 * len, u[0], u[1], u[2], u[3], u[4], u[5],
                         u[6], u[7], h->stream) != cudaSuccess)
      return fail_free(TN_ECUDA);
    const int d = g.degree(v);
    if (d >= 2 && launch_first_leg_last(bra, braA, d_off + k, 1, d, x, h->stream) != cudaSuccess)
      return fail_free(TN_ECUDA);
  }
  if (cudaMemsetAsync(scal, 0, 3 * sizeof(double) + sizeof(int), h->stream) != cudaSuccess)
    return fail_free(TN_ECUDA);
  for (auto it = order.rbegin(); it != order.rend() && st == TN_OK; ++it) {
    const int v = *it;
    const auto& lg = g.legs[v];
    const int d = (int)lg.size();
    const bool is_root = parent[v] == -1;
    float* out = is_root ? root_out : up + eidx[parent[v]] * 2 * c2;
    ChainSite c = handle_site(h, v, out);
    for (size_t k = 0; k < opsites.size(); ++k)
      if (opsites[k] == v) { c.bra = bra + op_off[k]; c.braA = braA + op_off[k]; }
    for (int j = 0; j < d; ++j)
      if (eidx[lg[j]] >= 0 && lg[j] != parent[v]) c.m[j] = upr + eidx[lg[j]] * 4 * c2;
    const int open = is_root ? 0 : g.leg_pos(v, parent[v]);
    Plan P;
    if (d == 3) deg3_chain_sites(h, P, open, {c}, false);
    else if (d == 2) deg2_chain_sites(h, P, open, {c}, false);
    else add_close(P, 1, 0, x, false, h->cfg.prec, {{c.T, c.bra, out}});
    st = run_adhoc(h, P, arena);
    if (st) break;
    if (!is_root) {
      if (launch_scale_unit(out, x, scal + 2, zflag, h->stream) != cudaSuccess ||
          launch_realify(out, 2 * c2, upr + eidx[parent[v]] * 4 * c2, 1, x, h->stream) != cudaSuccess)
        st = TN_ECUDA;
    } else {
      const int e = lg[0];
      const float* m_in = eidx[e] >= 0 ? up + eidx[e] * 2 * c2
                                       : msg_ptr(h, h->msg, dir_id(g, g.other(e, v), e));
      if (launch_dot_msgs(root_out, m_in, x, scal, h->stream) != cudaSuccess) st = TN_ECUDA;
    }
  }
  double hs[4] = {0, 0, 0, 0};
  if (st == TN_OK &&
      (cudaMemcpyAsync(hs, scal, 3 * sizeof(double) + sizeof(int), cudaMemcpyDeviceToHost,
                       h->stream) != cudaSuccess ||
       cudaStreamSynchronize(h->stream) != cudaSuccess))
    st = TN_ECUDA;
  if (st) return fail_free(st);
  dev_free(h, buf);
  *re = hs[0];
  *im = hs[1];
  *logscale = hs[2];
  int zf = 0;
  memcpy(&zf, &hs[3], sizeof(int));
  *zero = zf != 0;
  return TN_OK;
}

tn_status region_expectation(tn_handle* h, const tn_pauli& P, double* out) {
  std::vector<int> terms(P.sites, P.sites + P.weight);
  const std::vector<int> tree = steiner_edges(h->g, terms);
  std::vector<char> op(h->g.n, 0), none(h->g.n, 0);
  for (int j = 0; j < P.weight; ++j) op[P.sites[j]] = P.paulis[j];
  tn_status st = ensure_ta(h);
  if (st) return st;
  st = ensure_mrt(h);
  if (st) return st;
  double nr, ni, nl, dr, di, dl;
  bool nz, dz;
  st = region_contract(h, tree, op, &nr, &ni, &nl, &nz);
  if (st) return st;
  st = region_contract(h, tree, none, &dr, &di, &dl, &dz);
  if (st) return st;
  if (dz || !(dr * dr + di * di > 0.0)) {
    set_error("the region's norm contraction vanished");
    return TN_ENUMERIC;
  }
  if (nz) { *out = 0.0; return TN_OK; }
  // (n / d) exp(nl - dl), real part (P is Hermitian)
  const double den = dr * dr + di * di;
  *out = (nr * dr + ni * di) / den * exp(nl - dl);
  return TN_OK;
}

tn_status tn_expect(tn_handle* h, const tn_pauli* ops, int32_t n_ops, int32_t method,
                    double* out) {
  if (!h || (!ops && n_ops > 0) || (!out && n_ops > 0)) { set_error("null argument"); return TN_EINVAL; }
  if (method != 0 && method != 1) { set_error("method must be 0 or 1"); return TN_EINVAL; }
  const int n = h->g.n;
  for (int i = 0; i < n_ops; ++i) {
    if (ops[i].weight < 1 || !ops[i].sites || !ops[i].paulis) {
      set_error("Pauli string " + std::to_string(i) + " is empty");
      return TN_EINVAL;
    }
    std::vector<int> seen(n, 0);
    for (int j = 0; j < ops[i].weight; ++j) {
      const int q = ops[i].sites[j];
      const char p = ops[i].paulis[j];
      if (q < 0 || q >= n || seen[q] || (p != 'X' && p != 'Y' && p != 'Z')) {
        set_error("Pauli string " + std::to_string(i) + " has a bad site or letter");
        return TN_EINVAL;
      }
      seen[q] = 1;
    }
  }
  std::vector<double> rho;
  bool have_rho = false;
  for (int i = 0; i < n_ops; ++i) {
    const tn_pauli& P = ops[i];
    const double sgn = P.sign < 0 ? -1.0 : 1.0;
    if (P.weight == 1) {
      if (!have_rho) {
        tn_status st = compute_rho(h, &rho);
        if (st) return st;
        have_rho = true;
      }
      out[i] = sgn * pauli_from_rho(&rho[8 * P.sites[0]], P.paulis[0]);
      continue;
    }
    if (method == 0) {
      double v = 0.0;
      tn_status st = region_expectation(h, P, &v);
      if (st) return st;
      out[i] = sgn * v;
      continue;
    }
    PauliString s;
    s.ops.assign(n, 0);
    for (int j = 0; j < P.weight; ++j)
      s.ops[P.sites[j]] = P.paulis[j] == 'X' ? 1 : P.paulis[j] == 'Y' ? 2 : 3;
    int site = -1, np = 0, zs = 1;
    if (!reduce_to_single_z(s, h->g, 32, &site, &np, &zs)) {
      set_error("string " + std::to_string(i) + " is not U^n'(pi/2) Z_i U^-n'(pi/2) for n' <= 32");
      return TN_EUNSUPPORTED;
    }
    tn_status st = backup_state(h, false);
    if (st) return st;
    tn_stats keep = h->stats;
    st = evolve(h, 0.0, np, true);
    if (st && st != TN_ENOTCONVERGED) { backup_state(h, true); return st; }
    std::vector<double> r2;
    st = compute_rho(h, &r2);
    tn_status st2 = backup_state(h, true);
    h->stats = keep;
    if (st) return st;
    if (st2) return st2;
    out[i] = sgn * zs * pauli_from_rho(&r2[8 * site], 'Z');
  }
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return TN_OK;
}

tn_status tn_state_size(const tn_handle* h, size_t* bytes) {
  if (!h || !bytes) { set_error("null argument"); return TN_EINVAL; }
  *bytes = ckpt_bytes(ckpt_header(h));
  return TN_OK;
}

tn_status tn_save_state(tn_handle* h, void* host, size_t bytes) {
  if (!h || !host) { set_error("null argument"); return TN_EINVAL; }
  const CkptHeader c = ckpt_header(h);
  if (bytes < ckpt_bytes(c)) {
    set_error("checkpoint buffer too small: " + std::to_string(ckpt_bytes(c)) + " bytes needed");
    return TN_EINVAL;
  }
  unsigned char* p = (unsigned char*)host;
  memcpy(p, &c, sizeof(c));
  p += sizeof(c);
  TN_CUDA_TRY(cudaMemcpyAsync(p, h->T, sizeof(float) * c.t_floats, cudaMemcpyDeviceToHost,
                              h->stream));
  p += sizeof(float) * c.t_floats;
  TN_CUDA_TRY(cudaMemcpyAsync(p, h->msg, sizeof(float) * c.msg_floats, cudaMemcpyDeviceToHost,
                              h->stream));
  p += sizeof(float) * c.msg_floats;
  TN_CUDA_TRY(cudaMemcpyAsync(p, h->spectra, sizeof(double) * c.spec_doubles,
                              cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return TN_OK;
}

tn_status tn_load_state(tn_handle* h, const void* host, size_t bytes) {
  if (!h || !host) { set_error("null argument"); return TN_EINVAL; }
  const CkptHeader want = ckpt_header(h);
  CkptHeader c;
  if (bytes < sizeof(c)) { set_error("checkpoint too short"); return TN_EINVAL; }
  memcpy(&c, host, sizeof(c));
  if (c.magic != kCkptMagic) { set_error("not a checkpoint of this library"); return TN_EINVAL; }
  if (c.graph_hash != want.graph_hash || c.n_vertices != want.n_vertices ||
      c.n_edges != want.n_edges || c.chi != want.chi || c.t_floats != want.t_floats ||
      c.msg_floats != want.msg_floats || c.spec_doubles != want.spec_doubles) {
    set_error("checkpoint of another graph or chi");
    return TN_EINVAL;
  }
  if (bytes < ckpt_bytes(c)) { set_error("checkpoint truncated"); return TN_EINVAL; }
  const unsigned char* p = (const unsigned char*)host + sizeof(c);
  TN_CUDA_TRY(cudaMemcpyAsync(h->T, p, sizeof(float) * c.t_floats, cudaMemcpyHostToDevice,
                              h->stream));
  p += sizeof(float) * c.t_floats;
  TN_CUDA_TRY(cudaMemcpyAsync(h->msg, p, sizeof(float) * c.msg_floats, cudaMemcpyHostToDevice,
                              h->stream));
  p += sizeof(float) * c.msg_floats;
  TN_CUDA_TRY(cudaMemcpyAsync(h->spectra, p, sizeof(double) * c.spec_doubles,
                              cudaMemcpyHostToDevice, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->ta_valid = false;
  h->mrt_valid = false;
  return TN_OK;
}

tn_status tn_bond_spectrum(tn_handle* h, int32_t e, double* out) {
  if (!h || !out) { set_error("null argument"); return TN_EINVAL; }
  if (e < 0 || e >= (int32_t)h->g.eu.size()) { set_error("edge out of range"); return TN_EINVAL; }
  TN_CUDA_TRY(cudaMemcpyAsync(out, h->spectra + (int64_t)h->spec_row[e] * h->chi,
                              sizeof(double) * h->chi, cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return TN_OK;
}

tn_status tn_entanglement_entropy(tn_handle* h, int32_t e, double* out) {
  if (!out) { set_error("null argument"); return TN_EINVAL; }
  std::vector<double> sp(h ? h->chi : 0);
  tn_status st = tn_bond_spectrum(h, e, sp.data());
  if (st) return st;
  double s = 0.0;
  for (double l : sp) {
    const double p = l * l;
    if (p > 0.0) s -= p * std::log2(p);
  }
  *out = s;
  return TN_OK;
}

tn_status tn_vidal_gauge(tn_handle* h, double* lambda_out) {
  if (!h || !lambda_out) { set_error("null argument"); return TN_EINVAL; }
  const HostGraph& g = h->g;
  const int E = (int)g.eu.size(), x = h->chi;
  const int64_t c2 = (int64_t)x * x;
  if (!h->gamma) {
    h->gamma = (float*)dev_alloc(h, sizeof(float) * h->t_floats);
    if (!h->gamma) { set_error("device allocation of the Vidal-gauge tensors failed"); return TN_ENOMEM; }
  }
  // per-edge scratch, leg matrices, bond weights, message ids and the pointer
  // arena of the site contractions (one entry per site and leg: 2 E in all)
  const size_t n_ptr = 3 * 2 * (size_t)E;
  const size_t work_d = vidal_work_doubles(x) * (size_t)std::max(E, 1);
  const size_t bytes = sizeof(double) * (work_d + (size_t)E * x) + sizeof(float) * 4 * c2 * E +
                       sizeof(int32_t) * 2 * E + sizeof(void*) * n_ptr + 64;
  unsigned char* buf = (unsigned char*)dev_alloc(h, bytes);
  if (!buf) { set_error("device allocation for the Vidal gauge failed"); return TN_ENOMEM; }
  double* work = (double*)buf;
  double* lam = work + work_d;
  float* gout = (float*)(lam + (size_t)E * x);
  int32_t* ddir = (int32_t*)(gout + 4 * c2 * E);
  void* arena = (void*)(((uintptr_t)(ddir + 2 * E) + 15) & ~uintptr_t(15));
  auto fail_free = [&](tn_status code) { cudaStreamSynchronize(h->stream); dev_free(h, buf); return code; };
  // Gamma_v = T_v with leg j contracted into the leg matrix of (v, legs[v][j]),
  // leg by leg through the site-shaped intermediates
  Plan P;
  for (int d = 1; d <= 3; ++d) {
    const std::vector<int>& sites = h->sites_by_deg[d];
    if (sites.empty()) continue;
    for (int j = 0; j < d; ++j) {
      std::vector<std::array<const float*, 3>> ent;
      for (int v : sites) {
        const int e = g.legs[v][j];
        const float* X = j == 0 ? site_ptr(h, h->T, v) : site_ptr(h, (j & 1) ? h->Y1 : h->Y2, v);
        const float* Y = j == d - 1 ? h->gamma + h->t_off[v] : site_ptr(h, (j & 1) ? h->Y2 : h->Y1, v);
        const float* G = gout + (int64_t)(2 * e + (g.eu[e] == v ? 0 : 1)) * 2 * c2;
        ent.push_back({X, G, Y});
      }
      add_mode_product(P, d, j, x, TN_FP32, ent);
    }
  }
  std::vector<int32_t> dir(2 * E);
  for (int e = 0; e < E; ++e) {
    dir[2 * e] = dir_id(g, g.eu[e], e);
    dir[2 * e + 1] = dir_id(g, g.ew[e], e);
  }
  std::vector<const void*> host;
  for (auto& L : P.L) {
    for (auto q : L.A) host.push_back(q);
    for (auto q : L.B) host.push_back(q);
    for (auto q : L.C) host.push_back(q);
  }
  if (host.size() > n_ptr) return fail_free(TN_EINVAL);
  if (E > 0 && (cudaMemcpyAsync(ddir, dir.data(), sizeof(int32_t) * 2 * E, cudaMemcpyHostToDevice,
                                h->stream) != cudaSuccess ||
                launch_vidal_edges(h->msg, ddir, E, x, work, gout, lam, h->flags, h->stream) !=
                    cudaSuccess))
    return fail_free(TN_ECUDA);
  h->stats.kernel_launches += E > 0 ? 1 : 0;
  if (!host.empty() && cudaMemcpyAsync(arena, host.data(), host.size() * sizeof(void*),
                                       cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return fail_free(TN_ECUDA);
  {
    const void** base = (const void**)arena;
    size_t pos = 0;
    for (auto& L : P.L) {
      L.d.A = (const float* const*)(base + pos); pos += L.A.size();
      L.d.B = (const float* const*)(base + pos); pos += L.B.size();
      L.d.C = (float* const*)(base + pos); pos += L.C.size();
      // FP32 CUDA-core contractions whatever the handle's precision
      if (launch_cgemm(L.d, h->stream) != cudaSuccess) return fail_free(TN_ECUDA);
      h->stats.kernel_launches++;
    }
  }
  for (int v : h->sites_by_deg[0])
    if (cudaMemcpyAsync(h->gamma + h->t_off[v], site_ptr(h, h->T, v),
                        sizeof(float) * 4 * h->t_len[v], cudaMemcpyDeviceToDevice,
                        h->stream) != cudaSuccess)
      return fail_free(TN_ECUDA);
  if (E > 0 && cudaMemcpyAsync(lambda_out, lam, sizeof(double) * E * x, cudaMemcpyDeviceToHost,
                               h->stream) != cudaSuccess)
    return fail_free(TN_ECUDA);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_free(TN_ECUDA);
  dev_free(h, buf);
  return check_flags(h, "the Vidal gauge");
}

tn_status tn_selftest_bounded_wait(void* cuda_stream, int32_t* flags_out) {
  if (!flags_out) { set_error("null argument"); return TN_EINVAL; }
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  TN_CUDA_TRY(cudaMalloc(&d, sizeof(int)));
  int f = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_wait_selftest(d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  TN_CUDA_TRY(e);
  *flags_out = f;
  return TN_OK;
}

tn_status tn_graph_info(const tn_handle* h, int32_t* n_vertices, int32_t* n_edges, int32_t* chi,
                        int32_t* edges_out, int32_t capacity) {
  if (!h || !n_vertices || !n_edges || !chi) { set_error("null argument"); return TN_EINVAL; }
  const int32_t m = (int32_t)h->g.eu.size();
  *n_vertices = h->g.n;
  *n_edges = m;
  *chi = h->chi;
  if (edges_out) {
    if (capacity < m) { set_error("edge buffer too small"); return TN_EINVAL; }
    for (int32_t e = 0; e < m; ++e) {
      edges_out[2 * e] = h->g.eu[e];
      edges_out[2 * e + 1] = h->g.ew[e];
    }
  }
  return TN_OK;
}

tn_status tn_get_gamma(tn_handle* h, int32_t v, float* host_out, size_t n_floats) {
  if (!h || !host_out) { set_error("null argument"); return TN_EINVAL; }
  if (!h->gamma) { set_error("tn_vidal_gauge has not run on this handle"); return TN_EINVAL; }
  if (v < 0 || v >= h->g.n) { set_error("vertex out of range"); return TN_EINVAL; }
  const int64_t len = h->t_len[v];
  if (n_floats != (size_t)(4 * len)) { set_error("site buffer must hold 4*chi^d floats"); return TN_EINVAL; }
  std::vector<float> planar(4 * len);
  TN_CUDA_TRY(cudaMemcpyAsync(planar.data(), h->gamma + h->t_off[v], sizeof(float) * 4 * len,
                              cudaMemcpyDeviceToHost, h->stream));
  TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int64_t i = 0; i < 2 * len; ++i) {
    host_out[2 * i] = planar[i];
    host_out[2 * i + 1] = planar[2 * len + i];
  }
  return TN_OK;
}

}  // extern "C"

namespace tnbp {
// Device view of the Vidal-gauge site tensor of v from the last tn_vidal_gauge
// call (planar: the real plane [p][legs], then the imaginary plane), its
// length chi^d and the handle's stream.
tn_status gamma_view(tn_handle* h, int v, const float** ptr, int64_t* len, cudaStream_t* stream) {
  if (!h->gamma) { set_error("tn_vidal_gauge has not run on this handle"); return TN_EINVAL; }
  if (v < 0 || v >= h->g.n) { set_error("vertex out of range"); return TN_EINVAL; }
  *ptr = h->gamma + h->t_off[v];
  *len = h->t_len[v];
  *stream = h->stream;
  return TN_OK;
}
}  // namespace tnbp

extern "C" {

tn_status tn_truncation_solve(const float* gram, float* dmat, double* s_out, int32_t n_edges,
                              int32_t chi, int32_t sign, double svd_cutoff, void* cuda_stream) {
  return tn_truncation_solve_ex(gram, dmat, s_out, n_edges, chi, sign, svd_cutoff, TN_SOLVE_FP64,
                                cuda_stream);
}

tn_status tn_truncation_solve_ex(const float* gram, float* dmat, double* s_out, int32_t n_edges,
                                 int32_t chi, int32_t sign, double svd_cutoff, int32_t solve,
                                 void* cuda_stream) {
  if (solve != TN_SOLVE_AUTO && solve != TN_SOLVE_SHARED && solve != TN_SOLVE_FP64 &&
      solve != TN_SOLVE_REFINED) {
    set_error("unknown truncation solve");
    return TN_EINVAL;
  }
  if ((solve == TN_SOLVE_SHARED && !solve32_supported(chi)) ||
      (solve == TN_SOLVE_REFINED && !solve_refined_supported(chi))) {
    set_error("the shared-memory and refined solves support chi <= 64");
    return TN_EUNSUPPORTED;
  }
  if (!gram || !dmat || !s_out) { set_error("null argument"); return TN_EINVAL; }
  if (n_edges < 1 || chi < 1 || 2 * chi > 512 || (sign != 1 && sign != -1)) {
    set_error("n_edges >= 1, 1 <= chi <= 256 and sign = +-1 required");
    return TN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t wbytes = sizeof(double) * (size_t)n_edges * solve_work_doubles(chi);
  const size_t sbytes = sizeof(double) * 4 * (size_t)n_edges;
  void *work = nullptr, *stats = nullptr, *flags = nullptr;
  TN_CUDA_TRY(cudaMallocAsync(&work, wbytes, st));
  TN_CUDA_TRY(cudaMallocAsync(&stats, sbytes, st));
  TN_CUDA_TRY(cudaMallocAsync(&flags, sizeof(int), st));
  TN_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), st));
  SolveArgs a;
  a.n_edges = n_edges;
  a.chi = chi;
  a.sign = sign;
  a.gram_cut = 1e-13;
  a.svd_cut = svd_cutoff > 0 ? svd_cutoff : 1e-6;
  a.gram = gram;
  a.dmat = dmat;
  a.msg = nullptr;
  a.msg_vw = nullptr;
  a.s_out = s_out;
  a.work = (double*)work;
  a.stats = (double*)stats;
  a.flags = (int*)flags;
  a.max_sweeps = 30;
  cudaError_t le;
  const int kind = solve_kind(solve, chi);
  if (kind == TN_SOLVE_SHARED) {
    a.max_sweeps = 20;
    le = launch_solve32(a, st);
  } else if (kind == TN_SOLVE_REFINED) {
    a.max_sweeps = 20;
    le = launch_solve_refined(a, st);
  } else {
    le = launch_solve(a, st);
  }
  int f = 0;
  cudaError_t ce = cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(work, st);
  cudaFreeAsync(stats, st);
  cudaFreeAsync(flags, st);
  TN_CUDA_TRY(le);
  TN_CUDA_TRY(ce);
  TN_CUDA_TRY(cudaStreamSynchronize(st));
  if (f) { set_error("non-finite or zero bond spectrum in the truncation solve"); return TN_ENUMERIC; }
  return TN_OK;
}

tn_status tn_get_stats(const tn_handle* h, tn_stats* out) {
  if (!h || !out) { set_error("null argument"); return TN_EINVAL; }
  *out = h->stats;
  return TN_OK;
}

static tn_status site_io(tn_handle* h, int v, float* buf, size_t n_floats, bool get) {
  if (!h || !buf) { set_error("null argument"); return TN_EINVAL; }
  if (v < 0 || v >= h->g.n) { set_error("vertex out of range"); return TN_EINVAL; }
  const int64_t len = h->t_len[v];
  if (n_floats != (size_t)(4 * len)) { set_error("site buffer must hold 4*chi^d floats"); return TN_EINVAL; }
  std::vector<float> planar(4 * len);
  if (get) {
    TN_CUDA_TRY(cudaMemcpyAsync(planar.data(), h->T + h->t_off[v], sizeof(float) * 4 * len,
                                cudaMemcpyDeviceToHost, h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < 2 * len; ++i) {
      buf[2 * i] = planar[i];
      buf[2 * i + 1] = planar[2 * len + i];
    }
  } else {
    for (int64_t i = 0; i < 2 * len; ++i) {
      planar[i] = buf[2 * i];
      planar[2 * len + i] = buf[2 * i + 1];
    }
    TN_CUDA_TRY(cudaMemcpyAsync(h->T + h->t_off[v], planar.data(), sizeof(float) * 4 * len,
                                cudaMemcpyHostToDevice, h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->ta_valid = false;
  }
  return TN_OK;
}

tn_status tn_get_site(tn_handle* h, int32_t v, float* host_out, size_t n_floats) {
  return site_io(h, v, host_out, n_floats, true);
}
tn_status tn_set_site(tn_handle* h, int32_t v, const float* host_in, size_t n_floats) {
  return site_io(h, v, const_cast<float*>(host_in), n_floats, false);
}

static tn_status msg_io(tn_handle* h, int e, int src, float* buf, size_t n_floats, bool get) {
  if (!h || !buf) { set_error("null argument"); return TN_EINVAL; }
  if (e < 0 || e >= (int)h->g.eu.size() || (src != h->g.eu[e] && src != h->g.ew[e])) {
    set_error("edge or source vertex out of range");
    return TN_EINVAL;
  }
  const int64_t c2 = (int64_t)h->chi * h->chi;
  if (n_floats != (size_t)(2 * c2)) { set_error("message buffer must hold 2*chi^2 floats"); return TN_EINVAL; }
  float* dev = h->msg + (int64_t)dir_id(h->g, src, e) * 2 * c2;
  std::vector<float> planar(2 * c2);
  if (get) {
    TN_CUDA_TRY(cudaMemcpyAsync(planar.data(), dev, sizeof(float) * 2 * c2, cudaMemcpyDeviceToHost,
                                h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < c2; ++i) { buf[2 * i] = planar[i]; buf[2 * i + 1] = planar[c2 + i]; }
  } else {
    for (int64_t i = 0; i < c2; ++i) { planar[i] = buf[2 * i]; planar[c2 + i] = buf[2 * i + 1]; }
    TN_CUDA_TRY(cudaMemcpyAsync(dev, planar.data(), sizeof(float) * 2 * c2, cudaMemcpyHostToDevice,
                                h->stream));
    TN_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->mrt_valid = false;
  }
  return TN_OK;
}

tn_status tn_get_message(tn_handle* h, int32_t e, int32_t src, float* host_out, size_t n_floats) {
  return msg_io(h, e, src, host_out, n_floats, true);
}
tn_status tn_set_message(tn_handle* h, int32_t e, int32_t src, const float* host_in,
                         size_t n_floats) {
  return msg_io(h, e, src, const_cast<float*>(host_in), n_floats, false);
}

tn_status tn_clifford_reduce(const tn_graph* graph, const tn_pauli* op, int32_t max_steps,
                             int32_t* site_out, int32_t* nprime_out, int32_t* sign_out) {
  if (!graph || !op || !site_out || !nprime_out || !sign_out) { set_error("null argument"); return TN_EINVAL; }
  HostGraph g;
  std::string why;
  if (!build_graph(graph->n_vertices, graph->n_edges, graph->edges, graph->colour, &g, &why)) {
    set_error(why);
    return TN_EINVAL;
  }
  PauliString s;
  s.ops.assign(g.n, 0);
  if (op->weight < 1 || !op->sites || !op->paulis) { set_error("empty Pauli string"); return TN_EINVAL; }
  for (int j = 0; j < op->weight; ++j) {
    const int q = op->sites[j];
    const char p = op->paulis[j];
    if (q < 0 || q >= g.n || s.ops[q] || (p != 'X' && p != 'Y' && p != 'Z')) {
      set_error("bad site or letter in the Pauli string");
      return TN_EINVAL;
    }
    s.ops[q] = p == 'X' ? 1 : p == 'Y' ? 2 : 3;
  }
  int site = -1, np = 0, zs = 1;
  if (!reduce_to_single_z(s, g, max_steps, &site, &np, &zs)) {
    set_error("no n' <= max_steps reduces the string to a single Z");
    return TN_EUNSUPPORTED;
  }
  *site_out = site;
  *nprime_out = np;
  *sign_out = zs * (op->sign < 0 ? -1 : 1);
  return TN_OK;
}

tn_status tn_footprint(const tn_handle* h, size_t* bytes_out) {
  if (!h || !bytes_out) { set_error("null argument"); return TN_EINVAL; }
  *bytes_out = h->bytes;
  return TN_OK;
}

}  // extern "C"
