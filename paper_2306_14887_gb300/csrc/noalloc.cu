// Allocation-free variant of the standalone FP64 truncation solve.
//
// Some callers cannot allocate device memory: a host application or serving
// runtime that owns the whole device memory pool and forbids foreign
// allocations, or a latency-bound loop that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree may imply.  tn_truncation_solve_noalloc
// serves them: its FP64 workspace is a fixed file-scope device array instead
// of memory obtained at call time.  The caller still passes the input and
// output buffers.
#include <mutex>

#include "common.cuh"
#include "tnbp.h"

namespace tnbp {
namespace {

// 16 MiB of FP64 workspace, held by every GPU that loads the library until
// the process exits.
constexpr size_t kScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_solve_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_solve_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current and cached for the life of the process
// (a cudaDeviceReset by the application would leave the cached address
// pointing into a destroyed context; the header says so).
tn_status scratch_address(double** out) {
  int dev = 0;
  TN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal beyond the allocation-free solve's table");
    return TN_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    TN_CUDA_TRY(cudaGetSymbolAddress(&p, g_solve_scratch));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return TN_OK;
}

}  // namespace
}  // namespace tnbp

using namespace tnbp;

extern "C" tn_status tn_truncation_solve_noalloc(const float* gram, float* dmat, double* s_out,
                                                 int32_t n_edges, int32_t chi, int32_t sign,
                                                 double svd_cutoff, void* cuda_stream) {
  if (!gram || !dmat || !s_out) { set_error("null argument"); return TN_EINVAL; }
  if (n_edges < 1 || chi < 1 || 2 * chi > 512 || (sign != 1 && sign != -1)) {
    set_error("n_edges >= 1, 1 <= chi <= 256 and sign = +-1 required");
    return TN_EINVAL;
  }
  const size_t work = (size_t)n_edges * solve_work_doubles(chi);
  const size_t need = work + 4 * (size_t)n_edges + 1;
  if (need > kScratchDoubles) {
    set_error("allocation-free solve needs " + std::to_string(need * 8) +
              " bytes of workspace (12 (2 chi)^2 + 4 doubles per edge); its fixed workspace is " +
              std::to_string(kScratchDoubles * 8) + " bytes: lower n_edges or chi");
    return TN_EINVAL;
  }
  double* base = nullptr;
  tn_status st = scratch_address(&base);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* stats = base + work;
  int* flags = reinterpret_cast<int*>(stats + 4 * (size_t)n_edges);
  // the array keeps the previous call's contents: the error flag must start at zero
  TN_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
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
  a.work = base;
  a.stats = stats;
  a.flags = flags;
  a.max_sweeps = 30;
  TN_CUDA_TRY(launch_solve(a, s));
  int f = 0;
  TN_CUDA_TRY(cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  TN_CUDA_TRY(cudaStreamSynchronize(s));
  if (f) { set_error("non-finite or zero bond spectrum in the truncation solve"); return TN_ENUMERIC; }
  return TN_OK;
}
