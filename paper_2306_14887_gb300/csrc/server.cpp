// Serving: a request loop that takes (graph, chi, theta_h, steps) jobs as they
// arrive, keeps each job's tensors and messages on the device across its
// Floquet steps, and admits jobs by HBM footprint (continuous batching: a job
// that arrives while others run starts as soon as a slot and memory are free,
// and its kernels overlap theirs on the device).
//
// Design: max_slots host threads ("slots"), each with its own non-blocking CUDA
// stream.  A slot takes a queued job once the sum of the resident jobs'
// footprints (tn_footprint_estimate) plus the job's own stays within the
// budget: the oldest (TN_SERVE_FIFO) or the one with the least estimated work
// among those that fit (TN_SERVE_SHORTEST); it creates the job's handle on its stream with stream-ordered
// allocation (cudaMallocAsync / cudaFreeAsync, so that freeing never
// synchronises the device), runs every step, reads <Z_v> for all vertices and
// destroys the handle.  Jobs never share device memory or streams, and every
// kernel of the library is deterministic (fixed reduction orders), so a job's
// result is the same whether it runs alone or in a mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "tnbp.h"

namespace tnbp {
void set_error(const std::string& msg);  // the thread-local tn_last_error text (engine.cu)
}

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  int32_t n = 0;
  std::vector<int32_t> edges;
  std::vector<uint8_t> colours;
  bool has_colours = false;
  tn_config cfg{};
  double theta = 0.0;
  int32_t steps = 0;
  size_t footprint = 0;
  double work = 0.0;  // estimated work (TN_SERVE_SHORTEST)
  Clock::time_point t_submit, t_admit, t_done;
  tn_status status = TN_EAGAIN;
  int32_t steps_done = 0;
  std::vector<double> z;
  std::string error;  // the worker's error message when status is an error
  // the job's strings (deep copies of the submitted tn_pauli array)
  std::vector<std::vector<int32_t>> op_sites;
  std::vector<std::string> op_labels;
  std::vector<int8_t> op_signs;
  int32_t ops_method = 0;
  std::vector<double> op_values;
};

void* slot_alloc(size_t bytes, void*, void* stream) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void slot_free(void* p, size_t, void*, void* stream) {
  if (p) cudaFreeAsync(p, (cudaStream_t)stream);
}

}  // namespace

struct tn_server {
  tn_server_config cfg{};
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  bool stopping = false;
  tn_server_stats st{};
  std::vector<std::thread> slots;

  void run_slot();
  // the queued job a free slot takes next under the policy (queue.end(): none fits)
  std::deque<std::shared_ptr<Job>>::iterator pick() {
    if (queue.empty()) return queue.end();
    if (cfg.policy != TN_SERVE_SHORTEST)
      return st.used_bytes + queue.front()->footprint <= budget ? queue.begin() : queue.end();
    auto best = queue.end();
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      if (st.used_bytes + (*it)->footprint > budget) continue;
      if (best == queue.end() || (*it)->work < (*best)->work) best = it;
    }
    return best;
  }
};

void tn_server::run_slot() {
  cudaStream_t stream = nullptr;
  bool dev_ok = cudaSetDevice(cfg.device) == cudaSuccess &&
                cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  tn_allocator alloc{slot_alloc, slot_free, nullptr};
  while (true) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stopping || pick() != queue.end(); });
      if (stopping) break;
      const auto it = pick();
      job = *it;
      queue.erase(it);
      st.used_bytes += job->footprint;
      st.resident++;
      if (st.used_bytes > st.peak_bytes) st.peak_bytes = st.used_bytes;
      if (st.resident > st.peak_resident) st.peak_resident = st.resident;
      job->t_admit = Clock::now();
    }
    tn_status status = TN_ECUDA;
    std::string err = dev_ok ? "" : "cudaSetDevice or cudaStreamCreate failed for the slot";
    int32_t done_steps = 0;
    std::vector<double> z(job->n, 0.0), op_vals;
    if (dev_ok) {
      tn_graph g{job->n, (int32_t)(job->edges.size() / 2), job->edges.data(),
                 job->has_colours ? job->colours.data() : nullptr, 0};
      tn_handle* h = nullptr;
      status = tn_create(&g, &job->cfg, &alloc, stream, &h);
      if (status == TN_OK) {
        status = tn_apply_floquet(h, job->theta, job->steps);
        tn_stats s{};
        tn_get_stats(h, &s);
        done_steps = s.steps_done;
        if (status == TN_OK || status == TN_ENOTCONVERGED) {
          const tn_status zs = tn_expect_z_all(h, z.data());
          if (zs != TN_OK) status = zs;
        }
        if ((status == TN_OK || status == TN_ENOTCONVERGED) && !job->op_signs.empty()) {
          const size_t n_ops = job->op_signs.size();
          std::vector<tn_pauli> ops(n_ops);
          for (size_t k = 0; k < n_ops; ++k) {
            ops[k].weight = (int32_t)job->op_sites[k].size();
            ops[k].sites = job->op_sites[k].data();
            ops[k].paulis = job->op_labels[k].c_str();
            ops[k].sign = job->op_signs[k];
          }
          op_vals.assign(n_ops, 0.0);
          const tn_status os =
              tn_expect(h, ops.data(), (int32_t)n_ops, job->ops_method, op_vals.data());
          if (os != TN_OK) status = os;
        }
        if (status != TN_OK && status != TN_ENOTCONVERGED) err = tn_last_error();
        tn_destroy(h);
      } else {
        err = tn_last_error();
      }
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      job->status = status;
      job->error = err;
      job->op_values.swap(op_vals);
      job->steps_done = done_steps;
      job->z.swap(z);
      job->t_done = Clock::now();
      st.used_bytes -= job->footprint;
      st.resident--;
      if (status == TN_OK || status == TN_ENOTCONVERGED) st.completed++;
      else st.failed++;
    }
    cv.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

extern "C" {

tn_status tn_server_create(const tn_server_config* cfg, tn_server** out) {
  if (!cfg || !out) return TN_EINVAL;
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->device < 0) return TN_EINVAL;
  if (cfg->policy != TN_SERVE_FIFO && cfg->policy != TN_SERVE_SHORTEST) return TN_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || cfg->device >= count) {
    cudaGetLastError();
    return TN_ECUDA;
  }
  size_t budget = cfg->hbm_budget;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(cfg->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      return TN_ECUDA;
    }
    cudaSetDevice(prev);
    budget = free_b / 10 * 9;
  }
  tn_server* s = new tn_server();
  s->cfg = *cfg;
  s->budget = budget;
  s->st.budget_bytes = budget;
  for (int i = 0; i < cfg->max_slots; ++i) s->slots.emplace_back([s] { s->run_slot(); });
  *out = s;
  return TN_OK;
}

tn_status tn_server_submit(tn_server* s, const tn_job* job, uint64_t* ticket) {
  if (!s || !job || !ticket || !job->graph.edges || job->steps < 0) return TN_EINVAL;
  size_t fp = 0;
  tn_status v = tn_footprint_estimate(&job->graph, &job->cfg, &fp);
  if (v != TN_OK) return v;
  if (job->cfg.chi < 1 || job->cfg.chi > 256) return TN_EINVAL;
  auto j = std::make_shared<Job>();
  j->n = job->graph.n_vertices;
  j->edges.assign(job->graph.edges, job->graph.edges + 2 * (size_t)job->graph.n_edges);
  if (job->graph.colour) {
    j->colours.assign(job->graph.colour, job->graph.colour + job->graph.n_edges);
    j->has_colours = true;
  }
  j->cfg = job->cfg;
  j->theta = job->theta_h;
  j->steps = job->steps;
  j->footprint = fp;
  {
    // estimated work: BP message updates (chi^(d+1) per site and leg) and the
    // truncation solves (chi^3 per edge), per step
    std::vector<int> deg(j->n, 0);
    for (size_t k = 0; k < j->edges.size(); ++k)
      if (j->edges[k] >= 0 && j->edges[k] < j->n) deg[j->edges[k]]++;
    const double x = job->cfg.chi;
    double w = 8.0 * (double)job->graph.n_edges * x * x * x;
    for (int d : deg) w += d * std::pow(x, d + 1);
    j->work = w * std::max(1, job->steps);
  }
  if (job->n_ops < 0 || (job->n_ops > 0 && !job->ops) ||
      (job->n_ops > 0 && job->ops_method != 0 && job->ops_method != 1))
    return TN_EINVAL;
  j->ops_method = job->ops_method;
  for (int32_t k = 0; k < job->n_ops; ++k) {
    const tn_pauli& p = job->ops[k];
    if (p.weight < 1 || !p.sites || !p.paulis) return TN_EINVAL;
    j->op_sites.emplace_back(p.sites, p.sites + p.weight);
    j->op_labels.emplace_back(p.paulis, p.paulis + p.weight);
    j->op_signs.push_back(p.sign);
  }
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (fp > s->budget) return TN_ENOMEM;
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    s->st.submitted++;
    *ticket = j->ticket;
  }
  s->cv.notify_all();
  return TN_OK;
}

static tn_status take_result(tn_server* s, std::unordered_map<uint64_t, std::shared_ptr<Job>>::iterator it,
                             double* z, double* ops_out, tn_result* info) {
  Job& j = *it->second;
  if (z) for (int32_t i = 0; i < j.n; ++i) z[i] = j.z.empty() ? 0.0 : j.z[i];
  if (ops_out)
    for (size_t k = 0; k < j.op_signs.size(); ++k)
      ops_out[k] = k < j.op_values.size() ? j.op_values[k] : 0.0;
  if (info) {
    info->status = j.status;
    info->n_vertices = j.n;
    info->steps_done = j.steps_done;
    info->queue_s = std::chrono::duration<double>(j.t_admit - j.t_submit).count();
    info->latency_s = std::chrono::duration<double>(j.t_done - j.t_submit).count();
  }
  const tn_status status = j.status;
  // the message was set on the worker's thread; repeat it on the caller's
  if (status != TN_OK && status != TN_ENOTCONVERGED) tnbp::set_error(j.error);
  s->jobs.erase(it);
  return status;
}

tn_status tn_server_poll_ex(tn_server* s, uint64_t ticket, double* z, double* ops_out,
                            tn_result* info) {
  if (!s) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return TN_EINVAL;
  if (it->second->status == TN_EAGAIN) return TN_EAGAIN;
  return take_result(s, it, z, ops_out, info);
}

tn_status tn_server_poll(tn_server* s, uint64_t ticket, double* z, tn_result* info) {
  return tn_server_poll_ex(s, ticket, z, nullptr, info);
}

tn_status tn_server_wait(tn_server* s, uint64_t ticket, double timeout_s, double* z,
                         tn_result* info) {
  return tn_server_wait_ex(s, ticket, timeout_s, z, nullptr, info);
}

tn_status tn_server_wait_ex(tn_server* s, uint64_t ticket, double timeout_s, double* z,
                            double* ops_out, tn_result* info) {
  if (!s) return TN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return TN_EINVAL;
  std::shared_ptr<Job> j = it->second;
  // at most about 30 years ahead, so that the deadline fits the clock's range
  const double wait_s = timeout_s > 0 ? std::min(timeout_s, 1e9) : 0.0;
  const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(wait_s));
  while (j->status == TN_EAGAIN) {
    if (timeout_s <= 0 || s->cv.wait_until(lk, limit) == std::cv_status::timeout) {
      if (j->status == TN_EAGAIN) return TN_EAGAIN;
    }
  }
  it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return TN_EINVAL;  // taken by a concurrent poll
  return take_result(s, it, z, ops_out, info);
}

tn_status tn_server_get_stats(tn_server* s, tn_server_stats* out) {
  if (!s || !out) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (int32_t)s->queue.size();
  return TN_OK;
}

tn_status tn_server_destroy(tn_server* s) {
  if (!s) return TN_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto& t : s->slots) t.join();
  delete s;
  return TN_OK;
}

}  // extern "C"
