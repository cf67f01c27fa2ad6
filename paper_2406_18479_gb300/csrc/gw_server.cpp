// Request loop for scGW jobs: admission by device-memory budget, one worker
// thread and one CUDA stream per slot, continuous batching.
//
// A job is the self-consistency loop of Sec. 2.4 (gw_scgw): self-energy, iteration
// mixing or DIIS (Sec. 5.3), optionally the static part and the chemical-potential search,
// and the Dyson update of G, until max |dSigma| < tol or itermax evaluations.
// Jobs that arrive while others run are admitted as soon as a slot and enough
// of the budget are free; admitted jobs run on their own streams, so their
// kernels overlap on the device. Every job computes exactly what it computes
// alone: no state is shared between jobs and no kernel depends on timing.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gw_internal.h"

namespace gwi {
namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Job {
  uint64_t id = 0;
  gw_job spec{};
  size_t bytes = 0;
  bool done = false;
  gw_job_result result{};
};

}  // namespace
}  // namespace gwi

using namespace gwi;

struct gw_server {
  size_t budget = 0, in_use = 0;
  int slots = 0;
  bool stopping = false;
  uint64_t next_id = 1;
  std::mutex m;
  std::condition_variable cv_work;   // workers wait for admissible jobs
  std::condition_variable cv_done;   // pollers wait for results
  std::deque<Job*> pending;
  std::map<uint64_t, Job*> jobs;
  std::vector<std::thread> workers;
  int device = 0;
};

namespace {

gw_scgw_options job_options(const gw_job& s) {
  gw_scgw_options o{};
  o.alpha = s.alpha;
  o.tol = s.tol;
  o.itermax = s.itermax;
  o.static_part = s.static_part;
  o.diis_size = s.diis_size;
  o.diis_start = s.diis_start;
  o.n_electrons = s.n_electrons;
  o.mu_lo = s.mu_lo;
  o.mu_hi = s.mu_hi;
  o.mu_tol = s.mu_tol;
  o.diis_kind = s.diis_kind;
  o.method = s.method;
  return o;
}

int run_job(Job* j) {
  const gw_job& s = j->spec;
  const gw_config& c = s.cfg;
  const long long nk = (long long)c.nk[0] * c.nk[1] * c.nk[2];
  const long long nao2 = (long long)c.nao * c.nao;
  const size_t bV = sizeof(gw_c128) * (c.v_packed ? (size_t)packed_pairs((int)nk) : (size_t)(nk * nk)) * c.naux * nao2;
  const size_t bH = sizeof(gw_c128) * nk * nao2;
  const size_t bG = sizeof(gw_c128) * nk * c.ntau * nao2;
  cudaStream_t st = nullptr;
  gw_c128 *V = nullptr, *H = nullptr, *G = nullptr, *S = nullptr, *Ov = nullptr;
  gw_ctx* ctx = nullptr;
  int rc = GW_OK;
  auto cleanup = [&]() {
    if (ctx) gw_destroy(ctx);
    if (st) cudaStreamSynchronize(st);
    for (void* p : {(void*)V, (void*)H, (void*)G, (void*)S, (void*)Ov})
      if (p) cudaFree(p);
    if (st) cudaStreamDestroy(st);
  };
  do {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(GW_ECUDA, "job %llu: cannot create a stream", (unsigned long long)j->id);
      break;
    }
    if (cudaMalloc((void**)&V, bV) != cudaSuccess || cudaMalloc((void**)&H, bH) != cudaSuccess ||
        cudaMalloc((void**)&G, bG) != cudaSuccess || cudaMalloc((void**)&S, bG) != cudaSuccess ||
        (s.S_host && cudaMalloc((void**)&Ov, bH) != cudaSuccess)) {
      rc = fail(GW_ENOMEM, "job %llu: device allocation failed", (unsigned long long)j->id);
      break;
    }
    cudaMemcpyAsync(V, s.V_host, bV, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(H, s.H_host, bH, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(G, s.G0_host, bG, cudaMemcpyHostToDevice, st);
    if ((rc = gw_create(&ctx, &c, st)) != GW_OK) break;
    if ((rc = gw_set_coulomb(ctx, V)) != GW_OK) break;
    if (Ov) {
      cudaMemcpyAsync(Ov, s.S_host, bH, cudaMemcpyHostToDevice, st);
      if ((rc = gw_set_overlap(ctx, Ov)) != GW_OK) break;
    }
    const gw_scgw_options o = job_options(s);
    gw_scgw_result r{};
    rc = gw_scgw(ctx, H, G, S, nullptr, &o, &r);
    if (rc != GW_OK && rc != GW_ENOTCONV) break;
    j->result.iterations = r.iterations;
    j->result.max_abs_dsigma = r.max_abs_dsigma;
    j->result.mu = r.mu;
    if (s.Sigma_out_host) cudaMemcpyAsync(s.Sigma_out_host, S, bG, cudaMemcpyDeviceToHost, st);
    if (s.G_out_host) cudaMemcpyAsync(s.G_out_host, G, bG, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(GW_ECUDA, "job %llu: result copy failed", (unsigned long long)j->id);
      break;
    }
  } while (false);
  cleanup();
  return rc;
}

void worker(gw_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->m);
  while (true) {
    // first pending job (arrival order) that fits the free budget
    Job* pick = nullptr;
    for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it) {
      if ((*it)->bytes <= srv->budget - srv->in_use) {
        pick = *it;
        srv->pending.erase(it);
        break;
      }
    }
    if (!pick) {
      if (srv->stopping) return;
      srv->cv_work.wait(lk);
      continue;
    }
    srv->in_use += pick->bytes;
    pick->result.t_start = now_s();
    lk.unlock();
    const int rc = run_job(pick);
    lk.lock();
    srv->in_use -= pick->bytes;
    pick->result.status = rc;
    pick->result.t_end = now_s();
    pick->done = true;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

size_t gw_job_bytes(const gw_config* cfg) { return cfg ? job_device_bytes(cfg) : 0; }

int gw_server_create(gw_server** out, size_t hbm_budget, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget == 0)
    return fail(GW_EINVAL, "gw_server_create: bad arguments");
  gw_server* s = new gw_server();
  s->budget = hbm_budget;
  s->slots = max_slots;
  cudaGetDevice(&s->device);
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return GW_OK;
}

int gw_server_destroy(gw_server* s) {
  if (!s) return GW_OK;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stopping = true;
    // jobs that were never admitted are dropped
    for (Job* j : s->pending) {
      j->result.status = GW_EINVAL;
      j->done = true;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return GW_OK;
}

int gw_submit(gw_server* s, const gw_job* job, uint64_t* job_id) {
  if (!s || !job || !job_id || !job->H_host || !job->V_host || !job->G0_host || job->itermax < 1)
    return fail(GW_EINVAL, "gw_submit: bad arguments");
  size_t bytes = job_device_bytes(&job->cfg);
  if (bytes == 0) return fail(GW_EINVAL, "gw_submit: configuration out of range");
  const gw_scgw_options o = job_options(*job), o0{};
  bytes += scgw_device_bytes(&job->cfg, &o) - scgw_device_bytes(&job->cfg, &o0);
  if (bytes > s->budget)
    return fail(GW_ENOMEM, "gw_submit: job needs %zu bytes, budget is %zu", bytes, s->budget);
  Job* j = new Job();
  j->spec = *job;
  j->bytes = bytes;
  j->result.status = GW_EAGAIN;
  j->result.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->m);
    if (s->stopping) {
      delete j;
      return fail(GW_EINVAL, "gw_submit: server is stopping");
    }
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->pending.push_back(j);
    *job_id = j->id;
  }
  s->cv_work.notify_one();
  return GW_OK;
}

int gw_poll(gw_server* s, uint64_t job_id, gw_job_result* out, int timeout_us) {
  if (!s || !out) return fail(GW_EINVAL, "gw_poll: null argument");
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return fail(GW_EINVAL, "gw_poll: unknown job %llu", (unsigned long long)job_id);
  Job* j = it->second;
  if (!j->done && timeout_us != 0) {
    if (timeout_us < 0)
      s->cv_done.wait(lk, [&] { return j->done; });
    else
      s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return j->done; });
  }
  *out = j->result;
  if (!j->done) return timeout_us == 0 ? GW_EAGAIN : GW_ETIMEOUT;
  return GW_OK;
}

}  // extern "C"
