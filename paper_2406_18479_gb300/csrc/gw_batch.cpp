// Batched self-energy evaluation of many independent systems (molecules or
// k-meshes of uneven size): one gw_ctx per system, the systems spread over a
// few CUDA streams by predicted cost (longest first onto the least-loaded
// stream), and the whole batch captured once into a CUDA graph whose branches
// run concurrently; later evaluations are one graph launch. In the grouped
// modes the aux Dyson inversions of all systems (the FP64 stage whose one
// launch per system fills few SMs: one block per canonical frequency) run as
// one launch over the ragged list of every system's matrices (one block per
// matrix, largest first), between the two halves of each system's
// evaluation; a system whose aux basis exceeds the blocked kernel's limit
// (800) keeps its own inversion and runs whole in the first half. A
// per-system serial loop and eager concurrent streams are kept for comparison.
//
// Each system computes exactly what a lone gw_sigma_eval computes: the
// branches share no memory and no kernel depends on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "gw_internal.h"

using namespace gwi;

#define GW_TRY_BATCH(x)           \
  do {                            \
    const int _rc = (x);          \
    if (_rc != GW_OK) return _rc; \
  } while (0)

struct gw_batch {
  int n = 0;
  std::vector<gw_config> cfg;
  std::vector<gw_ctx*> ctx;
  std::vector<int> lane;                 // stream index of each system
  std::vector<cudaStream_t> streams;
  cudaStream_t user = nullptr;           // the caller's stream: calls start after and end before it
  cudaStream_t main = nullptr;           // the batch's own origin stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaEvent_t> ev;           // fork event, one join event per stream
  std::vector<const gw_c128*> V;
  std::vector<int> max_chunk;            // largest tau batch within each system's budget share
  // captured graph and the pointers it was captured with
  cudaGraphExec_t exec = nullptr;
  std::vector<const gw_c128*> gG;
  std::vector<gw_c128*> gS;
  int graph_grouped = 0;                 // the captured graph is of the grouped flow
  // grouped inversion: items of every system, split by panel class (n <= 430, n > 430) so that each
  // matrix gets the panel width of its lone inversion, largest first; in device memory
  GjItem* items_dev[2] = {nullptr, nullptr};
  int items_n[2] = {0, 0}, items_maxn[2] = {0, 0};
  double items_flops[2] = {0.0, 0.0};
  std::vector<char> whole;               // systems evaluated whole in the grouped flow (naux > 800)
};

namespace {

double predicted_cost(const gw_config& c) {
  const double nk = (double)c.nk[0] * c.nk[1] * c.nk[2];
  const double nao = c.nao, naux = c.naux;
  // both contractions (Eqs. tilde_P0_tau, sigma_gw) plus the aux Dyson solves
  return nk * nk * c.ntau * (2.0 * naux * nao * nao * nao + naux * naux * nao * nao) +
         nk * c.ntau * naux * naux * naux;
}

std::vector<int> by_cost(const gw_batch* b) {
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int x, int y) { return predicted_cost(b->cfg[x]) > predicted_cost(b->cfg[y]); });
  return order;
}

void assign_lanes(gw_batch* b) {
  std::vector<double> load(b->streams.size(), 0.0);
  b->lane.assign(b->n, 0);
  for (int i : by_cost(b)) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane[i] = l;
    load[l] += predicted_cost(b->cfg[i]);
  }
}

// Systems left at the automatic tau batch get the largest equal batch whose device bytes fit
// their share of the budget. A share is the system's need with every tau node in one batch,
// scaled by one factor for all systems so that the needs add up to the budget (no share
// below 256 MiB).
void fit_tau_batches(gw_batch* b, size_t budget) {
  std::vector<double> need(b->n, 0.0);
  double total = 0.0;
  for (int i = 0; i < b->n; ++i) {
    gw_config t = b->cfg[i];
    t.tau_chunk = t.ntau;
    need[i] = (double)job_device_bytes(&t);
    total += need[i];
  }
  const double scale = total > 0.0 ? std::min(1.0, (double)budget / total) : 1.0;
  b->max_chunk.assign(b->n, 0);
  for (int i = 0; i < b->n; ++i) {
    gw_config& c = b->cfg[i];
    if (c.tau_chunk != 0) {
      b->max_chunk[i] = c.tau_chunk;
      continue;
    }
    const double share = std::max(268435456.0, need[i] * scale);
    int chosen = 1;
    for (int d = 1; d <= c.ntau; ++d) {
      gw_config t = c;
      t.tau_chunk = (c.ntau + d - 1) / d;
      const size_t bytes = job_device_bytes(&t);
      if (bytes != 0 && (double)bytes <= share) {
        chosen = t.tau_chunk;
        break;
      }
    }
    c.tau_chunk = chosen;
    b->max_chunk[i] = chosen;
  }
}

void drop_items(gw_batch* b) {
  for (int c = 0; c < 2; ++c) {
    if (b->items_dev[c]) cudaFree(b->items_dev[c]);
    b->items_dev[c] = nullptr;
    b->items_n[c] = b->items_maxn[c] = 0;
    b->items_flops[c] = 0.0;
  }
}

// the inversion items of every context, by panel class and largest first
int build_items(gw_batch* b) {
  drop_items(b);
  std::vector<GjItem> all;
  b->whole.assign(b->n, 0);
  for (int i = 0; i < b->n; ++i) {
    if (b->cfg[i].naux > kGjBlockedMaxN8)
      b->whole[i] = 1;
    else
      inverse_items(b->ctx[i], &all);
  }
  std::stable_sort(all.begin(), all.end(), [](const GjItem& x, const GjItem& y) { return x.n > y.n; });
  std::vector<GjItem> cls[2];
  for (const GjItem& it : all) cls[it.n > kGjBlockedMaxN16 ? 1 : 0].push_back(it);
  for (int c = 0; c < 2; ++c) {
    if (cls[c].empty()) continue;
    if (cudaMalloc(reinterpret_cast<void**>(&b->items_dev[c]), cls[c].size() * sizeof(GjItem)) != cudaSuccess ||
        cudaMemcpy(b->items_dev[c], cls[c].data(), cls[c].size() * sizeof(GjItem), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      drop_items(b);
      return fail(GW_ENOMEM, "gw_batch: inversion item list");
    }
    b->items_n[c] = (int)cls[c].size();
    for (const GjItem& it : cls[c]) {
      b->items_maxn[c] = std::max(b->items_maxn[c], it.n);
      b->items_flops[c] += 8.0 * (double)it.n * it.n * it.n;
    }
  }
  return GW_OK;
}

void drop_graph(gw_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->gG.clear();
  b->gS.clear();
}

int create_contexts(gw_batch* b) {
  for (int i = 0; i < b->n; ++i) {
    if (b->ctx[i]) gw_destroy(b->ctx[i]);
    b->ctx[i] = nullptr;
    GW_TRY_BATCH(gw_create(&b->ctx[i], &b->cfg[i], b->streams[b->lane[i]]));
    if (b->V[i]) GW_TRY_BATCH(gw_set_coulomb(b->ctx[i], b->V[i]));
  }
  drop_graph(b);
  return build_items(b);
}

// every system on its stream, eager; the streams fork from and join into main
int enqueue_concurrent(gw_batch* b, const gw_c128* const* G, gw_c128* const* S) {
  const int ns = (int)b->streams.size();
  if (cudaEventRecord(b->ev[0], b->main) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: fork record");
  for (int l = 0; l < ns; ++l)
    if (cudaStreamWaitEvent(b->streams[l], b->ev[0], 0) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: fork wait");
  for (int i : by_cost(b)) GW_TRY_BATCH(gw_sigma_eval(b->ctx[i], G[i], S[i]));   // larger systems first
  for (int l = 0; l < ns; ++l) {
    if (cudaEventRecord(b->ev[1 + l], b->streams[l]) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: join record");
    if (cudaStreamWaitEvent(b->main, b->ev[1 + l], 0) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: join wait");
  }
  return GW_OK;
}

int fork_lanes(gw_batch* b) {
  if (cudaEventRecord(b->ev[0], b->main) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: fork record");
  for (cudaStream_t s : b->streams)
    if (cudaStreamWaitEvent(s, b->ev[0], 0) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: fork wait");
  return GW_OK;
}

int join_lanes(gw_batch* b) {
  for (size_t l = 0; l < b->streams.size(); ++l) {
    if (cudaEventRecord(b->ev[1 + l], b->streams[l]) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: join record");
    if (cudaStreamWaitEvent(b->main, b->ev[1 + l], 0) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: join wait");
  }
  return GW_OK;
}

// every system's first half on its stream; all aux Dyson inversions as one launch per panel class
// on main; every system's second half on its stream
int enqueue_grouped(gw_batch* b, const gw_c128* const* G, gw_c128* const* S) {
  GW_TRY_BATCH(fork_lanes(b));
  const std::vector<int> order = by_cost(b);
  for (int i : order)
    GW_TRY_BATCH(b->whole[i] ? gw_sigma_eval(b->ctx[i], G[i], S[i])
                             : sigma_eval_part(b->ctx[i], reinterpret_cast<const double2*>(G[i]),
                                               reinterpret_cast<double2*>(S[i]), 0));
  GW_TRY_BATCH(join_lanes(b));
  for (int c = 0; c < 2; ++c)
    GW_TRY_BATCH(batched_inverse_group_fp64(b->items_dev[c], b->items_n[c], b->items_maxn[c], b->items_flops[c],
                                            b->main));
  GW_TRY_BATCH(fork_lanes(b));
  for (int i : order)
    if (!b->whole[i])
      GW_TRY_BATCH(sigma_eval_part(b->ctx[i], reinterpret_cast<const double2*>(G[i]), reinterpret_cast<double2*>(S[i]), 1));
  return join_lanes(b);
}

// one system after another, each waiting for the previous one
int enqueue_serial(gw_batch* b, const gw_c128* const* G, gw_c128* const* S) {
  cudaStream_t prev = b->main;
  for (int i = 0; i < b->n; ++i) {
    cudaStream_t s = b->streams[b->lane[i]];
    if (cudaEventRecord(b->ev[0], prev) != cudaSuccess || cudaStreamWaitEvent(s, b->ev[0], 0) != cudaSuccess)
      return fail(GW_ECUDA, "gw_batch: serial chaining");
    GW_TRY_BATCH(gw_sigma_eval(b->ctx[i], G[i], S[i]));
    prev = s;
  }
  if (cudaEventRecord(b->ev[0], prev) != cudaSuccess || cudaStreamWaitEvent(b->main, b->ev[0], 0) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch: serial join");
  return GW_OK;
}

int capture(gw_batch* b, const gw_c128* const* G, gw_c128* const* S, bool grouped) {
  drop_graph(b);
  if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch: begin capture failed");
  const int rc = grouped ? enqueue_grouped(b, G, S) : enqueue_concurrent(b, G, S);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->main, &graph);
  if (rc != GW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess || !graph) return fail(GW_ECUDA, "gw_batch: capture failed: %s", cudaGetErrorString(e));
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->exec = nullptr;
    return fail(GW_ECUDA, "gw_batch: instantiate failed: %s", cudaGetErrorString(ei));
  }
  b->gG.assign(G, G + b->n);
  b->gS.assign(S, S + b->n);
  b->graph_grouped = grouped ? 1 : 0;
  return GW_OK;
}

// Replays the captured graph; (re)captures it when the buffers differ from the captured ones.
// The first evaluation after (re)creating the contexts runs uncaptured: one-time kernel
// attribute and tensor-map setup happen outside the capture, and that call's results come
// from it; the graph serves the calls that follow.
int graph_eval(gw_batch* b, const gw_c128* const* G, gw_c128* const* S, bool grouped) {
  const bool same = b->exec && b->graph_grouped == (grouped ? 1 : 0) && std::equal(b->gG.begin(), b->gG.end(), G) &&
                    std::equal(b->gS.begin(), b->gS.end(), S);
  if (!same) {
    const bool first = !b->exec;
    if (first) GW_TRY_BATCH(grouped ? enqueue_grouped(b, G, S) : enqueue_concurrent(b, G, S));
    GW_TRY_BATCH(capture(b, G, S, grouped));
    if (first) return GW_OK;
  }
  if (cudaGraphLaunch(b->exec, b->main) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: graph launch failed");
  return GW_OK;
}

// orders the batch's streams after the work already queued on the caller's stream
int fork_from_user(gw_batch* b, bool lanes) {
  if (cudaEventRecord(b->ev_in, b->user) != cudaSuccess || cudaStreamWaitEvent(b->main, b->ev_in, 0) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch: fork from the caller's stream");
  if (lanes)
    for (cudaStream_t s : b->streams)
      if (cudaStreamWaitEvent(s, b->ev_in, 0) != cudaSuccess) return fail(GW_ECUDA, "gw_batch: fork");
  return GW_OK;
}

int join_to_user(gw_batch* b) {
  if (cudaEventRecord(b->ev_out, b->main) != cudaSuccess || cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch: join into the caller's stream");
  return GW_OK;
}

bool all_set(const gw_batch* b, const gw_c128* const* G, gw_c128* const* S) {
  for (int i = 0; i < b->n; ++i)
    if (!G[i] || !S[i] || !b->V[i]) return false;
  return true;
}

}  // namespace

extern "C" {

int gw_batch_create(gw_batch** out, const gw_config* cfgs, int n, int max_streams, size_t hbm_budget,
                    void* cuda_stream) {
  if (!out || !cfgs || n < 1 || n > 4096 || max_streams < 1 || max_streams > 64)
    return fail(GW_EINVAL, "gw_batch_create: bad arguments");
  *out = nullptr;
  gw_batch* b = new gw_batch();
  b->n = n;
  b->cfg.assign(cfgs, cfgs + n);
  b->ctx.assign(n, nullptr);
  b->V.assign(n, nullptr);
  b->user = (cudaStream_t)cuda_stream;
  const int ns = std::min(max_streams, n);
  b->streams.assign(ns, nullptr);
  b->ev.assign(1 + ns, nullptr);
  int rc = GW_OK;
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    rc = fail(GW_ECUDA, "gw_batch_create: stream or event");
  for (int l = 0; l < ns && rc == GW_OK; ++l)
    if (cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking) != cudaSuccess)
      rc = fail(GW_ECUDA, "gw_batch_create: stream");
  for (auto& e : b->ev)
    if (rc == GW_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      rc = fail(GW_ECUDA, "gw_batch_create: event");
  if (rc == GW_OK) {
    assign_lanes(b);
    fit_tau_batches(b, hbm_budget ? hbm_budget : (size_t)128 << 30);
    rc = create_contexts(b);
  }
  if (rc != GW_OK) {
    gw_batch_destroy(b);
    return rc;
  }
  *out = b;
  return GW_OK;
}

int gw_batch_destroy(gw_batch* b) {
  if (!b) return GW_OK;
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  if (b->main) cudaStreamSynchronize(b->main);
  drop_graph(b);
  drop_items(b);
  for (gw_ctx* c : b->ctx)
    if (c) gw_destroy(c);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  delete b;
  return GW_OK;
}

int gw_batch_set_coulomb(gw_batch* b, const gw_c128* const* V_dev) {
  if (!b || !V_dev) return fail(GW_EINVAL, "gw_batch_set_coulomb: null argument");
  for (int i = 0; i < b->n; ++i)
    if (!V_dev[i]) return fail(GW_EINVAL, "gw_batch_set_coulomb: system %d has no V", i);
  GW_TRY_BATCH(fork_from_user(b, true));
  for (int i = 0; i < b->n; ++i) {
    b->V[i] = V_dev[i];
    GW_TRY_BATCH(gw_set_coulomb(b->ctx[i], V_dev[i]));
  }
  drop_graph(b);
  return GW_OK;
}

int gw_batch_sigma_eval(gw_batch* b, const gw_c128* const* G_dev, gw_c128* const* Sig_dev, int mode) {
  if (!b || !G_dev || !Sig_dev) return fail(GW_EINVAL, "gw_batch_sigma_eval: null argument");
  if (!all_set(b, G_dev, Sig_dev)) return fail(GW_EINVAL, "gw_batch_sigma_eval: a system has no V, G or Sigma");
  if (mode < GW_BATCH_SERIAL || mode > GW_BATCH_GROUPED_GRAPH)
    return fail(GW_EINVAL, "gw_batch_sigma_eval: unknown mode %d", mode);
  GW_TRY_BATCH(fork_from_user(b, false));
  if (mode == GW_BATCH_SERIAL)
    GW_TRY_BATCH(enqueue_serial(b, G_dev, Sig_dev));
  else if (mode == GW_BATCH_STREAMS)
    GW_TRY_BATCH(enqueue_concurrent(b, G_dev, Sig_dev));
  else if (mode == GW_BATCH_GROUPED)
    GW_TRY_BATCH(enqueue_grouped(b, G_dev, Sig_dev));
  else
    GW_TRY_BATCH(graph_eval(b, G_dev, Sig_dev, mode == GW_BATCH_GROUPED_GRAPH));
  return join_to_user(b);
}

int gw_batch_autotune(gw_batch* b, const gw_c128* const* G_dev, gw_c128* const* Sig_dev, int* chosen) {
  if (!b || !G_dev || !Sig_dev) return fail(GW_EINVAL, "gw_batch_autotune: null argument");
  if (!all_set(b, G_dev, Sig_dev)) return fail(GW_EINVAL, "gw_batch_autotune: a system has no V, G or Sigma");
  GW_TRY_BATCH(fork_from_user(b, true));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch_autotune: events");
  // device time of the second of two evaluations of system i under cfg (1e30 if cfg does not fit)
  auto time_cfg = [&](int i, const gw_config& cfg, float* ms) -> int {
    *ms = 1e30f;
    cudaStream_t s = b->streams[b->lane[i]];
    gw_ctx* ctx = nullptr;
    if (gw_create(&ctx, &cfg, s) != GW_OK) return GW_OK;   // a candidate that does not fit is skipped
    if (gw_set_coulomb(ctx, b->V[i]) == GW_OK && gw_sigma_eval(ctx, G_dev[i], Sig_dev[i]) == GW_OK &&
        cudaEventRecord(e0, s) == cudaSuccess && gw_sigma_eval(ctx, G_dev[i], Sig_dev[i]) == GW_OK &&
        cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
      cudaEventElapsedTime(ms, e0, e1);
    const int sync_rc = gw_synchronize(ctx);
    gw_destroy(ctx);
    return sync_rc;
  };
  // systems of one shape (sizes, precision, V layout, budget share) share one tuning
  auto same_shape = [&](int i, int j) {
    const gw_config &x = b->cfg[i], &y = b->cfg[j];
    return std::equal(x.nk, x.nk + 3, y.nk) && x.nao == y.nao && x.naux == y.naux && x.ntau == y.ntau &&
           x.precision == y.precision && x.v_slices == y.v_slices && x.v_packed == y.v_packed &&
           x.slice_pass == y.slice_pass && b->max_chunk[i] == b->max_chunk[j];
  };
  std::vector<int> done;
  int rc = GW_OK;
  for (int i = 0; i < b->n && rc == GW_OK; ++i) {
    bool reused = false;
    for (int j : done)
      if (same_shape(i, j)) {
        b->cfg[i].tau_chunk = b->cfg[j].tau_chunk;
        b->cfg[i].tile_n = b->cfg[j].tile_n;
        reused = true;
        break;
      }
    if (!reused) {
      // tau batch: equal batches of ntau / {1, 2, 3, 4, 6, 8} nodes within the system's budget share
      const int T = b->cfg[i].ntau;
      std::vector<int> cand;
      for (int d : {1, 2, 3, 4, 6, 8}) {
        const int c = (T + d - 1) / d;
        if (c <= b->max_chunk[i] && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
      }
      if (cand.empty()) cand.push_back(b->max_chunk[i]);
      float best_ms = 1e30f;
      gw_config best = b->cfg[i];
      for (int c : cand) {
        gw_config cfg = b->cfg[i];
        cfg.tau_chunk = c;
        float ms;
        if ((rc = time_cfg(i, cfg, &ms)) != GW_OK) break;
        if (ms < best_ms) best_ms = ms, best = cfg;
      }
      // then the tile width of the free-width GEMMs (mixed precisions), at that tau batch
      if (rc == GW_OK && b->cfg[i].precision != GW_FP64) {
        for (int w : {0, 56, 72, 80}) {
          if (w == best.tile_n) continue;
          gw_config cfg = best;
          cfg.tile_n = w;
          float ms;
          if ((rc = time_cfg(i, cfg, &ms)) != GW_OK) break;
          if (ms < best_ms) best_ms = ms, best = cfg;
        }
      }
      b->cfg[i].tau_chunk = best.tau_chunk;
      b->cfg[i].tile_n = best.tile_n;
      done.push_back(i);
    }
    if (chosen) chosen[i] = b->cfg[i].tau_chunk;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == GW_OK) rc = create_contexts(b);
  return rc;
}

int gw_batch_tuned(const gw_batch* b, int i, int* tau_chunk, int* tile_n) {
  if (!b || i < 0 || i >= b->n) return fail(GW_EINVAL, "gw_batch_tuned: no system %d", i);
  if (tau_chunk) *tau_chunk = b->cfg[i].tau_chunk;
  if (tile_n) *tile_n = b->cfg[i].tile_n;
  return GW_OK;
}

int gw_batch_synchronize(gw_batch* b) {
  if (!b) return fail(GW_EINVAL, "gw_batch_synchronize: null argument");
  if (cudaStreamSynchronize(b->main) != cudaSuccess || cudaStreamSynchronize(b->user) != cudaSuccess)
    return fail(GW_ECUDA, "gw_batch_synchronize");
  for (gw_ctx* c : b->ctx) GW_TRY_BATCH(gw_synchronize(c));
  return GW_OK;
}

}  // extern "C"
