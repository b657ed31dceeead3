// Request server over a resident base table (ringo_server_*, ringo_result_*).
//
// Each request is select (a set of tags and a time window, the Section 3.3
// table operation) + convert (Section 3.4) + the top-k degrees of the graph
// in both directions.  Worker threads, each with its own CUDA stream, take
// every request that has arrived when they become free (continuous
// batching): the selected rows are counted with one batch of binary
// searches, requests are admitted in arrival order while the estimated
// device bytes of everything in flight stay within the budget, and the
// admitted requests run as one captured wave of the multi-segment pipeline.
// While one worker's wave runs on the device, the next worker already counts,
// admits and launches the requests that arrived meanwhile.  One more worker
// (the small lane) serves only requests of at most cfg.small_rows rows, on a
// stream of the device's highest priority: a small request that arrives
// while a large wave runs starts at once, its kernels' blocks taking SMs as
// the large wave's blocks finish, instead of waiting for the whole wave.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ringo.h"
#include "batch_internal.h"
#include "host_util.h"

using namespace ringo;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int32_t kMaxTopk = 4096;

// The lock, wake-ups and budget count of a server.  Results that keep a
// graph hold a reference: its bytes stay charged until the result is freed,
// possibly after the server is gone.
struct Core {
  std::mutex mu;
  std::condition_variable cv_sched;  // pending work, or memory freed
  std::condition_variable cv_done;   // a request finished
  int64_t inflight = 0;              // device bytes charged to the budget
  int64_t peak = 0;
  void add(int64_t b) {
    inflight += b;
    peak = std::max(peak, inflight);
  }
};

struct KeptGraph {
  char* block = nullptr;
  int64_t bytes = 0;
  int32_t* node_ids = nullptr;
  int64_t* out_off = nullptr;
  int32_t* out_nbr = nullptr;
  int64_t* in_off = nullptr;
  int32_t* in_nbr = nullptr;
};

}  // namespace

struct ringo_result {
  ringo_result_info info;
  std::vector<int32_t> ids[2];
  std::vector<int64_t> degs[2];
  KeptGraph kept;
  std::shared_ptr<Core> core;  // kept graph bytes are returned here
};

namespace {

struct Req {
  uint64_t ticket = 0;
  std::vector<int32_t> tags;
  int64_t t0 = 0, t1 = 0;
  int32_t topk = 0;
  int32_t flags = 0;
  int64_t rows = -1;  // selected rows, once counted
  std::vector<uint32_t> lo, cnt;  // its (tag, window) ranges of clustered rows
  bool counting = false;
  bool done = false;
  int64_t est = 0;  // bytes charged while in flight
  ringo_result* result = nullptr;
};

}  // namespace

struct ringo_server {
  const ringo_base* base = nullptr;
  int device = 0;
  int64_t budget_bytes = 0;
  ringo_server_config cfg{};
  std::shared_ptr<Core> core = std::make_shared<Core>();
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;  // every request not yet claimed by wait
  uint64_t next_ticket = 1;
  bool stop = false;
  int active = 0;
  ringo_server_stats stats{};
  std::vector<std::thread> workers;
};

namespace {

int64_t request_bytes(const Req* r) {
  const uint32_t n = (uint32_t)std::min<int64_t>(r->rows, 0x7FFFFFFF);
  int64_t b = (int64_t)wave_seg_bytes(n, (uint32_t)r->topk);
  if (r->flags & RINGO_SERVE_KEEP_GRAPH) b += (int64_t)wave_seg_output_bytes(n);
  return b;
}

void finish(ringo_server* S, Req* r, int status) {
  r->result->info.status = status;
  r->result->info.t_done_ns = now_ns();
  r->done = true;
  if (status == RINGO_OK) S->stats.completed++;
  else S->stats.failed++;
}

// Counts the selected rows of `batch` (all uncounted, marked counting) and
// keeps each request's ranges for its wave.
int count_rows(ringo_server* S, const std::vector<Req*>& batch, cudaStream_t st,
               std::vector<int64_t>* rows) {
  std::vector<ringo_select> preds(batch.size());
  for (size_t i = 0; i < batch.size(); ++i)
    preds[i] = ringo_select{batch[i]->tags.data(), (int32_t)batch[i]->tags.size(), batch[i]->t0,
                            batch[i]->t1};
  const std::vector<Pair> pairs = make_pairs(preds.data(), (int32_t)preds.size());
  Ranges rg;
  HostScope hs("host:serve_count");
  const int rc = select_ranges(S->base, pairs, st, &rg, true);
  pool_free(rg.block, st);
  rows->assign(batch.size(), 0);
  if (rc != RINGO_OK) return rc;
  for (size_t i = 0; i < pairs.size(); ++i) {
    Req* r = batch[pairs[i].seg];
    (*rows)[pairs[i].seg] += rg.h_cnt[i];
    r->lo.push_back(rg.h_lo[i]);
    r->cnt.push_back(rg.h_cnt[i]);
  }
  return RINGO_OK;
}

// Runs one admitted batch as one wave, with the ranges its requests got
// when they were counted; fills each request's result.
int run_batch(ringo_server* S, const std::vector<Req*>& batch, cudaStream_t st) {
  uint32_t topk = 0;
  const uint32_t nseg = (uint32_t)batch.size();
  std::vector<size_t> first(nseg + 1, 0);
  std::vector<uint32_t> h_lo, h_cnt;
  for (uint32_t i = 0; i < nseg; ++i) {
    topk = std::max(topk, (uint32_t)batch[i]->topk);
    h_lo.insert(h_lo.end(), batch[i]->lo.begin(), batch[i]->lo.end());
    h_cnt.insert(h_cnt.end(), batch[i]->cnt.begin(), batch[i]->cnt.end());
    first[i + 1] = h_lo.size();
  }
  WaveResult w;
  int rc = run_wave(S->base, nullptr, nullptr, h_lo.data(), h_cnt.data(), first, nseg, topk, st,
                    &w);
  int64_t batch_rows = 0;
  for (Req* r : batch) batch_rows += r->rows;
  for (uint32_t j = 0; j < nseg && rc == RINGO_OK; ++j) {
    Req* r = batch[j];
    ringo_result* res = r->result;
    const WaveSeg& g = w.seg[j];
    res->info.nrows = g.res_rows;
    res->info.num_nodes = g.res.V;
    res->info.num_edges = g.res.E;
    res->info.batch_requests = (int32_t)nseg;
    res->info.batch_rows = batch_rows;
    const uint32_t ke = std::min<uint32_t>((uint32_t)r->topk, g.res.V);
    for (int d = 0; d < 2; ++d) {
      const size_t o = ((size_t)j * 2 + d) * topk;
      res->ids[d].assign(w.topk_ids.begin() + o, w.topk_ids.begin() + o + ke);
      res->degs[d].assign(w.topk_degs.begin() + o, w.topk_degs.begin() + o + ke);
    }
    res->info.k_out = res->info.k_in = (int32_t)ke;
    if (r->flags & RINGO_SERVE_KEEP_GRAPH) {
      // copy the graph out of the wave's block into its own allocation
      const uint64_t V = g.res.V, E = g.res.E;
      const uint64_t a_ids = (4 * V + 255) & ~255ull, a_off = (8 * (V + 1) + 255) & ~255ull,
                     a_nbr = (4 * E + 255) & ~255ull;
      KeptGraph& k = res->kept;
      k.bytes = (int64_t)wave_seg_output_bytes(g.res_rows);
      k.block = (char*)pool_alloc(a_ids + 2 * a_off + 2 * a_nbr, st);
      if (!k.block) {
        rc = RINGO_ENOMEM;
        break;
      }
      k.node_ids = (int32_t*)k.block;
      k.out_off = (int64_t*)(k.block + a_ids);
      k.in_off = (int64_t*)(k.block + a_ids + a_off);
      k.out_nbr = (int32_t*)(k.block + a_ids + 2 * a_off);
      k.in_nbr = (int32_t*)(k.block + a_ids + 2 * a_off + a_nbr);
      if (V) cudaMemcpyAsync(k.node_ids, g.node_ids, 4 * V, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(k.out_off, g.out_off, 8 * (V + 1), cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(k.in_off, g.in_off, 8 * (V + 1), cudaMemcpyDeviceToDevice, st);
      if (E) {
        cudaMemcpyAsync(k.out_nbr, g.out_nbr, 4 * E, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(k.in_nbr, g.in_nbr, 4 * E, cudaMemcpyDeviceToDevice, st);
      }
      res->core = S->core;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == RINGO_OK) rc = RINGO_ECUDA;
  pool_free(w.block, st);
  return rc;
}

// Releases a kept graph that was never charged (its batch failed).
void free_kept_locked(ringo_result* r) {
  if (!r->kept.block) return;
  pool_free(r->kept.block, nullptr);
  r->kept = KeptGraph{};
  r->core.reset();
}

// Releases a kept graph and returns its bytes to the budget.
void free_kept(ringo_result* r) {
  if (!r->kept.block) return;
  pool_free(r->kept.block, nullptr);
  cudaStreamSynchronize(nullptr);
  if (r->core) {
    std::lock_guard<std::mutex> lk(r->core->mu);
    r->core->inflight -= r->kept.bytes;
    r->core->cv_sched.notify_all();
  }
  r->kept = KeptGraph{};
  r->core.reset();
}

bool front_admissible(ringo_server* S) {
  if (S->pending.empty()) return false;
  const Req* r = S->pending.front();
  if (r->rows < 0) return false;
  if (r->rows > 0x7FFFFFFF) return true;  // fails at once
  const int64_t b = request_bytes(r);
  return b > S->budget_bytes || S->core->inflight + b <= S->budget_bytes;
}

bool has_uncounted(ringo_server* S) {
  for (Req* r : S->pending)
    if (r->rows < 0 && !r->counting) return true;
  return false;
}

bool is_small(const ringo_server* S, const Req* r) {
  return r->rows >= 0 && r->rows <= S->cfg.small_rows;
}

// A counted small request that fits in the budget now.  The small lane's
// admission below admits the first such request whenever this is true (it
// skips, never stops at, small requests that do not fit), so a woken small
// lane always makes progress or sleeps again.
bool small_admissible(ringo_server* S) {
  for (Req* r : S->pending)
    if (is_small(S, r) && S->core->inflight + request_bytes(r) <= S->budget_bytes) return true;
  return false;
}

// lane 0: the regular workers; lane 1: the small lane (see the top).
void worker_main(ringo_server* S, int lane) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (lane == 1) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest);
  } else {
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  }
  Core& C = *S->core;
  std::unique_lock<std::mutex> lk(C.mu);
  while (true) {
    C.cv_sched.wait(lk, [&] {
      if (S->stop && S->pending.empty()) return true;
      if (has_uncounted(S)) return true;
      if (lane == 1) return small_admissible(S) || S->stop;
      if (front_admissible(S)) return true;
      return S->stop && S->active == 0 && S->pending.front()->rows >= 0;
    });
    if (S->stop && S->pending.empty()) break;
    if (lane == 1 && S->stop && !has_uncounted(S) && !small_admissible(S)) break;
    // 1. count what has arrived
    std::vector<Req*> tocount;
    for (Req* r : S->pending)
      if (r->rows < 0 && !r->counting && tocount.size() < 4096) {
        r->counting = true;
        tocount.push_back(r);
      }
    if (!tocount.empty()) {
      lk.unlock();
      std::vector<int64_t> rows;
      const int rc = count_rows(S, tocount, st, &rows);
      lk.lock();
      for (size_t i = 0; i < tocount.size(); ++i) {
        tocount[i]->counting = false;
        tocount[i]->rows = rc == RINGO_OK ? rows[i] : 0;
        if (rc != RINGO_OK) {
          finish(S, tocount[i], rc);
          S->pending.erase(std::find(S->pending.begin(), S->pending.end(), tocount[i]));
        }
      }
      if (rc != RINGO_OK) C.cv_done.notify_all();
      C.cv_sched.notify_all();
    }
    // 2. admit in arrival order within the budget
    std::vector<Req*> batch;
    int64_t rows = 0, bytes = 0;
    if (lane == 1) {
      for (auto it = S->pending.begin(); it != S->pending.end();) {
        Req* r = *it;
        if (!is_small(S, r)) {
          ++it;
          continue;
        }
        const int64_t b = request_bytes(r);
        if ((int64_t)batch.size() >= S->cfg.max_batch) break;
        if ((!batch.empty() && rows + r->rows > S->cfg.max_batch_rows) ||
            C.inflight + bytes + b > S->budget_bytes) {
          ++it;  // a later small request may still fit
          continue;
        }
        r->est = b;
        r->result->info.t_admit_ns = now_ns();
        batch.push_back(r);
        rows += r->rows;
        bytes += b;
        it = S->pending.erase(it);
      }
      if (!batch.empty()) C.add(bytes);
    } else {
      while (!S->pending.empty()) {
        Req* r = S->pending.front();
        if (r->rows < 0) break;
        if (r->rows > 0x7FFFFFFF) {
          finish(S, r, RINGO_ERANGE);
          S->pending.pop_front();
          C.cv_done.notify_all();
          continue;
        }
        const int64_t b = request_bytes(r);
        if (b > S->budget_bytes) {
          finish(S, r, RINGO_ENOMEM);
          S->pending.pop_front();
          C.cv_done.notify_all();
          continue;
        }
        if (!batch.empty() &&
            ((int64_t)batch.size() >= S->cfg.max_batch || rows + r->rows > S->cfg.max_batch_rows))
          break;
        if (C.inflight + bytes + b > S->budget_bytes) break;
        r->est = b;
        r->result->info.t_admit_ns = now_ns();
        batch.push_back(r);
        rows += r->rows;
        bytes += b;
        S->pending.pop_front();
      }
      if (!batch.empty()) C.add(bytes);
    }
    if (batch.empty()) {
      // stopping, nothing in flight, and the head still does not fit: only
      // kept graphs the caller holds can be in the way, so give up on it
      if (lane == 0 && S->stop && S->active == 0 && !S->pending.empty() &&
          S->pending.front()->rows >= 0 && !front_admissible(S)) {
        finish(S, S->pending.front(), RINGO_EBUSY);
        S->pending.pop_front();
        C.cv_done.notify_all();
      }
      continue;
    }
    S->active++;
    S->stats.batches++;
    S->stats.rows += rows;
    S->stats.max_concurrent_batches = std::max<int64_t>(S->stats.max_concurrent_batches, S->active);
    lk.unlock();
    const int rc = run_batch(S, batch, st);
    lk.lock();
    for (Req* r : batch) {
      // a kept graph stays charged until its result is freed
      const int64_t keep = (rc == RINGO_OK && r->result->kept.block) ? r->result->kept.bytes : 0;
      C.inflight -= r->est - keep;
      if (rc != RINGO_OK) free_kept_locked(r->result);
    }
    for (Req* r : batch) finish(S, r, rc);
    S->active--;
    C.cv_done.notify_all();
    C.cv_sched.notify_all();
  }
  lk.unlock();
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int64_t ringo_clock_ns(void) { return now_ns(); }

int ringo_server_create(const ringo_base* b, int64_t hbm_budget_bytes,
                        const ringo_server_config* cfg, ringo_server** out) {
  if (!out) return RINGO_EINVAL;
  *out = nullptr;
  if (!b || hbm_budget_bytes <= 0) {
    set_error("ringo_server_create: NULL base or budget <= 0");
    return RINGO_EINVAL;
  }
  ringo_server_config c{};
  if (cfg) c = *cfg;
  if (c.workers < 0 || c.max_batch < 0 || c.max_batch_rows < 0) return RINGO_EINVAL;
  if (c.workers == 0) c.workers = 1;
  if (c.max_batch == 0) c.max_batch = 1024;
  if (c.max_batch_rows == 0) c.max_batch_rows = 256ll << 20;
  if (c.small_rows == 0) c.small_rows = 1ll << 21;
  if (c.workers > 16) return RINGO_ERANGE;
  ringo_server* S = new ringo_server();
  S->base = b;
  cudaGetDevice(&S->device);
  S->budget_bytes = hbm_budget_bytes;
  S->cfg = c;
  {
    // hold the budget in the library's device pool (which keeps freed
    // memory), so no request waits on device memory being mapped; skipped
    // when the device cannot hold it all at once
    void* p = pool_alloc((size_t)hbm_budget_bytes, nullptr);
    if (p) {
      pool_free(p, nullptr);
      cudaStreamSynchronize(nullptr);
    }
    cudaGetLastError();
  }
  for (int i = 0; i < c.workers; ++i) S->workers.emplace_back(worker_main, S, 0);
  if (c.small_rows > 0) S->workers.emplace_back(worker_main, S, 1);
  *out = S;
  return RINGO_OK;
}

int ringo_server_submit(ringo_server* S, const ringo_select* pred, int32_t topk, int32_t flags,
                        uint64_t* ticket) {
  if (!S || !pred || !ticket) return RINGO_EINVAL;
  if (int rc = check_preds(pred, 1)) return rc;
  if (topk < 0 || (flags & ~RINGO_SERVE_KEEP_GRAPH)) return RINGO_EINVAL;
  if (topk > kMaxTopk) return RINGO_ERANGE;
  Req* r = new Req();
  r->tags.assign(pred->tags, pred->tags + pred->ntags);
  r->t0 = pred->t0;
  r->t1 = pred->t1;
  r->topk = topk;
  r->flags = flags;
  r->result = new ringo_result();
  memset(&r->result->info, 0, sizeof(r->result->info));
  r->result->info.t_submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(S->core->mu);
    if (S->stop) {
      delete r->result;
      delete r;
      return RINGO_EBUSY;
    }
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    S->stats.submitted++;
  }
  S->core->cv_sched.notify_all();
  *ticket = r->ticket;
  return RINGO_OK;
}

int ringo_server_wait(ringo_server* S, uint64_t ticket, int64_t timeout_us, ringo_result** out) {
  if (!S || !out) return RINGO_EINVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(S->core->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return RINGO_ENOTFOUND;
  Req* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_us < 0) {
    S->core->cv_done.wait(lk, ready);
  } else if (!S->core->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
    return RINGO_ETIMEOUT;
  }
  S->reqs.erase(ticket);
  *out = r->result;
  delete r;
  return RINGO_OK;
}

int ringo_server_get_stats(const ringo_server* S, ringo_server_stats* st) {
  if (!S || !st) return RINGO_EINVAL;
  std::lock_guard<std::mutex> lk(S->core->mu);
  *st = S->stats;
  st->inflight_bytes = S->core->inflight;
  st->max_inflight_bytes = S->core->peak;
  st->pending = (int64_t)S->pending.size();
  return RINGO_OK;
}

void ringo_server_destroy(ringo_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->core->mu);
    S->stop = true;
  }
  S->core->cv_sched.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs) {  // results nobody claimed
    ringo_result_free(kv.second->result);
    delete kv.second;
  }
  delete S;
}

int ringo_result_get_info(const ringo_result* r, ringo_result_info* info) {
  if (!r || !info) return RINGO_EINVAL;
  *info = r->info;
  return RINGO_OK;
}

int ringo_result_topk(const ringo_result* r, int dir, int32_t* h_ids, int64_t* h_degs,
                      int32_t cap, int32_t* n_out) {
  if (!r || !n_out || (dir != RINGO_OUT && dir != RINGO_IN) || cap < 0) return RINGO_EINVAL;
  const size_t n = r->ids[dir].size();
  *n_out = (int32_t)n;
  if ((size_t)cap < n) return RINGO_ERANGE;
  if (n && (!h_ids || !h_degs)) return RINGO_EINVAL;
  if (n) {
    memcpy(h_ids, r->ids[dir].data(), 4 * n);
    memcpy(h_degs, r->degs[dir].data(), 8 * n);
  }
  return RINGO_OK;
}

int ringo_result_copy_graph_to_host(const ringo_result* r, int32_t* h_node_ids, int64_t* h_out_off,
                                    int32_t* h_out_nbr, int64_t* h_in_off, int32_t* h_in_nbr) {
  if (!r) return RINGO_EINVAL;
  if (!r->kept.block) {
    set_error("ringo_result_copy_graph_to_host: the request did not keep its graph");
    return RINGO_EINVAL;
  }
  const size_t V = (size_t)r->info.num_nodes, E = (size_t)r->info.num_edges;
  const KeptGraph& k = r->kept;
  if (h_node_ids && V) RINGO_CUDA_TRY(cudaMemcpy(h_node_ids, k.node_ids, 4 * V, cudaMemcpyDeviceToHost));
  if (h_out_off) RINGO_CUDA_TRY(cudaMemcpy(h_out_off, k.out_off, 8 * (V + 1), cudaMemcpyDeviceToHost));
  if (h_out_nbr && E) RINGO_CUDA_TRY(cudaMemcpy(h_out_nbr, k.out_nbr, 4 * E, cudaMemcpyDeviceToHost));
  if (h_in_off) RINGO_CUDA_TRY(cudaMemcpy(h_in_off, k.in_off, 8 * (V + 1), cudaMemcpyDeviceToHost));
  if (h_in_nbr && E) RINGO_CUDA_TRY(cudaMemcpy(h_in_nbr, k.in_nbr, 4 * E, cudaMemcpyDeviceToHost));
  return RINGO_OK;
}

void ringo_result_free(ringo_result* r) {
  if (!r) return;
  free_kept(r);
  delete r;
}

}  // extern "C"
