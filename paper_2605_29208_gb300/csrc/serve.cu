// Request server with continuous batching (host runtime around the kernels).
//
// Threads: one dispatcher and n_slots slot workers.  The dispatcher admits
// requests in arrival order: when a slot is idle and the oldest pending
// request fits the remaining device-memory budget, it takes that request and
// every later pending request with the same batching key (kind, family, N,
// dim, iterations) that still fits, up to max_batch, and hands the group to
// the slot.  The slot packs the group into one ragged batch with one model
// per request (model_id = position in the group) and runs it on its own
// context and non-blocking stream; several slots run at once, so batches
// admitted later overlap the ones already on the device.  A slot caches its
// models (M = max_batch, one per key), statistics, plan and buffers, so a
// warm slot allocates no device memory.  Each model's arithmetic depends
// only on its own sequences (per-sequence recursions, per-model fixed-order
// reductions), so a request gives the same result alone and in a mix, up to
// the float32 summation order of the recursions.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

using Clock = std::chrono::steady_clock;

namespace hmm {
namespace {

struct ServeReq {
  uint64_t ticket = 0;
  int kind = 0, family = 0, N = 0, D = 1, n_iter = 0;
  int64_t T = 0;
  size_t bytes = 0;
  std::vector<double> params;
  std::vector<float> values;
  // results
  hmm_status status = HMM_OK;
  std::string error;
  double loglik = 0.0, score = 0.0;
  std::vector<int32_t> path;
  std::vector<float> gamma;
  std::vector<double> out_params, trace;
  Clock::time_point t_submit, t_done;
  bool done = false, running = false;
};

std::string key_of(const ServeReq* r) {
  return std::to_string(r->kind) + "/" + std::to_string(r->family) + "/" + std::to_string(r->N) + "/" +
         std::to_string(r->D) + "/" + std::to_string(r->kind == HMM_REQ_FIT ? r->n_iter : 0);
}
std::string model_key(const ServeReq* r) {
  return std::to_string(r->family) + "/" + std::to_string(r->N) + "/" + std::to_string(r->D);
}

// Host staging that only grows.  Pageable on purpose: cudaMallocHost /
// cudaFreeHost synchronise the whole device, which would make one slot's
// growth wait for every other slot's kernels; the copies from and to pageable
// memory only block the calling slot thread.
struct Staging {
  std::vector<char> buf;
  void* p = nullptr;
  void ensure(size_t n) {
    if (n <= buf.size()) return;
    buf.resize(std::max(n, 2 * buf.size()));
    p = buf.data();
  }
  template <class T>
  T* as() {
    return reinterpret_cast<T*>(p);
  }
};

struct Slot {
  int index = 0;
  hmm_ctx ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::thread th;
  std::vector<ServeReq*> work;
  size_t bytes = 0;
  bool busy = false;
  std::map<std::string, hmm_model> models;
  std::map<std::string, hmm_stats> stats;
  hmm_plan plan = nullptr;
  DevBuf values, offsets, model_id, loglik, score, path, gamma;
  Staging h_in, h_out;
};

}  // namespace
}  // namespace hmm

struct hmm_server_s {
  hmm_ctx owner = nullptr;
  int device = 0;
  int n_slots = 4, max_batch = 16;
  size_t max_queue = 4096, budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv_dispatch, cv_slot, cv_done;
  std::deque<hmm::ServeReq*> queue;
  std::map<uint64_t, hmm::ServeReq*> reqs;
  std::vector<hmm::Slot*> slots;
  std::thread dispatcher;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<double> lat_ms;
  uint64_t submitted = 0, completed = 0, batches = 0;
  double busy_s = 0.0;          // summed slot time spent running batches
  int running = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace hmm {
namespace {

int padded(int n) {
  int p = 2;
  while (p < n) p <<= 1;
  return p;
}

// Device-memory footprint of one request (admission estimate): observations,
// recursion rows, occupancies, backpointers and its model's tables.
size_t footprint(const ServeReq* r) {
  const size_t NP = (size_t)padded(r->N), T = (size_t)std::max<int64_t>(r->T, 1);
  const size_t P = (size_t)std::max(1, hmm_family_param_count(r->family, r->D));
  const size_t od = r->family == HMM_DISCRETE ? 1 : (size_t)r->D;
  return T * (4 * od + 16 * NP + 4 * (size_t)r->N + 2 * NP + 32) + NP * NP * 40 + NP * P * 16 + 4096;
}

void run_batch(hmm_server s, Slot* sl, std::vector<ServeReq*>& group) {
  const ServeReq* r0 = group[0];
  const int K = (int)group.size(), MB = s->max_batch;
  const int kind = r0->kind, N = r0->N, D = r0->D;
  const int OD = r0->family == HMM_DISCRETE ? 1 : D;   // values per step
  HMM_CUDA(cudaSetDevice(s->device));
  // the slot's model for this family / N / dim (M = max_batch, unused models
  // carry a copy of the last request's parameters and no sequences)
  hmm_model& model = sl->models[model_key(r0)];
  if (!model) {
    std::vector<int32_t> fam(MB, r0->family);
    hmm_status st = hmm_model_create(sl->ctx, MB, N, D, fam.data(), &model);
    if (st != HMM_OK) {
      model = nullptr;
      throw Error{st, hmm_last_error()};
    }
  }
  const int64_t blob1 = hmm_param_blob_size(1, N, D, &r0->family);
  std::vector<double> blob((size_t)blob1 * MB);
  for (int m = 0; m < MB; ++m) {
    const ServeReq* src = group[std::min(m, K - 1)];
    std::memcpy(blob.data() + (size_t)m * blob1, src->params.data(), (size_t)blob1 * 8);
  }
  hmm_status st = hmm_model_set_params(model, blob.data(), (int64_t)blob.size());
  if (st != HMM_OK) throw Error{st, hmm_last_error()};

  // pack the group: values, offsets, model ids (one model per request)
  int64_t TT = 0;
  for (auto* r : group) TT += r->T;
  std::vector<int64_t> off(K + 1, 0);
  std::vector<int32_t> mid(K);
  for (int k = 0; k < K; ++k) {
    off[k + 1] = off[k] + group[k]->T;
    mid[k] = k;
  }
  const size_t vbytes = (size_t)TT * OD * 4;
  sl->h_in.ensure(vbytes + (K + 1) * 8 + K * 4 + 64);
  float* hv = sl->h_in.as<float>();
  for (int k = 0; k < K; ++k)
    std::memcpy(hv + (size_t)off[k] * OD, group[k]->values.data(), group[k]->values.size() * 4);
  sl->values.ensure(std::max<size_t>(vbytes, 16));
  sl->offsets.ensure((K + 1) * 8);
  sl->model_id.ensure(K * 4);
  cudaStream_t strm = sl->stream;
  HMM_CUDA(cudaMemcpyAsync(sl->values.p, hv, vbytes, cudaMemcpyHostToDevice, strm));
  int64_t* ho = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(sl->h_in.p) + ((vbytes + 15) & ~size_t(15)));
  int32_t* hm = reinterpret_cast<int32_t*>(ho + K + 1);
  std::memcpy(ho, off.data(), (K + 1) * 8);
  std::memcpy(hm, mid.data(), K * 4);
  HMM_CUDA(cudaMemcpyAsync(sl->offsets.p, ho, (K + 1) * 8, cudaMemcpyHostToDevice, strm));
  HMM_CUDA(cudaMemcpyAsync(sl->model_id.p, hm, K * 4, cudaMemcpyHostToDevice, strm));
  hmm_batch b;
  b.values = sl->values.as<float>();
  b.offsets = sl->offsets.as<int64_t>();
  b.model_id = sl->model_id.as<int32_t>();
  b.n_seq = K;
  b.total_T = TT;
  b.dim = OD;
  b.plan = nullptr;
  if (!sl->plan) sl->plan = new hmm_plan_s();
  fill_plan(sl->plan, sl->ctx, model, &b, off.data(), mid.data());
  b.plan = sl->plan;

  size_t out_bytes = 0;
  if (kind == HMM_REQ_DECODE) {
    sl->path.ensure(std::max<int64_t>(TT, 1) * 4);
    sl->score.ensure(K * 8);
    st = hmm_viterbi(sl->ctx, model, &b, nullptr, sl->path.as<int32_t>(), sl->score.as<double>(), strm);
    if (st != HMM_OK) throw Error{st, hmm_last_error()};
    out_bytes = (size_t)TT * 4 + K * 8;
    sl->h_out.ensure(out_bytes + 64);
    HMM_CUDA(cudaMemcpyAsync(sl->h_out.p, sl->path.p, (size_t)TT * 4, cudaMemcpyDeviceToHost, strm));
    HMM_CUDA(cudaMemcpyAsync(sl->h_out.as<char>() + (((size_t)TT * 4 + 15) & ~size_t(15)), sl->score.p, K * 8,
                             cudaMemcpyDeviceToHost, strm));
  } else if (kind == HMM_REQ_POSTERIOR) {
    sl->gamma.ensure(std::max<int64_t>(TT, 1) * N * 4);
    sl->loglik.ensure(K * 8);
    st = hmm_forward_backward(sl->ctx, model, &b, nullptr, sl->gamma.as<float>(), nullptr, sl->loglik.as<double>(),
                              strm);
    if (st != HMM_OK) throw Error{st, hmm_last_error()};
    out_bytes = (size_t)TT * N * 4 + K * 8;
    sl->h_out.ensure(out_bytes + 64);
    HMM_CUDA(cudaMemcpyAsync(sl->h_out.p, sl->gamma.p, (size_t)TT * N * 4, cudaMemcpyDeviceToHost, strm));
    HMM_CUDA(cudaMemcpyAsync(sl->h_out.as<char>() + (((size_t)TT * N * 4 + 15) & ~size_t(15)), sl->loglik.p, K * 8,
                             cudaMemcpyDeviceToHost, strm));
  } else {
    hmm_stats& stats = sl->stats[model_key(r0)];
    if (!stats) {
      st = hmm_stats_create(sl->ctx, model, &stats);
      if (st != HMM_OK) {
        stats = nullptr;
        throw Error{st, hmm_last_error()};
      }
    }
    const int iters = r0->n_iter;
    const double* d_trace = fit_async(sl->ctx, model, &b, sl->plan, stats, nullptr, iters, strm);
    const int NP = model->NP, P = model->P;
    const size_t tb = (size_t)std::max(iters, 1) * MB * 8;
    const size_t pb = (size_t)MB * NP * 8, ab = (size_t)MB * NP * NP * 8, thb = (size_t)MB * NP * P * 8;
    out_bytes = tb + pb + ab + thb;
    sl->h_out.ensure(out_bytes + 64);
    char* ob = sl->h_out.as<char>();
    if (iters > 0) HMM_CUDA(cudaMemcpyAsync(ob, d_trace, (size_t)iters * MB * 8, cudaMemcpyDeviceToHost, strm));
    HMM_CUDA(cudaMemcpyAsync(ob + tb, model->pi.p, pb, cudaMemcpyDeviceToHost, strm));
    HMM_CUDA(cudaMemcpyAsync(ob + tb + pb, model->A.p, ab, cudaMemcpyDeviceToHost, strm));
    HMM_CUDA(cudaMemcpyAsync(ob + tb + pb + ab, model->theta.p, thb, cudaMemcpyDeviceToHost, strm));
  }
  HMM_CUDA(cudaStreamSynchronize(strm));
  {
    int dst = 0;
    HMM_CUDA(cudaMemcpy(&dst, sl->ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dst) {
      HMM_CUDA(cudaMemset(sl->ctx->status, 0, sizeof(int)));
      throw Error{(dst & ST_TIMEOUT) ? HMM_E_TIMEOUT : HMM_E_NUMERIC, "device status set during the batch"};
    }
  }
  // scatter results
  const char* ob = sl->h_out.as<char>();
  for (int k = 0; k < K; ++k) {
    ServeReq* r = group[k];
    const int64_t T = r->T, b0 = off[k];
    if (kind == HMM_REQ_DECODE) {
      const int32_t* hp = reinterpret_cast<const int32_t*>(ob);
      r->path.assign(hp + b0, hp + b0 + T);
      r->score = reinterpret_cast<const double*>(ob + (((size_t)TT * 4 + 15) & ~size_t(15)))[k];
    } else if (kind == HMM_REQ_POSTERIOR) {
      const float* hg = reinterpret_cast<const float*>(ob);
      r->gamma.assign(hg + (size_t)b0 * N, hg + (size_t)(b0 + T) * N);
      r->loglik = reinterpret_cast<const double*>(ob + (((size_t)TT * N * 4 + 15) & ~size_t(15)))[k];
    } else {
      const int iters = r->n_iter, NP = model->NP, P = model->P;
      const int pc = hmm_family_param_count(r->family, D);
      const size_t tb = (size_t)std::max(iters, 1) * MB * 8, pb = (size_t)MB * NP * 8, ab = (size_t)MB * NP * NP * 8;
      const double* tr = reinterpret_cast<const double*>(ob);
      r->trace.resize(iters);
      for (int i = 0; i < iters; ++i) r->trace[i] = tr[(size_t)i * MB + k];
      r->loglik = iters > 0 ? r->trace[iters - 1] : 0.0;
      const double* pi = reinterpret_cast<const double*>(ob + tb) + (size_t)k * NP;
      const double* A = reinterpret_cast<const double*>(ob + tb + pb) + (size_t)k * NP * NP;
      const double* th = reinterpret_cast<const double*>(ob + tb + pb + ab) + (size_t)k * NP * P;
      r->out_params.clear();
      for (int j = 0; j < N; ++j) r->out_params.push_back(pi[j]);
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) r->out_params.push_back(A[(size_t)i * NP + j]);
      for (int j = 0; j < N; ++j)
        for (int z = 0; z < pc; ++z) r->out_params.push_back(th[(size_t)j * P + z]);
    }
    r->status = HMM_OK;
  }
}

void slot_main(hmm_server s, Slot* sl) {
  cudaSetDevice(s->device);
  alloc_stream() = sl->stream;   // this slot's buffers grow without device-wide syncs
  for (;;) {
    std::vector<ServeReq*> group;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_slot.wait(lk, [&] { return s->stop || !sl->work.empty(); });
      if (sl->work.empty()) return;   // stopping
      group.swap(sl->work);
    }
    hmm_status bst = HMM_OK;
    std::string msg;
    const auto tb = Clock::now();
    try {
      run_batch(s, sl, group);
    } catch (const Error& e) {
      bst = e.st;
      msg = e.msg;
    } catch (const std::exception& e) {
      bst = HMM_E_ARG;
      msg = e.what();
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const auto now = Clock::now();
      for (auto* r : group) {
        if (bst != HMM_OK) {
          r->status = bst;
          r->error = msg;
        }
        r->done = true;
        r->running = false;
        r->t_done = now;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        ++s->completed;
      }
      s->t_last = now;
      s->busy_s += std::chrono::duration<double>(now - tb).count();
      ++s->batches;
      s->used -= sl->bytes;
      sl->bytes = 0;
      sl->busy = false;
      s->running -= (int)group.size();
    }
    s->cv_dispatch.notify_all();
    s->cv_done.notify_all();
  }
}

void dispatcher_main(hmm_server s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->stop) return;
    Slot* free_slot = nullptr;
    for (auto* sl : s->slots)
      if (!sl->busy) {
        free_slot = sl;
        break;
      }
    bool admitted = false;
    if (free_slot && !s->queue.empty()) {
      ServeReq* head = s->queue.front();
      // the oldest request is admitted first (no overtaking by smaller ones)
      if (s->used + head->bytes <= s->budget || s->used == 0) {
        const std::string key = key_of(head);
        std::vector<ServeReq*> group;
        size_t bytes = 0;
        for (auto it = s->queue.begin(); it != s->queue.end() && (int)group.size() < s->max_batch;) {
          ServeReq* r = *it;
          if (key_of(r) == key && (group.empty() || s->used + bytes + r->bytes <= s->budget)) {
            group.push_back(r);
            bytes += r->bytes;
            r->running = true;
            it = s->queue.erase(it);
          } else {
            ++it;
          }
        }
        s->used += bytes;
        s->running += (int)group.size();
        free_slot->bytes = bytes;
        free_slot->busy = true;
        free_slot->work = std::move(group);
        admitted = true;
        s->cv_slot.notify_all();
      }
    }
    if (!admitted) s->cv_dispatch.wait(lk);
  }
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" {

hmm_status hmm_serve_create(hmm_ctx ctx, const hmm_serve_opts* opts, hmm_server* out) {
  try {
    HMM_REQUIRE(ctx && out, "NULL argument");
    *out = nullptr;
    auto* s = new hmm_server_s();
    s->owner = ctx;
    s->device = ctx->device;
    if (opts) {
      if (opts->n_slots > 0) s->n_slots = opts->n_slots;
      if (opts->max_batch > 0) s->max_batch = opts->max_batch;
      if (opts->max_queue > 0) s->max_queue = (size_t)opts->max_queue;
      s->budget = opts->mem_budget;
    }
    try {
      HMM_CUDA(cudaSetDevice(s->device));
      {
        // keep freed stream-ordered memory in this process's pool
        cudaMemPool_t pool;
        HMM_CUDA(cudaDeviceGetDefaultMemPool(&pool, s->device));
        uint64_t thr = UINT64_MAX;
        HMM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
      }
      if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        HMM_CUDA(cudaMemGetInfo(&fr, &tot));
        s->budget = fr / 2;
      }
      for (int i = 0; i < s->n_slots; ++i) {
        auto* sl = new Slot();
        sl->index = i;
        s->slots.push_back(sl);
        hmm_status st = hmm_ctx_create(s->device, 0, &sl->ctx);
        if (st != HMM_OK) throw Error{st, hmm_last_error()};
        HMM_CUDA(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
      }
      for (auto* sl : s->slots) sl->th = std::thread(slot_main, s, sl);
      s->dispatcher = std::thread(dispatcher_main, s);
    } catch (...) {
      hmm_serve_destroy(s);
      throw;
    }
    *out = s;
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HMM_E_ARG;
  }
}

hmm_status hmm_serve_submit(hmm_server s, const hmm_request* q, uint64_t* ticket) {
  try {
    HMM_REQUIRE(s && q && ticket, "NULL argument");
    HMM_REQUIRE(q->kind >= HMM_REQ_DECODE && q->kind <= HMM_REQ_FIT, "unknown request kind");
    HMM_REQUIRE(q->family >= 0 && q->family <= HMM_PARETO, "unknown family");
    HMM_REQUIRE(q->n_states >= 1 && q->n_states <= 1024 && q->dim >= 1, "bad model sizes");
    HMM_REQUIRE(q->T >= 0 && (q->T == 0 || q->values), "bad observations");
    HMM_REQUIRE(q->kind != HMM_REQ_FIT || q->n_iter >= 0, "n_iter must be >= 0");
    const int64_t need = hmm_param_blob_size(1, q->n_states, q->dim, &q->family);
    HMM_REQUIRE(need > 0 && q->params && q->n_params == need, "parameter blob has the wrong size");
    auto* r = new ServeReq();
    r->kind = q->kind;
    r->family = q->family;
    r->N = q->n_states;
    r->D = q->dim;
    r->T = q->T;
    r->n_iter = q->kind == HMM_REQ_FIT ? q->n_iter : 0;
    r->params.assign(q->params, q->params + need);
    // observations: dim values per step (one symbol index for the discrete family)
    r->values.assign(q->values, q->values + (size_t)q->T * (q->family == HMM_DISCRETE ? 1 : q->dim));
    r->bytes = footprint(r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (r->bytes > s->budget) {
        delete r;
        throw Error{HMM_E_NOMEM, "request footprint exceeds the server's memory budget"};
      }
      if (s->queue.size() >= s->max_queue) {
        delete r;
        throw Error{HMM_E_BUSY, "request queue is full"};
      }
      r->ticket = s->next_ticket++;
      r->t_submit = Clock::now();
      if (!s->any) {
        s->t_first = r->t_submit;
        s->any = true;
      }
      s->queue.push_back(r);
      s->reqs[r->ticket] = r;
      ++s->submitted;
      *ticket = r->ticket;
    }
    s->cv_dispatch.notify_all();
    return HMM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::exception& e) {
    set_error(e.what());
    return HMM_E_ARG;
  }
}

static void fill_result(const ServeReq* r, hmm_result* out) {
  out->status = r->status;
  out->kind = r->kind;
  out->T = r->T;
  out->loglik = r->loglik;
  out->score = r->score;
  out->path = r->path.empty() ? nullptr : r->path.data();
  out->gamma = r->gamma.empty() ? nullptr : r->gamma.data();
  out->params = r->out_params.empty() ? nullptr : r->out_params.data();
  out->trace = r->trace.empty() ? nullptr : r->trace.data();
  out->n_iter = r->n_iter;
  out->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  out->error = r->error.c_str();
}

hmm_status hmm_serve_poll(hmm_server s, uint64_t ticket, hmm_result* out) {
  if (!s || !out) {
    set_error("NULL argument");
    return HMM_E_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return HMM_E_ARG;
  }
  if (!it->second->done) return HMM_E_NOTREADY;
  fill_result(it->second, out);
  return HMM_OK;
}

hmm_status hmm_serve_wait(hmm_server s, uint64_t ticket, double timeout_ms, hmm_result* out) {
  if (!s || !out) {
    set_error("NULL argument");
    return HMM_E_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return HMM_E_ARG;
  }
  ServeReq* r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                      [&] { return r->done; });
  if (!ok) {
    set_error("request still pending");
    return HMM_E_TIMEOUT;
  }
  fill_result(r, out);
  return HMM_OK;
}

hmm_status hmm_serve_release(hmm_server s, uint64_t ticket) {
  if (!s) {
    set_error("NULL argument");
    return HMM_E_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return HMM_E_ARG;
  }
  if (!it->second->done) {
    set_error("request still pending");
    return HMM_E_NOTREADY;
  }
  delete it->second;
  s->reqs.erase(it);
  return HMM_OK;
}

hmm_status hmm_serve_stats(hmm_server s, double* h) {
  if (!s || !h) {
    set_error("NULL argument");
    return HMM_E_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)std::ceil(p * v.size()) - (p > 0 ? 1 : 0));
    return v[i];
  };
  double mean = 0.0;
  for (double x : v) mean += x;
  mean = v.empty() ? 0.0 : mean / v.size();
  const double span = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  h[0] = (double)s->submitted;
  h[1] = (double)s->completed;
  h[2] = pct(0.50);
  h[3] = pct(0.99);
  h[4] = mean;
  h[5] = span > 0 ? s->completed / span : 0.0;
  h[6] = (double)s->queue.size();
  h[7] = (double)s->running;
  h[8] = (double)s->batches;
  h[9] = span > 0 ? s->busy_s / (span * s->n_slots) : 0.0;
  return HMM_OK;
}

hmm_status hmm_serve_destroy(hmm_server s) {
  if (!s) return HMM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto* r : s->queue) r->running = false;
  }
  s->cv_dispatch.notify_all();
  s->cv_slot.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  for (auto* sl : s->slots)
    if (sl->th.joinable()) sl->th.join();
  cudaSetDevice(s->device);
  for (auto* sl : s->slots) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    alloc_stream() = sl->stream;
    for (auto& kv : sl->stats) hmm_stats_destroy(kv.second);
    for (auto& kv : sl->models) hmm_model_destroy(kv.second);
    if (sl->plan) destroy_plan(sl->plan);
    for (auto* b : {&sl->values, &sl->offsets, &sl->model_id, &sl->loglik, &sl->score, &sl->path, &sl->gamma})
      b->release();
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    alloc_stream() = nullptr;
    if (sl->ctx) hmm_ctx_destroy(sl->ctx);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return HMM_OK;
}

}  // extern "C"
