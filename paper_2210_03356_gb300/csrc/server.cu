// Serving: continuous batching of sign solves on one GPU.
//
// The server has one or two lanes. Each lane is a worker thread that owns a
// Solver and a CUDA stream and runs the solver's rounds back to back; between
// rounds it admits requests from its own queue (first come first served)
// while the predicted footprints of everything on the GPU fit the memory
// budget and fewer than max_active requests are in flight. An admitted
// request joins the next round of the entry stage beside those already in
// flight, and leaves the round it stops in. With two lanes, requests whose
// iterate is predicted to fill in (no Gershgorin gap, or a predicted quarter
// of the row or more) go to the second lane: their rounds are long (dense
// products, FP64 finish), and on a lane of their own they do not hold up the
// rounds of sparse requests; the two streams overlap on the device.
// Submission (copy, validation, footprint statistics) runs on the submitting
// thread with the server's upload stream, so the workers never wait for it.
// Per-matrix arithmetic is that of a lone solve, so a result does not depend
// on the requests it shared rounds with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "solver_core.cuh"

namespace sgn {
void set_last_error(const std::string &msg);
bool check_opts(const sign_opts *o, std::string &why);
}  // namespace sgn

namespace {

enum { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_DONE = 2 };

struct Request {
  sign_ctx *h = nullptr;  // input copy, then the result; owned until taken
  sign_info info{};
  sign_request_times t{};
  int state = RQ_QUEUED;
};

struct Lane {
  int idx = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::deque<Request *> queue;
  std::unordered_map<int, Request *> by_mat;  // solver id -> request on the GPU
  int64_t active = 0;
  std::deque<double> done_t;  // times of the last 64 completions (the rate estimate)
  // Predicted wait for admission of a request queued now: the requests
  // ahead of it over the lane's recent completion rate; -1 before 8 completions.
  double predicted_wait() const {
    if (done_t.size() < 8) return -1.0;
    const double span = done_t.back() - done_t.front();
    if (!(span > 0.0)) return 0.0;
    return double(queue.size()) * span / double(done_t.size() - 1);
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Predicted entries per row of the filtered iterate (the footprint model).
double predicted_width(int64_t n, double delta, double rho, int64_t bw) {
  if (!(delta > 0.0) || !std::isfinite(delta) || !std::isfinite(rho)) return double(n);
  double band = std::ceil(1.5 * (rho / delta) * (2.0 * double(bw) + 1.0));
  return std::min(double(n), std::max(32.0, band));
}

}  // namespace

struct sign_server_s {
  sign_server_opts o;
  int device = 0;
  cudaStream_t upload = nullptr;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;  // every ticket not yet taken
  uint64_t next_ticket = 1;
  bool stop = false;
  sign_server_stats st{};

  void serve(Lane &L);
  void finish(Lane &L, Request *r, const MatState *ms, int status);
  int64_t queued() const {
    int64_t q = 0;
    for (const auto &l : lanes) q += int64_t(l->queue.size());
    return q;
  }
};

// Marks a request done (caller holds mu) and releases its reservation.
void sign_server_s::finish(Lane &L, Request *r, const MatState *ms, int status) {
  r->info.status = status;
  if (ms) {
    r->info.iters = ms->k;
    r->info.resid = ms->resid;
    r->info.count = ms->trace_count;
  }
  r->info.nnz_final = r->h->has_result ? r->h->result.nnz : 0;
  r->t.t_done = now_s();
  L.done_t.push_back(r->t.t_done);
  if (L.done_t.size() > 64) L.done_t.pop_front();
  r->state = RQ_DONE;
  L.active--;
  st.active--;
  st.completed++;
  st.reserved = st.active > 0 ? std::max(0.0, st.reserved - r->t.footprint) : 0.0;
}

void sign_server_s::serve(Lane &L) {
  cudaSetDevice(device);
  auto fresh = [&] {
    auto sv = std::make_unique<Solver>();
    sv->s = L.stream;
    sv->o = o.solve;
    return sv;
  };
  std::unique_ptr<Solver> sv = fresh();
  for (;;) {
    std::vector<Request *> adm;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop && L.active == 0) break;
        while (!stop && !L.queue.empty()) {
          Request *r = L.queue.front();
          if (st.active >= o.max_active || st.reserved + r->t.footprint > o.mem_budget) break;
          L.queue.pop_front();
          r->state = RQ_ACTIVE;
          r->t.t_admit = now_s();
          st.reserved += r->t.footprint;
          st.active++;
          L.active++;
          st.admitted++;
          adm.push_back(r);
        }
        st.queued = queued();
        if (st.active > st.max_active_seen) st.max_active_seen = st.active;
        if (!adm.empty() || L.active > 0) break;
        // nothing to run: wait for a submission, freed budget or the stop
        cv_work.wait(lk);
      }
      if (adm.empty() && L.active == 0) break;  // stopping
    }
    try {
      if (!adm.empty()) {
        std::vector<sign_t> hs;
        std::vector<sign_info *> infos;
        for (Request *r : adm) {
          hs.push_back(r->h);
          infos.push_back(&r->info);
        }
        std::vector<int> ids = sv->admit(hs, infos, false);
        for (size_t i = 0; i < ids.size(); ++i) L.by_mat[ids[i]] = adm[i];
        adm.clear();
      }
      const bool ran = sv->busy();
      if (ran) {
        sv->step();
      } else if (sv->retired.empty()) {
        std::lock_guard<std::mutex> lk(mu);
        if (!L.by_mat.empty()) throw Error(SIGN_ESTATE, "requests on the GPU but nothing to run");
      }
      std::vector<int> fin = sv->collect();
      if (!fin.empty()) SGN_CUDA(cudaStreamSynchronize(L.stream));  // results complete
      bool freed = false;
      {
        std::lock_guard<std::mutex> lk(mu);
        st.rounds += ran;
        for (int id : fin) {
          auto it = L.by_mat.find(id);
          if (it == L.by_mat.end()) continue;
          Request *r = it->second;
          L.by_mat.erase(it);
          r->h->a.rp.release();  // the input is no longer needed
          r->h->a.col.release();
          r->h->a.val.release();
          finish(L, r, &sv->m[id], sv->m[id].status);
          freed = true;
        }
      }
      if (freed) {
        cv_done.notify_all();
        cv_work.notify_all();  // budget and slots freed: the other lane may admit
      }
    } catch (const std::exception &e) {
      // the round failed: every request of this lane on the GPU fails with it,
      // and the lane's solver starts over empty
      int status = SIGN_ECUDA;
      if (const Error *er = dynamic_cast<const Error *>(&e)) status = er->status;
      cudaStreamSynchronize(L.stream);
      cudaGetLastError();
      {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &kv : L.by_mat) adm.push_back(kv.second);
        for (Request *r : adm) {  // by_mat, and admitted requests the solver never took
          r->h->has_result = false;
          finish(L, r, nullptr, status);
        }
        L.by_mat.clear();
      }
      sv = fresh();
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
}

extern "C" {

double sign_footprint_bytes(int64_t n, int64_t nnz, double delta, double rho, int64_t bw) {
  const double w = predicted_width(n, delta, rho, bw);
  // a predicted fill of a quarter or more takes the dense path: FP64 blocks and
  // digit planes (80 bytes per n^2 entry, the FP32 stage's 28 reuse them)
  const double dense = 4.0 * w >= double(n) ? 80.0 * double(n) * double(n) : 0.0;
  return 96.0 * double(n) * w + dense + 24.0 * double(nnz);
}

void sign_server_default_opts(sign_server_opts *o) {
  if (!o) return;
  sign_default_opts(&o->solve);
  o->solve.prec = SIGN_PREC_MIXED;
  o->mem_budget = 120e9;
  o->max_active = 1024;
  o->max_queue = 65536;
  o->lanes = 2;
  o->max_wait_s = 0.0;
}

static sign_status server_create(const sign_server_opts *o, sign_server_t *out);
static sign_status server_submit(sign_server_t S, int64_t n, int64_t nnz, const int64_t *rowptr,
                                 const int32_t *col, const double *val, int on_device,
                                 uint64_t *ticket);

// No C++ exception crosses the C ABI: allocation failures become SIGN_ENOMEM.
sign_status sign_server_create(const sign_server_opts *o, sign_server_t *out) {
  try {
    return server_create(o, out);
  } catch (const std::bad_alloc &) {
    return set_last_error("host allocation failed"), SIGN_ENOMEM;
  } catch (const std::exception &e) {
    return set_last_error(e.what()), SIGN_ECUDA;
  }
}

sign_status sign_server_submit(sign_server_t S, int64_t n, int64_t nnz, const int64_t *rowptr,
                               const int32_t *col, const double *val, int on_device,
                               uint64_t *ticket) {
  try {
    return server_submit(S, n, nnz, rowptr, col, val, on_device, ticket);
  } catch (const std::bad_alloc &) {
    return set_last_error("host allocation failed"), SIGN_ENOMEM;
  } catch (const std::exception &e) {
    return set_last_error(e.what()), SIGN_ECUDA;
  }
}

static sign_status server_create(const sign_server_opts *o, sign_server_t *out) {
  set_last_error("");
  if (!out) return set_last_error("out is NULL"), SIGN_EINVAL;
  *out = nullptr;
  std::string why;
  if (!o) return set_last_error("opts is NULL"), SIGN_EINVAL;
  if (!check_opts(&o->solve, why)) return set_last_error(why), SIGN_EINVAL;
  if (!(o->mem_budget > 0.0) || o->max_active < 1 || o->max_queue < 1 || o->lanes < 1 ||
      o->lanes > 2 || !(o->max_wait_s >= 0.0))
    return set_last_error("need mem_budget > 0, max_active >= 1, max_queue >= 1, lanes 1 or 2, "
                          "max_wait_s >= 0"),
           SIGN_EINVAL;
  auto S = std::make_unique<sign_server_s>();
  S->o = *o;
  // the sparse lane (and submission) at the highest stream priority: when
  // both lanes have work, the block scheduler serves the short rounds first
  // and the fill-in lane takes the rest of the device
  int least = 0, greatest = 0;
  bool ok = cudaGetDevice(&S->device) == cudaSuccess &&
            cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
            cudaStreamCreateWithPriority(&S->upload, cudaStreamNonBlocking, greatest) ==
                cudaSuccess;
  for (int i = 0; ok && i < o->lanes; ++i) {
    auto L = std::make_unique<Lane>();
    L->idx = i;
    ok = cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking,
                                      i == 0 ? greatest : least) == cudaSuccess;
    if (ok) S->lanes.push_back(std::move(L));
  }
  auto drop_streams = [&] {
    for (auto &L : S->lanes) cudaStreamDestroy(L->stream);
    if (S->upload) cudaStreamDestroy(S->upload);
  };
  if (!ok) {
    drop_streams();
    return set_last_error("stream creation failed"), SIGN_ECUDA;
  }
  try {
    for (auto &L : S->lanes)
      L->worker = std::thread([p = S.get(), l = L.get()] {
        sgn::block_cache_enable(false);  // lane memory goes back to the shared pool
        p->serve(*l);
      });
  } catch (const std::exception &e) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &L : S->lanes)
      if (L->worker.joinable()) L->worker.join();
    drop_streams();
    return set_last_error(e.what()), SIGN_ENOMEM;
  }
  *out = S.release();
  return SIGN_OK;
}

static sign_status server_submit(sign_server_t S, int64_t n, int64_t nnz, const int64_t *rowptr,
                                 const int32_t *col, const double *val, int on_device,
                                 uint64_t *ticket) {
  if (!S || !ticket) return set_last_error("NULL server or ticket"), SIGN_EINVAL;
  auto r = std::make_unique<Request>();  // before the copy: nothing to undo if this fails
  sign_t h = nullptr;
  sign_status st = sign_create(n, nnz, rowptr, col, val, on_device, S->upload, &h);
  if (st != SIGN_OK) return st;  // sign_create has set the message
  double fp = 0.0, width = 0.0;
  try {
    DevBuf g;
    GershStats init{0x7FF0000000000000ull, 0ull, 0, 0}, res;
    g.ensure(sizeof(GershStats), S->upload);
    SGN_CUDA(cudaMemcpyAsync(g.p, &init, sizeof(init), cudaMemcpyHostToDevice, S->upload));
    launch_gersh(n, h->a.d_rp(), h->a.d_col(), h->a.d_val(), g.as<GershStats>(), S->upload);
    SGN_CUDA(cudaMemcpyAsync(&res, g.p, sizeof(res), cudaMemcpyDeviceToHost, S->upload));
    SGN_CUDA(cudaStreamSynchronize(S->upload));
    double delta, rho;
    std::memcpy(&delta, &res.min_gap_bits, sizeof(double));
    std::memcpy(&rho, &res.max_rowsum_bits, sizeof(double));
    if (res.nogap) delta = 0.0;
    width = predicted_width(n, delta, rho, res.max_bw);
    fp = sign_footprint_bytes(n, nnz, delta, rho, res.max_bw);
  } catch (const Error &e) {
    sign_destroy(h);
    return set_last_error(e.what()), sign_status(e.status);
  }
  const int lane = (S->lanes.size() > 1 && 4.0 * width >= double(n)) ? 1 : 0;
  char msg[160] = "";
  sign_status refused = SIGN_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.submitted++;
    const double wait = S->o.max_wait_s > 0.0 ? S->lanes[lane]->predicted_wait() : -1.0;
    const bool full = fp > S->o.mem_budget || S->queued() >= S->o.max_queue;
    const bool late = S->o.max_wait_s > 0.0 && wait > S->o.max_wait_s;
    if (S->stop || full || late) {
      S->st.refused++;
      if (S->stop)
        std::snprintf(msg, sizeof msg, "server is stopping");
      else if (fp > S->o.mem_budget)
        std::snprintf(msg, sizeof msg, "predicted footprint %.3g bytes exceeds mem_budget %.3g",
                      fp, S->o.mem_budget);
      else if (full)
        std::snprintf(msg, sizeof msg, "%d requests already waiting (max_queue)",
                      S->o.max_queue);
      else
        std::snprintf(msg, sizeof msg, "predicted wait %.3g s exceeds max_wait_s %.3g", wait,
                      S->o.max_wait_s);
      refused = S->stop ? SIGN_ESTATE : full ? SIGN_ENOMEM : SIGN_EAGAIN;
    } else {
      r->h = h;
      r->t.t_submit = now_s();
      r->t.footprint = fp;
      r->t.lane = lane;
      const uint64_t t = S->next_ticket++;
      Request *rp = r.get();
      S->reqs[t] = std::move(r);  // owned by the ticket map first, then queued
      try {
        S->lanes[lane]->queue.push_back(rp);
        *ticket = t;
        S->st.queued = S->queued();
      } catch (const std::bad_alloc &) {  // not queued: refused, the copy is freed below
        S->reqs.erase(t);
        S->st.refused++;
        std::snprintf(msg, sizeof msg, "host allocation failed");
        refused = SIGN_ENOMEM;
      }
    }
  }
  if (refused != SIGN_OK) {
    sign_destroy(h);  // synchronizes the upload stream: outside the lock
    set_last_error(msg);
    return refused;
  }
  S->cv_work.notify_all();
  return SIGN_OK;
}

sign_status sign_server_poll(sign_server_t S, uint64_t ticket, int wait_ms, sign_info *info,
                             sign_request_times *times) {
  if (!S) return set_last_error("NULL server"), SIGN_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_last_error("unknown ticket"), SIGN_EINVAL;
  Request *r = it->second.get();
  if (r->state != RQ_DONE && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                        [&] { return r->state == RQ_DONE; });
  if (r->state != RQ_DONE) return SIGN_EAGAIN;
  if (info) {
    info->iters = r->info.iters;
    info->status = r->info.status;
    info->resid = r->info.resid;
    info->nnz_final = r->info.nnz_final;
    info->count = 0;
  }
  if (times) *times = r->t;
  return SIGN_OK;
}

sign_status sign_server_take(sign_server_t S, uint64_t ticket, void *cuda_stream, sign_t *out) {
  if (!S || !out) return set_last_error("NULL server or out"), SIGN_EINVAL;
  *out = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_last_error("unknown ticket"), SIGN_EINVAL;
  if (it->second->state != RQ_DONE) return SIGN_EAGAIN;
  sign_ctx *h = it->second->h;
  // the lane synchronized its stream before marking the request done, so the
  // buffers may move to the caller's stream (which also frees them later)
  cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
  h->stream = cs;
  h->a.rp.s = h->a.col.s = h->a.val.s = cs;
  h->result.rp.s = h->result.col.s = h->result.val.s = cs;
  S->reqs.erase(it);
  *out = h;
  return SIGN_OK;
}

sign_status sign_server_get_stats(sign_server_t S, sign_server_stats *out) {
  if (!S || !out) return set_last_error("NULL server or out"), SIGN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  return SIGN_OK;
}

void sign_server_destroy(sign_server_t S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto &L : S->lanes)
    if (L->worker.joinable()) L->worker.join();
  for (auto &L : S->lanes) cudaStreamSynchronize(L->stream);
  cudaStreamSynchronize(S->upload);
  for (auto &kv : S->reqs) {  // queued or finished, not taken
    sign_ctx *h = kv.second->h;
    h->stream = S->upload;
    h->a.rp.s = h->a.col.s = h->a.val.s = S->upload;
    h->result.rp.s = h->result.col.s = h->result.val.s = S->upload;
    sign_destroy(h);
  }
  S->reqs.clear();
  cudaStreamSynchronize(S->upload);
  for (auto &L : S->lanes) cudaStreamDestroy(L->stream);
  cudaStreamDestroy(S->upload);
  delete S;
}

}  // extern "C"
