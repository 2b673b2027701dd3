// Serving: continuous batching of sign solves on one GPU.
//
// A worker thread owns one Solver and runs its rounds back to back. Between
// rounds it admits queued requests (first come first served) while their
// predicted footprints fit the memory budget and the number on the GPU stays
// below max_active; an admitted request joins the next round of the entry
// stage beside those already in flight, and leaves the round it stops in.
// Submission (copy, validation, footprint statistics) runs on the
// submitting thread with the server's upload stream, so the worker never
// waits for it. Per-matrix arithmetic is that of a lone solve, so a result
// does not depend on the requests it shared rounds with.
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

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sign_server_s {
  sign_server_opts o;
  int device = 0;
  cudaStream_t stream = nullptr, upload = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;  // every ticket not yet taken
  std::unordered_map<int, Request *> by_mat;                    // solver id -> request on the GPU
  uint64_t next_ticket = 1;
  bool stop = false;
  sign_server_stats st{};

  void serve();
  void finish(Request *r, const MatState *ms, int status);
};

// Marks a request done (caller holds mu) and releases its reservation.
void sign_server_s::finish(Request *r, const MatState *ms, int status) {
  r->info.status = status;
  if (ms) {
    r->info.iters = ms->k;
    r->info.resid = ms->resid;
    r->info.count = ms->trace_count;
  }
  r->info.nnz_final = r->h->has_result ? r->h->result.nnz : 0;
  r->t.t_done = now_s();
  r->state = RQ_DONE;
  st.active--;
  st.completed++;
  st.reserved = st.active > 0 ? std::max(0.0, st.reserved - r->t.footprint) : 0.0;
}

void sign_server_s::serve() {
  cudaSetDevice(device);
  auto fresh = [&] {
    auto sv = std::make_unique<Solver>();
    sv->s = stream;
    sv->o = o.solve;
    return sv;
  };
  std::unique_ptr<Solver> sv = fresh();
  for (;;) {
    std::vector<Request *> adm;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty() || st.active > 0; });
      if (stop && st.active == 0) break;
      while (!stop && !queue.empty()) {
        Request *r = queue.front();
        if (st.active >= o.max_active || st.reserved + r->t.footprint > o.mem_budget) break;
        queue.pop_front();
        r->state = RQ_ACTIVE;
        r->t.t_admit = now_s();
        st.reserved += r->t.footprint;
        st.active++;
        st.admitted++;
        adm.push_back(r);
      }
      st.queued = int64_t(queue.size());
      if (st.active > st.max_active_seen) st.max_active_seen = st.active;
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
        for (size_t i = 0; i < ids.size(); ++i) by_mat[ids[i]] = adm[i];
        adm.clear();
      }
      if (sv->busy()) {
        sv->step();
      } else if (sv->retired.empty()) {
        std::lock_guard<std::mutex> lk(mu);
        if (!by_mat.empty()) throw Error(SIGN_ESTATE, "requests on the GPU but nothing to run");
      }
      std::vector<int> fin = sv->collect();
      if (!fin.empty()) SGN_CUDA(cudaStreamSynchronize(stream));  // results complete
      std::lock_guard<std::mutex> lk(mu);
      st.rounds++;
      for (int id : fin) {
        auto it = by_mat.find(id);
        if (it == by_mat.end()) continue;
        Request *r = it->second;
        by_mat.erase(it);
        r->h->a.rp.release();  // the input is no longer needed
        r->h->a.col.release();
        r->h->a.val.release();
        finish(r, &sv->m[id], sv->m[id].status);
      }
      if (!fin.empty()) cv_done.notify_all();
    } catch (const std::exception &e) {
      // the round failed: every request on the GPU fails with it, and the
      // solver starts over empty
      int status = SIGN_ECUDA;
      if (const Error *er = dynamic_cast<const Error *>(&e)) status = er->status;
      cudaStreamSynchronize(stream);
      cudaGetLastError();
      std::lock_guard<std::mutex> lk(mu);
      for (auto &kv : by_mat) adm.push_back(kv.second);
      for (Request *r : adm) {  // by_mat, and admitted requests the solver never took
        r->h->has_result = false;
        finish(r, nullptr, status);
      }
      by_mat.clear();
      sv = fresh();
      cv_done.notify_all();
    }
  }
}

extern "C" {

double sign_footprint_bytes(int64_t n, int64_t nnz, double delta, double rho, int64_t bw) {
  double w = double(n);
  if (delta > 0.0 && std::isfinite(delta) && std::isfinite(rho)) {
    double band = std::ceil(1.5 * (rho / delta) * (2.0 * double(bw) + 1.0));
    w = std::min(double(n), std::max(32.0, band));
  }
  return 96.0 * double(n) * w + 24.0 * double(nnz);
}

void sign_server_default_opts(sign_server_opts *o) {
  if (!o) return;
  sign_default_opts(&o->solve);
  o->solve.prec = SIGN_PREC_MIXED;
  o->mem_budget = 120e9;
  o->max_active = 1024;
  o->max_queue = 65536;
}

sign_status sign_server_create(const sign_server_opts *o, sign_server_t *out) {
  set_last_error("");
  if (!out) return set_last_error("out is NULL"), SIGN_EINVAL;
  *out = nullptr;
  std::string why;
  if (!o) return set_last_error("opts is NULL"), SIGN_EINVAL;
  if (!check_opts(&o->solve, why)) return set_last_error(why), SIGN_EINVAL;
  if (!(o->mem_budget > 0.0) || o->max_active < 1 || o->max_queue < 1)
    return set_last_error("need mem_budget > 0, max_active >= 1, max_queue >= 1"), SIGN_EINVAL;
  auto S = std::make_unique<sign_server_s>();
  S->o = *o;
  if (cudaGetDevice(&S->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking) != cudaSuccess) {
    if (S->stream) cudaStreamDestroy(S->stream);
    return set_last_error("stream creation failed"), SIGN_ECUDA;
  }
  try {
    S->worker = std::thread([p = S.get()] { p->serve(); });
  } catch (const std::exception &e) {
    cudaStreamDestroy(S->stream);
    cudaStreamDestroy(S->upload);
    return set_last_error(e.what()), SIGN_ENOMEM;
  }
  *out = S.release();
  return SIGN_OK;
}

sign_status sign_server_submit(sign_server_t S, int64_t n, int64_t nnz, const int64_t *rowptr,
                               const int32_t *col, const double *val, int on_device,
                               uint64_t *ticket) {
  if (!S || !ticket) return set_last_error("NULL server or ticket"), SIGN_EINVAL;
  sign_t h = nullptr;
  sign_status st = sign_create(n, nnz, rowptr, col, val, on_device, S->upload, &h);
  if (st != SIGN_OK) return st;  // sign_create has set the message
  double fp = 0.0;
  try {
    DevBuf g;
    GershStats init{0x7FF0000000000000ull, 0ull, 0, 0}, res;
    g.ensure(sizeof(GershStats), S->upload);
    SGN_CUDA(cudaMemcpyAsync(g.p, &init, sizeof(init), cudaMemcpyHostToDevice, S->upload));
    launch_gersh(n, h->a.d_rp(), h->a.d_col(), h->a.d_val(), g.as<GershStats>(), S->upload);
    SGN_CUDA(cudaMemcpyAsync(&res, g.p, sizeof(res), cudaMemcpyDeviceToHost, S->upload));
    SGN_CUDA(cudaStreamSynchronize(S->upload));
    double delta;
    std::memcpy(&delta, &res.min_gap_bits, sizeof(double));
    double rho;
    std::memcpy(&rho, &res.max_rowsum_bits, sizeof(double));
    fp = sign_footprint_bytes(n, nnz, res.nogap ? 0.0 : delta, rho, res.max_bw);
  } catch (const Error &e) {
    sign_destroy(h);
    return set_last_error(e.what()), sign_status(e.status);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->st.submitted++;
  if (S->stop || fp > S->o.mem_budget || int64_t(S->queue.size()) >= S->o.max_queue) {
    S->st.refused++;
    char msg[160];
    if (S->stop)
      std::snprintf(msg, sizeof msg, "server is stopping");
    else if (fp > S->o.mem_budget)
      std::snprintf(msg, sizeof msg, "predicted footprint %.3g bytes exceeds mem_budget %.3g",
                    fp, S->o.mem_budget);
    else
      std::snprintf(msg, sizeof msg, "%d requests already waiting (max_queue)", S->o.max_queue);
    sign_destroy(h);
    set_last_error(msg);
    return S->stop ? SIGN_ESTATE : SIGN_ENOMEM;
  }
  auto r = std::make_unique<Request>();
  r->h = h;
  r->t.t_submit = now_s();
  r->t.footprint = fp;
  *ticket = S->next_ticket++;
  S->queue.push_back(r.get());
  S->st.queued = int64_t(S->queue.size());
  S->reqs[*ticket] = std::move(r);
  S->cv_work.notify_one();
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
  // the worker synchronized its stream before marking the request done, so the
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
  if (S->worker.joinable()) S->worker.join();
  cudaStreamSynchronize(S->stream);
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
  cudaStreamDestroy(S->stream);
  cudaStreamDestroy(S->upload);
  delete S;
}

}  // extern "C"
