// C ABI of the filtered Newton-Schulz sign solver: handles, batch solves,
// results. The round loop itself is in solver_core.cuh.
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "solver_core.cuh"

namespace {
thread_local std::string g_err;
}  // namespace

namespace sgn {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace sgn

namespace {

sign_status fail(int status, const std::string &msg) {
  g_err = msg;
  return sign_status(status);
}

bool valid_opts(const sign_opts *o, std::string &why) {
  if (!o) return why = "opts is NULL", false;
  if (!(o->tol >= 0.0)) return why = "tol must be >= 0", false;
  if (o->filter < 0 || o->filter > 2) return why = "unknown filter", false;
  if (o->dense_frac < 0.0) return why = "dense_frac < 0", false;
  if (o->prec < 0 || o->prec > 1) return why = "unknown precision", false;
  if (o->max_iter < 0) return why = "max_iter < 0", false;
  if (!(o->c4 >= 0.0) || !(o->switch_resid >= 0.0) || !(o->fp32_until > 0.0))
    return why = "c4, switch_resid must be >= 0 and fp32_until > 0", false;
  if (!(o->div_limit > 0.0)) return why = "div_limit must be > 0", false;
  if (o->dense64_min_n < 0) return why = "dense64_min_n < 0", false;
  if (o->fp32_band < 0 || o->fp32_band > 1) return why = "fp32_band must be 0 or 1", false;
  if (o->filter_t < 0 || o->filter_t > 1) return why = "filter_t must be 0 or 1", false;
  if (o->budget_norm < 0 || o->budget_norm > 1) return why = "budget_norm must be 0 or 1", false;
  if (o->method < 0 || o->method > 1) return why = "unknown method", false;
  if (o->method == SIGN_METHOD_NMF && o->prec != SIGN_PREC_FP64)
    return why = "NMF runs in FP64 (prec = SIGN_PREC_FP64)", false;
  if (!(o->band_min_eff >= 0.0)) return why = "band_min_eff must be >= 0", false;
  if (!(o->group_margin == o->group_margin)) return why = "group_margin is NaN", false;
  if (o->pair_rows < 0 || o->pair_rows > 1) return why = "pair_rows must be 0 or 1", false;
  return true;
}

// Schedules chosen by sign_tune_batch, per workload key.
struct TuneKey {
  int prec, filter, method, count_log2, n_log2, deg_log2;
  bool operator<(const TuneKey &o) const {
    return std::tie(prec, filter, method, count_log2, n_log2, deg_log2) <
           std::tie(o.prec, o.filter, o.method, o.count_log2, o.n_log2, o.deg_log2);
  }
};
struct TunedSchedule {
  double band_min_eff, group_margin;
  int pair_rows;
  void apply(sign_opts &o) const {
    o.band_min_eff = band_min_eff;
    o.group_margin = group_margin;
    o.pair_rows = pair_rows;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TunedSchedule> g_tune;

int log2_bin(double v) { return v > 0.0 ? int(std::floor(std::log2(v))) : -1; }

// The device address of pinned, mapped host memory; nullptr for device,
// managed or pageable memory.
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // not an error of the solver: the pointer is just not CUDA's
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Copies between device memory and mapped pinned host memory queued as one
// gather kernel (k_copy_chunks) instead of one cudaMemcpyAsync per array: a
// batch of 512 results is 1536 arrays. The chunk list goes through a pinned
// arena of the calling thread; every user of the arena synchronises its
// stream before returning, so the arena is free at the next call.
thread_local Staging g_xfer_stage;

struct Gather {
  std::vector<CopyChunk> chunks;
  void add(const void *src, void *dst, int64_t bytes) {
    const int64_t step = int64_t(1) << 20;
    for (int64_t o = 0; o < bytes; o += step)
      chunks.push_back(CopyChunk{static_cast<const char *>(src) + o, static_cast<char *>(dst) + o,
                                 std::min(step, bytes - o)});
  }
  size_t staged_bytes() const { return sizeof(CopyChunk) * chunks.size() + 64; }
  // queues the copies on s; the arena must have room for staged_bytes(); list
  // is device scratch that must live until s is synchronised
  void launch(DevBuf &list, cudaStream_t s) {
    if (chunks.empty()) return;
    const size_t bytes = sizeof(CopyChunk) * chunks.size();
    list.ensure(bytes, s);
    SGN_CUDA(cudaMemcpyAsync(list.p, g_xfer_stage.put(chunks.data(), bytes), bytes,
                             cudaMemcpyHostToDevice, s));
    launch_copy_chunks(int(chunks.size()), list.as<CopyChunk>(), s);
  }
};

}  // namespace

namespace sgn {
bool check_opts(const sign_opts *o, std::string &why) { return valid_opts(o, why); }
}  // namespace sgn

extern "C" {

void sign_default_opts(sign_opts *o) {
  if (!o) return;
  o->tol = 1e-8;
  o->filter = SIGN_FILTER_EXACT;
  o->c4 = 1e-4;
  o->switch_resid = 1e-6;
  o->max_iter = 100;
  o->prec = SIGN_PREC_FP64;
  o->fp32_until = 1e-4;
  o->dense_frac = 0.25;
  o->scale_1norm = 1;
  o->div_limit = 1e6;
  o->dense64_min_n = 1024;
  o->fp32_band = 1;
  o->filter_t = 0;
  o->budget_norm = 0;
  o->method = SIGN_METHOD_NSF;
  o->band_min_eff = 0.08;
  o->group_margin = 0.05;
  o->pair_rows = 1;
}

const char *sign_last_error(void) { return g_err.c_str(); }

sign_status sign_create(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                        const double *val, int on_device, void *cuda_stream, sign_t *out) {
  g_err.clear();
  if (!out) return fail(SIGN_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > INT32_MAX || nnz < 0) return fail(SIGN_EINVAL, "need 1 <= n < 2^31, nnz >= 0");
  if (!rowptr || (nnz > 0 && (!col || !val))) return fail(SIGN_EINVAL, "NULL array");
  sign_ctx *h = new (std::nothrow) sign_ctx;
  if (!h) return fail(SIGN_ENOMEM, "host allocation failed");
  try {
    h->n = n;
    h->nnz = nnz;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaStream_t s = h->stream;
    h->a.ensure(n, nnz, s);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SGN_CUDA(cudaMemcpyAsync(h->a.rp.p, rowptr, sizeof(int64_t) * size_t(n + 1), kind, s));
    if (nnz > 0) {
      SGN_CUDA(cudaMemcpyAsync(h->a.col.p, col, sizeof(int32_t) * size_t(nnz), kind, s));
      SGN_CUDA(cudaMemcpyAsync(h->a.val.p, val, sizeof(double) * size_t(nnz), kind, s));
    }
    DevBuf flag;
    flag.ensure(sizeof(int), s);
    SGN_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    launch_validate(n, nnz, h->a.d_rp(), h->a.d_col(), h->a.d_val(), flag.as<int>(), s);
    int hf = 0;
    SGN_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    if (hf) {
      delete h;
      return fail(SIGN_EINVAL, "malformed CSR (rowptr, column order/range or non-finite value)");
    }
  } catch (const Error &e) {
    delete h;
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    delete h;
    return fail(SIGN_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    delete h;
    return fail(SIGN_ECUDA, e.what());
  }
  *out = h;
  return SIGN_OK;
}

sign_status sign_create_batch(int count, const int64_t *n, const int64_t *nnz,
                              const int64_t *const *rowptr, const int32_t *const *col,
                              const double *const *val, int on_device, void *cuda_stream,
                              sign_t *out) {
  g_err.clear();
  if (count < 1 || !n || !nnz || !rowptr || !col || !val || !out)
    return fail(SIGN_EINVAL, "need count >= 1 and non-NULL arrays");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > INT32_MAX || nnz[i] < 0)
      return fail(SIGN_EINVAL, "matrix " + std::to_string(i) + ": need 1 <= n < 2^31, nnz >= 0");
    if (!rowptr[i] || (nnz[i] > 0 && (!col[i] || !val[i])))
      return fail(SIGN_EINVAL, "matrix " + std::to_string(i) + ": NULL array");
  }
  std::vector<std::unique_ptr<sign_ctx>> hs;
  try {
    hs.reserve(size_t(count));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // device arrays, or host arrays that are all pinned and mapped: one
    // gather kernel reads them
    Gather g;
    std::vector<const void *> src(3 * size_t(count), nullptr);
    bool gather = true;
    for (int i = 0; i < count && gather; ++i) {
      auto dev = [&](const void *p) -> const void * { return on_device ? p : mapped_host(p); };
      src[3 * i] = dev(rowptr[i]);
      src[3 * i + 1] = nnz[i] > 0 ? dev(col[i]) : nullptr;
      src[3 * i + 2] = nnz[i] > 0 ? dev(val[i]) : nullptr;
      gather = src[3 * i] && (nnz[i] == 0 || (src[3 * i + 1] && src[3 * i + 2]));
    }
    std::vector<ValidateJob> jobs(static_cast<size_t>(count));
    std::vector<int64_t> row_off(size_t(count) + 1, 0);
    for (int i = 0; i < count; ++i) {  // copies queued back to back, one check, one wait
      hs.emplace_back(new sign_ctx);
      sign_ctx *h = hs.back().get();
      h->n = n[i];
      h->nnz = nnz[i];
      h->stream = s;
      h->a.ensure(n[i], nnz[i], s);
      if (gather) {
        g.add(src[3 * i], h->a.rp.p, int64_t(sizeof(int64_t)) * (n[i] + 1));
        if (nnz[i] > 0) {
          g.add(src[3 * i + 1], h->a.col.p, int64_t(sizeof(int32_t)) * nnz[i]);
          g.add(src[3 * i + 2], h->a.val.p, int64_t(sizeof(double)) * nnz[i]);
        }
      } else {
        SGN_CUDA(cudaMemcpyAsync(h->a.rp.p, rowptr[i], sizeof(int64_t) * size_t(n[i] + 1), kind, s));
        if (nnz[i] > 0) {
          SGN_CUDA(cudaMemcpyAsync(h->a.col.p, col[i], sizeof(int32_t) * size_t(nnz[i]), kind, s));
          SGN_CUDA(cudaMemcpyAsync(h->a.val.p, val[i], sizeof(double) * size_t(nnz[i]), kind, s));
        }
      }
      jobs[size_t(i)] = ValidateJob{n[i], nnz[i], h->a.d_rp(), h->a.d_col(), h->a.d_val()};
      row_off[size_t(i) + 1] = row_off[size_t(i)] + n[i];
    }
    // jobs, row offsets and flags in one device buffer, staged through the arena
    const size_t jb = sizeof(ValidateJob) * size_t(count), rb = sizeof(int64_t) * (size_t(count) + 1);
    const size_t jb_al = (jb + 255) & ~size_t(255), rb_al = (rb + 255) & ~size_t(255);
    DevBuf list, vbuf;
    g_xfer_stage.reserve(g.staged_bytes() + jb + rb + 256);
    g.launch(list, s);
    char *vb = static_cast<char *>(vbuf.ensure(jb_al + rb_al + sizeof(int) * size_t(count), s));
    SGN_CUDA(cudaMemcpyAsync(vb, g_xfer_stage.put(jobs.data(), jb), jb, cudaMemcpyHostToDevice, s));
    SGN_CUDA(cudaMemcpyAsync(vb + jb_al, g_xfer_stage.put(row_off.data(), rb), rb,
                             cudaMemcpyHostToDevice, s));
    int *flags = reinterpret_cast<int *>(vb + jb_al + rb_al);
    SGN_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * size_t(count), s));
    launch_validate_batch(count, reinterpret_cast<const ValidateJob *>(vb),
                          reinterpret_cast<const int64_t *>(vb + jb_al), row_off.back(), flags, s);
    std::vector<int> hf(size_t(count), 0);
    SGN_CUDA(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * size_t(count),
                             cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
      if (hf[size_t(i)])
        return fail(SIGN_EINVAL, "matrix " + std::to_string(i) +
                                     ": malformed CSR (rowptr, column order/range or non-finite value)");
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(SIGN_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(SIGN_ECUDA, e.what());
  }
  for (int i = 0; i < count; ++i) out[i] = hs[size_t(i)].release();
  return SIGN_OK;
}

sign_status sign_solve_batch(sign_t *hs, int count, const sign_opts *o, sign_info *infos) {
  g_err.clear();
  if (!hs || count < 1) return fail(SIGN_EINVAL, "need at least one handle");
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return fail(SIGN_EINVAL, "NULL handle");
  std::string why;
  if (!valid_opts(o, why)) return fail(SIGN_EINVAL, why);
  try {
    Solver sv;
    sv.s = hs[0]->stream;
    sv.o = *o;
    sv.run(hs, count, infos);
    SGN_CUDA(cudaStreamSynchronize(sv.s));
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(SIGN_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(SIGN_ECUDA, e.what());
  }
  return SIGN_OK;
}

sign_status sign_solve(sign_t h, const sign_opts *o, sign_info *info) {
  sign_info local;
  std::memset(&local, 0, sizeof(local));
  sign_info *in = info ? info : &local;
  sign_status st = sign_solve_batch(&h, 1, o, in);
  if (st != SIGN_OK) return st;
  return sign_status(in->status);
}

sign_status sign_get_csr(sign_t h, int64_t *nnz_out, int64_t *row_ptr, int32_t *col, double *val,
                         int on_device) {
  g_err.clear();
  if (!h) return fail(SIGN_EINVAL, "NULL handle");
  if (!h->has_result) return fail(SIGN_ESTATE, "no result: call sign_solve first");
  if (nnz_out) *nnz_out = h->result.nnz;
  if (!row_ptr && !col && !val) return SIGN_OK;
  try {
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t s = h->stream;
    if (row_ptr)
      SGN_CUDA(cudaMemcpyAsync(row_ptr, h->result.rp.p, sizeof(int64_t) * size_t(h->n + 1), kind, s));
    if (col && h->result.nnz > 0)
      SGN_CUDA(cudaMemcpyAsync(col, h->result.col.p, sizeof(int32_t) * size_t(h->result.nnz), kind, s));
    if (val && h->result.nnz > 0)
      SGN_CUDA(cudaMemcpyAsync(val, h->result.val.p, sizeof(double) * size_t(h->result.nnz), kind, s));
    SGN_CUDA(cudaStreamSynchronize(s));
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(SIGN_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(SIGN_ECUDA, e.what());
  }
  return SIGN_OK;
}

sign_status sign_get_csr_batch(int count, const sign_t *hs, int64_t *const *row_ptr,
                               int32_t *const *col, double *const *val, int on_device) {
  g_err.clear();
  if (count < 1 || !hs || !row_ptr || !col || !val)
    return fail(SIGN_EINVAL, "need count >= 1 and non-NULL arrays");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(SIGN_EINVAL, "handle " + std::to_string(i) + " is NULL");
    if (!hs[i]->has_result)
      return fail(SIGN_ESTATE, "handle " + std::to_string(i) + ": no result, call sign_solve first");
    if (!row_ptr[i] || (hs[i]->result.nnz > 0 && (!col[i] || !val[i])))
      return fail(SIGN_EINVAL, "handle " + std::to_string(i) + ": NULL output array");
  }
  try {
    // device arrays, or host arrays that are all pinned and mapped, handles
    // on one stream: one gather kernel writes every result into them
    bool gather = true;
    for (int i = 1; i < count && gather; ++i) gather = hs[i]->stream == hs[0]->stream;
    if (gather) {
      Gather g;
      for (int i = 0; i < count && gather; ++i) {
        const sign_ctx *h = hs[i];
        auto dev = [&](void *p) -> void * { return on_device ? p : mapped_host(p); };
        void *rp = dev(row_ptr[i]);
        void *cl = h->result.nnz > 0 ? dev(col[i]) : nullptr;
        void *vl = h->result.nnz > 0 ? dev(val[i]) : nullptr;
        gather = rp && (h->result.nnz == 0 || (cl && vl));
        if (!gather) break;
        g.add(h->result.rp.p, rp, int64_t(sizeof(int64_t)) * (h->n + 1));
        if (h->result.nnz > 0) {
          g.add(h->result.col.p, cl, int64_t(sizeof(int32_t)) * h->result.nnz);
          g.add(h->result.val.p, vl, int64_t(sizeof(double)) * h->result.nnz);
        }
      }
      if (gather) {
        cudaStream_t s = hs[0]->stream;
        DevBuf list;
        g_xfer_stage.reserve(g.staged_bytes());
        g.launch(list, s);
        SGN_CUDA(cudaStreamSynchronize(s));
        return SIGN_OK;
      }
    }
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    std::vector<cudaStream_t> streams;
    for (int i = 0; i < count; ++i) {
      sign_ctx *h = hs[i];
      cudaStream_t s = h->stream;
      SGN_CUDA(cudaMemcpyAsync(row_ptr[i], h->result.rp.p, sizeof(int64_t) * size_t(h->n + 1), kind,
                               s));
      if (h->result.nnz > 0) {
        SGN_CUDA(cudaMemcpyAsync(col[i], h->result.col.p, sizeof(int32_t) * size_t(h->result.nnz),
                                 kind, s));
        SGN_CUDA(cudaMemcpyAsync(val[i], h->result.val.p, sizeof(double) * size_t(h->result.nnz),
                                 kind, s));
      }
      if (std::find(streams.begin(), streams.end(), s) == streams.end()) streams.push_back(s);
    }
    for (cudaStream_t s : streams) SGN_CUDA(cudaStreamSynchronize(s));
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(SIGN_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(SIGN_ECUDA, e.what());
  }
  return SIGN_OK;
}

sign_status sign_tune_batch(sign_t *hs, int count, const sign_opts *base, int reps, int force,
                            sign_opts *best, sign_tune_report *rep) {
  g_err.clear();
  if (!hs || count < 1 || !best) return fail(SIGN_EINVAL, "need handles and best");
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return fail(SIGN_EINVAL, "NULL handle");
  if (reps < 1) return fail(SIGN_EINVAL, "reps must be >= 1");
  std::string why;
  if (!valid_opts(base, why)) return fail(SIGN_EINVAL, why);
  sign_tune_report local;
  if (!rep) rep = &local;
  std::memset(rep, 0, sizeof(*rep));
  double nsum = 0.0, nnzsum = 0.0;
  for (int i = 0; i < count; ++i) {
    nsum += double(hs[i]->n);
    nnzsum += double(hs[i]->nnz);
  }
  const TuneKey key{base->prec, base->filter, base->method, int(std::ceil(std::log2(double(count)))),
                    log2_bin(nsum / count), log2_bin(nnzsum / nsum)};
  *best = *base;
  if (!force) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      it->second.apply(*best);
      rep->cached = 1;
      return SIGN_OK;
    }
  }
  // best of reps full batch solves, host wall time (the solve waits for its stream)
  auto timed = [&](const sign_opts &o, double &ms) -> sign_status {
    ms = HUGE_VAL;
    for (int r = 0; r < reps; ++r) {
      const auto t0 = std::chrono::steady_clock::now();
      const sign_status st = sign_solve_batch(hs, count, &o, nullptr);
      if (st != SIGN_OK) return st;
      const auto t1 = std::chrono::steady_clock::now();
      ms = std::min(ms, std::chrono::duration<double, std::milli>(t1 - t0).count());
      ++rep->timed;
    }
    return SIGN_OK;
  };
  double cur_ms = 0.0;
  sign_status st = timed(*best, cur_ms);
  if (st != SIGN_OK) return st;
  rep->ms_base = cur_ms;
  // one field at a time; a candidate replaces the current choice only when it
  // is faster by more than 1% (the timing noise of a batch solve)
  auto sweep = [&](auto set, std::initializer_list<double> values) -> sign_status {
    for (double v : values) {
      sign_opts c = *best;
      set(c, v);
      if (std::memcmp(&c, best, sizeof(c)) == 0) continue;
      double ms = 0.0;
      const sign_status s2 = timed(c, ms);
      if (s2 != SIGN_OK) return s2;
      if (ms < 0.99 * cur_ms) {
        *best = c;
        cur_ms = ms;
      }
    }
    return SIGN_OK;
  };
  const bool fp32 = base->prec == SIGN_PREC_MIXED && base->method == SIGN_METHOD_NSF;
  if (fp32 && base->fp32_band) {
    st = sweep([](sign_opts &o, double v) { o.band_min_eff = v; }, {0.02, 0.04, 0.08, 0.16, 0.32});
    if (st != SIGN_OK) return st;
  }
  st = sweep([](sign_opts &o, double v) { o.group_margin = v; }, {-1.0, 0.0, 0.05, 0.15});
  if (st != SIGN_OK) return st;
  if (fp32) {
    st = sweep([](sign_opts &o, double v) { o.pair_rows = int(v); }, {0.0, 1.0});
    if (st != SIGN_OK) return st;
  }
  rep->ms_best = cur_ms;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = TunedSchedule{best->band_min_eff, best->group_margin, best->pair_rows};
  return SIGN_OK;
}

sign_status sign_result_nnz_batch(int count, const sign_t *hs, int64_t *nnz_out) {
  g_err.clear();
  if (count < 1 || !hs || !nnz_out) return fail(SIGN_EINVAL, "need count >= 1 and non-NULL arrays");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(SIGN_EINVAL, "handle " + std::to_string(i) + " is NULL");
    if (!hs[i]->has_result)
      return fail(SIGN_ESTATE, "handle " + std::to_string(i) + ": no result, call sign_solve first");
    nnz_out[i] = hs[i]->result.nnz;
  }
  return SIGN_OK;
}

void sign_destroy_batch(const sign_t *hs, int count) {
  if (!hs || count < 1) return;
  std::vector<cudaStream_t> streams;
  for (int i = 0; i < count; ++i)
    if (hs[i] && std::find(streams.begin(), streams.end(), hs[i]->stream) == streams.end())
      streams.push_back(hs[i]->stream);
  for (cudaStream_t s : streams) cudaStreamSynchronize(s);
  for (int i = 0; i < count; ++i) delete hs[i];
}

void sign_destroy(sign_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}

}  // extern "C"
