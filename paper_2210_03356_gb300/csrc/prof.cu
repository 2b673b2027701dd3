// Launch counting and per-kernel-class timing with CUDA events.
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/sign.h"
#include "common.cuh"

namespace sgn {
namespace {

std::atomic<int64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;

struct Rec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

struct Acc {
  int64_t launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};
Acc g_acc[KC_COUNT];

const char *kNames[KC_COUNT] = {"numeric_square_f64", "numeric_update_f64", "numeric_square_f32",
                                "numeric_update_f32", "bounds",             "scan",
                                "select_hist",        "select_extract",     "select_digits",
                                "select_bound",       "filter",             "reduce",
                                "assemble",           "onenorm",            "dense_tf32x3",
                                "dense_f64_slices", "band_layout",
                                "band_square_f32",    "band_update_f32",
                                "host_setup",
                                "host_check",         "host_decide",        "host_update",
                                "host_filter",        "host_rebuild",       "host_sync_gap"};

// the open sync-gap interval of this thread (its start event and stream)
thread_local cudaEvent_t t_gap = nullptr;
thread_local cudaStream_t t_gap_s = nullptr;

long long now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Folds finished records into the accumulators; caller holds g_mu.
void drain() {
  for (Rec &r : g_recs) {
    float ms = 0.0f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    Acc &a = g_acc[r.cls];
    a.launches += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace

HostScope::HostScope(int c) : cls(c) {
  if (g_prof_on.load(std::memory_order_relaxed)) t0 = now_ns();
}

void HostScope::stop() {
  if (t0 < 0) return;
  double ms = double(now_ns() - t0) * 1e-6;
  t0 = -1;
  std::lock_guard<std::mutex> lk(g_mu);
  g_acc[cls].launches += 1;
  g_acc[cls].ms += ms;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }


void prof_sync_point(cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_gap) g_pool.push_back(t_gap);  // an earlier mark that no scope closed
  t_gap = get_event();
  t_gap_s = s;
  cudaEventRecord(t_gap, s);
}

ProfScope::ProfScope(int c, cudaStream_t st, double f, double b) : cls(c), s(st), flops(f), bytes(b) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_gap && t_gap_s == s) {
    cudaEvent_t g = get_event();
    cudaEventRecord(g, s);
    g_recs.push_back(Rec{KH_SYNC_GAP, t_gap, g, 0.0, 0.0});
    t_gap = nullptr;
  }
  cudaEvent_t e = get_event();
  cudaEventRecord(e, s);
  ev0 = e;
}

ProfScope::~ProfScope() {
  if (!ev0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = get_event();
  cudaEventRecord(e, s);
  g_recs.push_back(Rec{cls, static_cast<cudaEvent_t>(ev0), e, flops, bytes});
  if (g_recs.size() > 4096) drain();
}

// Peak probe of the FMA pipes: every thread runs CHAINS independent
// register-resident chains x <- fma(x, a, b) for `iters` steps, so the pipe,
// not memory or latency, bounds the kernel. 2 * CHAINS * iters flops per
// thread. The result is stored only if it equals a value it cannot reach
// (|a| < 1 keeps every chain bounded), which keeps the arithmetic alive.
constexpr int PROBE_CHAINS = 8;
__device__ double g_probe_sink;

template <typename T>
__global__ void k_fma_probe(int iters) {
  const T a = T(0.5) + T(threadIdx.x & 31) * T(1.0 / 128.0);
  const T b = T(blockIdx.x & 7) * T(1.0 / 64.0);
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = T(c) * T(0.125);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == T(-12345.0)) g_probe_sink = double(s);
}

}  // namespace sgn

extern "C" {

sign_status sign_fma_probe(int fp64, int blocks, int threads, int iters, void *cuda_stream,
                           double *flops_out) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !flops_out)
    return SIGN_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (fp64)
    sgn::k_fma_probe<double><<<blocks, threads, 0, s>>>(iters);
  else
    sgn::k_fma_probe<float><<<blocks, threads, 0, s>>>(iters);
  sgn::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sgn::set_last_error(std::string("sign_fma_probe: ") + cudaGetErrorString(e));
    return SIGN_ECUDA;
  }
  *flops_out = 2.0 * sgn::PROBE_CHAINS * double(iters) * double(blocks) * double(threads);
  return SIGN_OK;
}

int64_t sign_kernel_launches(void) { return sgn::g_launches.load(); }


int sign_prof_enable(int on) { return sgn::g_prof_on.exchange(on ? 1 : 0); }

void sign_prof_reset(void) {
  std::lock_guard<std::mutex> lk(sgn::g_mu);
  sgn::drain();
  for (auto &a : sgn::g_acc) a = sgn::Acc();
}

int sign_prof_read(sign_prof_entry *out, int cap) {
  std::lock_guard<std::mutex> lk(sgn::g_mu);
  sgn::drain();
  int n = 0;
  for (int c = 0; c < sgn::KC_COUNT && n < cap; ++c) {
    if (!out) break;
    sign_prof_entry &e = out[n++];
    std::memset(&e, 0, sizeof(e));
    std::strncpy(e.name, sgn::kNames[c], sizeof(e.name) - 1);
    e.launches = sgn::g_acc[c].launches;
    e.ms = sgn::g_acc[c].ms;
    e.flops = sgn::g_acc[c].flops;
    e.bytes = sgn::g_acc[c].bytes;
  }
  return out ? n : int(sgn::KC_COUNT);
}

}  // extern "C"
