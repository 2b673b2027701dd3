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
                                "dense_f64_slices",
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

}  // namespace sgn

extern "C" {

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
