// Internal helpers shared by the CUDA translation units of the sign solver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <stdexcept>
#include <string>

namespace sgn {

// Error raised inside the library; converted to a sign_status at the ABI.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define SGN_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::sgn::Error(e_ == cudaErrorMemoryAllocation ? 2 : 5,                           \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

// Every kernel launch of the library goes through this check, which also
// counts it (sign_kernel_launches).
void count_launch();
#define SGN_LAUNCH_CHECK()        \
  do {                            \
    ::sgn::count_launch();        \
    SGN_CUDA(cudaGetLastError()); \
  } while (0)

// Shared-memory row accumulators: rows whose column range fits WARP_W slots
// are handled by one warp; wider rows by one CTA in chunks of CTA_W slots.
constexpr int WARP_W = 1024;
constexpr int WARPS_PER_CTA = 4;
constexpr int CTA_THREADS = 256;
template <typename T> struct CtaW;
template <> struct CtaW<double> { static constexpr int value = 12288; };
template <> struct CtaW<float> { static constexpr int value = 20480; };
// symbolic pass of wide rows: one bitmap covering up to SYM_BITS columns
constexpr int SYM_BITS = 1 << 18;
constexpr int K_BATCH = 256;  // k entries whose B-row ranges are located at once

// Kernel classes timed when profiling is on (sign_prof_enable).
enum KClass {
  KC_NUM_SQUARE_F64, KC_NUM_UPDATE_F64, KC_NUM_SQUARE_F32, KC_NUM_UPDATE_F32, KC_BOUNDS,
  KC_SCAN, KC_SEL_HIST, KC_SEL_EXTRACT, KC_SEL_DIGITS, KC_SELECT, KC_FILTER, KC_REDUCE,
  KC_ASSEMBLE, KC_NORM, KC_DENSE, KC_DENSE64, KC_BAND_LAYOUT, KC_BAND_SQUARE, KC_BAND_UPDATE,
  // host wall time of driver phases (synchronizations included)
  KH_SETUP, KH_CHECK, KH_DECIDE, KH_UPDATE, KH_FILTER, KH_REBUILD,
  // device time from the end of the work before a host synchronization to the
  // start of the next timed launch: the GPU's idle time around the wait
  KH_SYNC_GAP, KC_COUNT
};
// Records CUDA events around the enclosed launches on stream s (no-op when
// profiling is off); flops and bytes are the algorithmic work they do.
struct ProfScope {
  int cls;
  cudaStream_t s;
  double flops, bytes;
  void *ev0 = nullptr;
  ProfScope(int c, cudaStream_t st, double f = 0.0, double b = 0.0);
  ~ProfScope();
};

// Marks a host synchronization of stream s (profiling only): the next
// ProfScope on s closes a KH_SYNC_GAP interval that starts here.
void prof_sync_point(cudaStream_t s);

// The library's stream-ordered memory pool on the current device: it keeps
// freed memory for reuse (release threshold = unlimited), so repeated solves
// do not map and unmap device memory at every synchronization.
cudaMemPool_t lib_pool();

// Host wall time of the enclosed driver code, when profiling is on.
struct HostScope {
  int cls;
  long long t0 = -1;
  explicit HostScope(int c);
  void stop();  // records now; later calls and the destructor do nothing
  ~HostScope() { stop(); }
};

// Grow-only device buffer, allocated stream-ordered from lib_pool().
// Device blocks of the library pool, cached per host thread. A freed block is
// parked with the stream it was allocated on; a later request on the same
// stream takes the smallest parked block that holds it (and is at most about
// twice its size) before asking the pool. Reuse on the allocating stream is
// ordered exactly like cudaFreeAsync followed by a new allocation there. The
// round loop re-creates its buffers on every solve call, and a pool
// allocation costs the host tens to hundreds of microseconds, during which
// the GPU, just synchronized, waits.
// block_alloc returns the owner token of the allocating thread; block_free
// parks the block only on that thread (elsewhere it goes back to the pool).
void *block_alloc(size_t bytes, cudaStream_t s, size_t &cap, const void *&owner);
void block_free(void *p, size_t cap, cudaStream_t s, const void *owner);
// Returns this thread's parked blocks to the pool: waits for the device to
// be idle, then frees them (their streams may no longer exist). A thread that
// ends before the process calls it last.
void block_cache_flush();
// Turns parking off (flushing what is parked) or on for this thread. Server
// lanes turn it off: they keep their buffers across rounds, and blocks parked
// by one lane would be out of reach of the others under one memory budget.
void block_cache_enable(bool on);
void set_last_error(const std::string &msg);

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaStream_t s = nullptr;
  const void *owner = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) block_free(p, cap, s, owner);
    p = nullptr;
    cap = 0;
  }
  // Grows by a quarter more than asked (a sixteenth above 4 GB), so that a
  // buffer that grows round by round is seldom reallocated.
  void *ensure(size_t bytes, cudaStream_t st) {
    if (bytes <= cap && p) return p;
    release();
    s = st;
    const size_t slack = bytes > (size_t(4) << 30) ? bytes / 16 : bytes / 4;
    p = block_alloc(bytes + slack + 256, st, cap, owner);
    return p;
  }
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

}  // namespace sgn
