// The EXACT element threshold of sign_threshold_exact, for callers that cannot
// allocate device memory.
//
// Who needs it: a process that hands (nearly) all of the GPU's memory to its
// own pool at start-up, as serving systems often do, leaves nothing for a
// library's cudaMalloc, which then fails or competes with that pool; and a
// loop that must keep a steady cadence cannot afford cudaMalloc/cudaFree,
// which may synchronize the whole device. This entry point takes device
// values and keeps all of its scratch in one file-scope __device__ array, so
// it calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array (about 12 MiB) exists on every GPU that loads this library until
// the process exits. Its host-side name is only a stand-in: the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made while it is current. No call can
// be captured into a CUDA graph: each copies its small inputs and the result
// through host memory and waits for the stream. Every call reuses the same
// array, so calls that overlap on the GPU (other streams, other host threads
// on the same device) race and must be serialized by the caller.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/sign.h"
#include "common.cuh"
#include "kernels.h"

using namespace sgn;

namespace sgn {
void set_last_error(const std::string &msg);
}

namespace {

// Small per-call state at the front of the array, the select scratch after it.
struct NoAllocHead {
  int64_t eoff[2];
  int active[2];
  MatScalars ms;
};
constexpr size_t kHeadBytes = sel_align(sizeof(NoAllocHead));
constexpr size_t kScratchBytes = kHeadBytes + select_scratch_bytes(1, SIGN_NOALLOC_MAX_NNZ);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once).
void *scratch_address(std::string &why) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    why = "no usable current CUDA device";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

// Drops the current device's cached address, so that the next call looks it
// up again (a failed call may follow a reset of the device's context, after
// which the module and its array can sit elsewhere).
void forget_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_addr[dev] = nullptr;
}

}  // namespace

extern "C" sign_status sign_threshold_exact_noalloc(const double *val, int64_t nnz, double b,
                                                    void *cuda_stream, double *tau_out) {
  set_last_error("");
  if (!tau_out) return set_last_error("tau_out is NULL"), SIGN_EINVAL;
  if (nnz < 0 || (nnz > 0 && !val)) return set_last_error("need nnz >= 0 and values"), SIGN_EINVAL;
  if (nnz > SIGN_NOALLOC_MAX_NNZ)
    return set_last_error("nnz exceeds SIGN_NOALLOC_MAX_NNZ (" +
                          std::to_string(SIGN_NOALLOC_MAX_NNZ) +
                          "); use sign_threshold_exact"),
           SIGN_EINVAL;
  if (!(b >= 0.0) || !std::isfinite(b)) return set_last_error("budget must be finite and >= 0"), SIGN_EINVAL;
  std::string why;
  unsigned char *base = static_cast<unsigned char *>(scratch_address(why));
  if (!base) return set_last_error(why), SIGN_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    NoAllocHead h;
    std::memset(&h, 0, sizeof(h));
    h.eoff[1] = nnz;
    h.active[0] = 1;
    h.ms.b = b;
    h.ms.nnz_bar = nnz;
    NoAllocHead *d = reinterpret_cast<NoAllocHead *>(base);
    SGN_CUDA(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    // the select kernels clear their histograms and state themselves
    SelRows R{(nnz + kFlatRow - 1) / kFlatRow, nullptr, nullptr, nullptr, nnz};
    launch_select_exact(1, R, nnz, d->active, val, 0, &d->ms, base + kHeadBytes, nullptr, nullptr, s);
    SGN_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    *tau_out = h.ms.tau;
  } catch (const Error &e) {
    forget_address();  // after a CUDA error the next call looks the array up again
    set_last_error(e.what());
    return sign_status(e.status);
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return SIGN_ENOMEM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return SIGN_ECUDA;
  }
  return SIGN_OK;
}
