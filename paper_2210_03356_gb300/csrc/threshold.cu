// Standalone entry point of the EXACT element threshold (step a5) for one
// array of values, the same kernels the solver runs per matrix.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/sign.h"
#include "common.cuh"
#include "kernels.h"

using namespace sgn;

namespace sgn {
void set_last_error(const std::string &msg);
}

extern "C" sign_status sign_threshold_exact(const double *val, int64_t nnz, double b, int on_device,
                                            void *cuda_stream, double *tau_out) {
  set_last_error("");
  if (!tau_out) return set_last_error("tau_out is NULL"), SIGN_EINVAL;
  if (nnz < 0 || (nnz > 0 && !val)) return set_last_error("need nnz >= 0 and values"), SIGN_EINVAL;
  if (!(b >= 0.0) || !std::isfinite(b)) return set_last_error("budget must be finite and >= 0"), SIGN_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    DevBuf vals, small, scratch;
    const double *dval = val;
    if (!on_device && nnz > 0) {
      vals.ensure(sizeof(double) * size_t(nnz), s);
      SGN_CUDA(cudaMemcpyAsync(vals.p, val, sizeof(double) * size_t(nnz), cudaMemcpyHostToDevice, s));
      dval = vals.as<double>();
    }
    // eoff[2], active[1], ms[1] in one small buffer
    struct Small {
      int64_t eoff[2];
      int active[2];
      MatScalars ms;
    } hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.eoff[1] = nnz;
    hs.active[0] = 1;
    hs.ms.b = b;
    hs.ms.nnz_bar = nnz;
    small.ensure(sizeof(Small), s);
    SGN_CUDA(cudaMemcpyAsync(small.p, &hs, sizeof(Small), cudaMemcpyHostToDevice, s));
    Small *d = small.as<Small>();
    scratch.ensure(select_scratch_bytes(1, nnz), s);
    SelRows R{(nnz + kFlatRow - 1) / kFlatRow, nullptr, nullptr, nullptr, nnz};
    launch_select_exact(1, R, nnz, d->active, dval, 0, &d->ms, scratch.p, nullptr, nullptr, s);
    SGN_CUDA(cudaMemcpyAsync(&hs, small.p, sizeof(Small), cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    *tau_out = hs.ms.tau;
  } catch (const Error &e) {
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
