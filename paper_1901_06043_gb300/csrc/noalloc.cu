// tucker_gram_noalloc: the Gram step with its split-K scratch in a fixed
// device array instead of allocated memory, for callers that cannot call
// cudaMalloc (see the declaration in tucker_gb300.h).
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB of FP64 partial tiles
constexpr int kMaxDevices = 64;

// The scratch of every call on a device.  It lives in the module image, so
// each GPU that loads the library holds it until the process exits.
static __device__ __align__(256) double g_gram_scratch[kScratchBytes / sizeof(double)];

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

// Once per device, with that device current: the device address of the
// scratch array (its name is only a host-side stand-in in host code).
tucker_status setup_device(int dev) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_scratch_ptr[dev]) return TUCKER_OK;
  double* p = nullptr;
  if (cudaGetSymbolAddress((void**)&p, g_gram_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return TUCKER_ERR_CUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return TUCKER_ERR_CUDA;
  }
  g_num_sms[dev] = sms;
  g_scratch_ptr[dev] = p;
  return TUCKER_OK;
}

}  // namespace

extern "C" tucker_status tucker_gram_noalloc(const void* y_dev, tucker_dtype dtype, int ndim,
                                             const int64_t* dims, int mode, tucker_prec prec,
                                             double* S_dev, void* stream) {
  if (!y_dev || !S_dev || !dims || ndim < 1 || ndim > TUCKER_MAX_MODES || mode < 0 ||
      mode >= ndim || (dtype != TUCKER_F32 && dtype != TUCKER_F64))
    return TUCKER_ERR_INVALID;
  for (int k = 0; k < ndim; ++k)
    if (dims[k] < 1) return TUCKER_ERR_INVALID;
  if (prec != TUCKER_PREC_FP64 && prec != TUCKER_PREC_FP32) return TUCKER_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TUCKER_ERR_CUDA;
  }
  tucker_status s = setup_device(dev);
  if (s != TUCKER_OK) return s;
  const tk::SlabView v = tk::slab_view(ndim, dims, mode);
  int fits = 0;
  tk::GramPlan p =
      tk::plan_gram_simt_capped(v.L, v.I, v.Rt, g_num_sms[dev], kScratchBytes, &fits, v.L0);
  if (!fits) return TUCKER_ERR_INVALID;   // I_n above 1984: partial tiles exceed the scratch
  cudaError_t e = tk::launch_gram_simt(y_dev, dtype, prec == TUCKER_PREC_FP64, v.L, v.I, v.Rt, v.L0, p,
                                       g_scratch_ptr[dev], S_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TUCKER_ERR_CUDA;
  }
  return TUCKER_OK;
}
