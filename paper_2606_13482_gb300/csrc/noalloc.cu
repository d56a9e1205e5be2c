// Plane-wave right-hand sides without any device allocation.
//
// efie_rhs_planewave copies the caller's directions and polarisations into a
// small device buffer that it allocates and frees on every call.  Callers that
// must not allocate device memory once they are running -- code inside a
// memory-pool or no-allocation policy, real-time loops that cannot afford the
// implicit synchronisation of cudaMalloc/cudaFree, or hosts whose allocator is
// owned by another framework -- use efie_rhs_planewave_noalloc instead: it
// stages those inputs in the fixed array below, which every GPU that loads
// this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/efie.h"
#include "device_api.cuh"

namespace {

constexpr int kMaxPlaneWaves = 4096;  // 4096 x (3 + 3) doubles = 192 KiB

// [0, 3*max): directions, [3*max, 6*max): polarisations
static __device__ __align__(256) double g_pw_scratch[6 * kMaxPlaneWaves];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};
std::string g_err;

// Host code only sees a stand-in for g_pw_scratch; the real device address is
// looked up once per device, with that device current (the caller has checked
// that it is the handle's device).  The cached address stays valid until the
// device is reset (cudaDeviceReset unloads the module that holds the array).
cudaError_t scratch_for_device(int dev, double** out) {
  cudaError_t e = cudaSuccess;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pw_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

namespace efie {
// accessors implemented in api.cu (handle layout stays private there)
int handle_rhs_args(const efie_handle* h, const double** V, const int32_t** T, const double** area,
                    const int32_t** tri_pm, const int32_t** free_pm, int64_t* N, double* k, int* device);
void handle_set_error(efie_handle* h, const char* msg);
}  // namespace efie

extern "C" int efie_rhs_planewave_noalloc(efie_handle* h, int n_rhs, const double* khat, const double* pol,
                                          void* rhs, void* stream) {
  if (!h) return EFIE_EINVAL;
  if (n_rhs < 0 || n_rhs > kMaxPlaneWaves) {
    efie::handle_set_error(h, ("efie_rhs_planewave_noalloc: n_rhs must be in 0.." +
                               std::to_string(kMaxPlaneWaves) + " (fixed scratch size)").c_str());
    return EFIE_EINVAL;
  }
  if (n_rhs == 0) return EFIE_OK;
  if (!khat || !pol || !rhs) {
    efie::handle_set_error(h, "efie_rhs_planewave_noalloc: NULL argument");
    return EFIE_EINVAL;
  }
  const double *V, *area;
  const int32_t *T, *tri_pm, *free_pm;
  int64_t N;
  double k;
  int hdev = 0, cur = -1;
  if (efie::handle_rhs_args(h, &V, &T, &area, &tri_pm, &free_pm, &N, &k, &hdev) != EFIE_OK) return EFIE_EINVAL;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != hdev) {
    efie::handle_set_error(h, ("efie_rhs_planewave_noalloc: the current device (" + std::to_string(cur) +
                               ") is not the handle's device (" + std::to_string(hdev) + ")").c_str());
    return EFIE_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_device(hdev, &scratch);
  if (e != cudaSuccess) {
    efie::handle_set_error(h, (std::string("efie_rhs_planewave_noalloc: cudaGetSymbolAddress: ") +
                               cudaGetErrorString(e)).c_str());
    return EFIE_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every element the kernel reads is overwritten here, so nothing needs zeroing
  e = cudaMemcpyAsync(scratch, khat, sizeof(double) * 3 * n_rhs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scratch + 3 * kMaxPlaneWaves, pol, sizeof(double) * 3 * n_rhs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    efie::launch_rhs_planewave(V, T, area, tri_pm, free_pm, N, k, scratch, scratch + 3 * kMaxPlaneWaves, n_rhs,
                               (double2*)rhs, N, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host inputs may be released after return
  if (e != cudaSuccess) {
    efie::handle_set_error(h, (std::string("efie_rhs_planewave_noalloc: ") + cudaGetErrorString(e)).c_str());
    return EFIE_ECUDA;
  }
  return EFIE_OK;
}
